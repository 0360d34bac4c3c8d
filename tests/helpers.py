"""Shared helpers of the parity tests: field tolerance, contour comparison."""
from __future__ import annotations

import numpy as np

import oracle

FIELD_RTOL = 1e-5      # |Sigma_gpu - Sigma_ref| <= 1e-5 max(|Sigma_ref|, C)
BAND = 1e-5            # inside/outside must agree where |Sigma_ref - C| >= 1e-5 C
VERTEX_TOL_PX = 0.01   # contour vertices within 0.01 pixel


def field_error(sig_gpu, sig_ref, C):
    """max over pixels of |gpu - ref| / max(|ref|, C)."""
    sig_gpu = np.asarray(sig_gpu, dtype=np.float64)
    sig_ref = np.asarray(sig_ref, dtype=np.float64)
    return float(np.max(np.abs(sig_gpu - sig_ref) / np.maximum(np.abs(sig_ref), C)))


def assert_field(sig_gpu, sig_ref, C):
    err = field_error(sig_gpu, sig_ref, C)
    assert err <= FIELD_RTOL, f"field error {err:.3e} > {FIELD_RTOL}"
    # classification identical outside the band
    ref_in = sig_ref >= C
    gpu_in = np.asarray(sig_gpu) >= np.float32(C)
    clear = np.abs(sig_ref - C) >= BAND * C
    assert np.array_equal(ref_in[clear], gpu_in[clear])
    return err


def band_cells(sig_ref, C):
    """bool [ny+1, nx+1] over the padded cell grid: cells whose corner values
    (or, for a saddle, the mean of the corners) lie within the tolerance band."""
    ny, nx = sig_ref.shape
    P = np.zeros((ny + 2, nx + 2))
    P[1:-1, 1:-1] = sig_ref
    corners = [P[:-1, :-1], P[:-1, 1:], P[1:, 1:], P[1:, :-1]]
    near = np.zeros((ny + 1, nx + 1), bool)
    tol_c = BAND * C
    pad_mask = np.zeros((ny + 2, nx + 2), bool)
    pad_mask[1:-1, 1:-1] = True
    pm = [pad_mask[:-1, :-1], pad_mask[:-1, 1:], pad_mask[1:, 1:], pad_mask[1:, :-1]]
    for v, m in zip(corners, pm):
        near |= m & (np.abs(v - C) < tol_c)
    ins = [(v >= C) & m for v, m in zip(corners, pm)]
    saddle = (ins[0] & ins[2] & ~ins[1] & ~ins[3]) | (ins[1] & ins[3] & ~ins[0] & ~ins[2])
    mean = 0.25 * sum(corners)
    scale = np.maximum(np.max(np.abs(np.stack(corners)), axis=0), C)
    near |= saddle & (np.abs(mean - C) < FIELD_RTOL * scale * 2)
    return near


def _edge_cells(eids, nx):
    W = nx + 2
    e = np.asarray(eids, dtype=np.int64)
    s = e // 2
    I, J = s % W, s // W
    horiz = (e % 2) == 0
    # cells (I, J) and (I, J-1) for horizontal; (I, J) and (I-1, J) for vertical
    c1 = np.stack([I, J], 1)
    c2 = np.stack([np.where(horiz, I, I - 1), np.where(horiz, J - 1, J)], 1)
    return np.concatenate([c1, c2])


def compare_layer_contours(gpu_loops, sig_ref, *, x0, y0, pixel, C):
    """gpu_loops: list of (edge_id array, xy array) of one layer. Compares with
    the oracle's marching squares of the FP64 field. Returns (matched, excluded)."""
    ny, nx = sig_ref.shape
    off, eid, xy = oracle.marching_squares(sig_ref, x0=x0, y0=y0, pixel=pixel, C=C)
    band = band_cells(sig_ref, C)
    gpu_by_head = {}
    for e, p in gpu_loops:
        assert e[0] == e.min(), "GPU loop does not start at its smallest edge id"
        gpu_by_head[int(e[0])] = (e, p)
    heads = [int(e[0]) for e, _ in gpu_loops]
    assert heads == sorted(heads), "GPU loops not listed by head edge id"
    matched = excluded = 0
    ref_heads = set()
    for li in range(len(off) - 1):
        a, b = off[li], off[li + 1]
        le, lxy = eid[a:b], xy[a:b]
        cells = _edge_cells(le, nx)
        ok = (cells[:, 0] >= 0) & (cells[:, 1] >= 0) & (cells[:, 0] <= nx) & (cells[:, 1] <= ny)
        cells = cells[ok]
        if band[cells[:, 1], cells[:, 0]].any():
            excluded += 1
            continue
        ref_heads.add(int(le[0]))
        assert int(le[0]) in gpu_by_head, f"loop with head {le[0]} missing on the GPU"
        ge, gxy = gpu_by_head[int(le[0])]
        assert np.array_equal(ge, le), "loop topology differs"
        d = np.max(np.hypot(gxy[:, 0] - lxy[:, 0], gxy[:, 1] - lxy[:, 1])) / pixel
        assert d <= VERTEX_TOL_PX, f"vertex distance {d:.4f} px"
        matched += 1
    if excluded == 0:
        assert len(gpu_loops) == len(off) - 1, "GPU has extra loops"
    return matched, excluded


def oracle_contour_set(cfg, layers):
    """The oracle's marching-squares contours of the given layers of a
    configuration (its field in FP64, vertices rounded to float32), in the
    layout of csl_contours: (layer_loop_off, loop_vert_off, xy float32 [n, 2],
    edge_id int32). Post-processing stages take these as their input, so no
    oracle input comes from the GPU path."""
    lo, vo, xys, eids = [0], [0], [], []
    for k in layers:
        sig = oracle.slice_sigma(cfg["nodes"], cfg["edges"], cfg["radius"], R=cfg["R"],
                                 C=cfg["C"], z0=cfg["z0"] + k * cfg["dz"], dz=cfg["dz"],
                                 n_layers=1, x0=cfg["x0"], y0=cfg["y0"], nx=cfg["nx"],
                                 ny=cfg["ny"], pixel=cfg["pixel"])[0]
        off, eid, xy = oracle.marching_squares(sig, x0=cfg["x0"], y0=cfg["y0"],
                                               pixel=cfg["pixel"], C=cfg["C"])
        base = vo[-1]
        vo.extend(int(base + o) for o in off[1:])
        lo.append(lo[-1] + len(off) - 1)
        xys.append(np.asarray(xy, dtype=np.float32).reshape(-1, 2))
        eids.append(np.asarray(eid, dtype=np.int32))
    return (np.array(lo, np.int64), np.array(vo, np.int64),
            np.concatenate(xys) if xys else np.zeros((0, 2), np.float32),
            np.concatenate(eids) if eids else np.zeros(0, np.int32))


def layer_arrays(lo, vo, xy, eid, k):
    """One layer's (loop_off from 0, edge ids, xy) out of a contour set."""
    l0, l1 = int(lo[k]), int(lo[k + 1])
    v0, v1 = int(vo[l0]), int(vo[l1])
    return vo[l0:l1 + 1] - v0, eid[v0:v1], xy[v0:v1]
