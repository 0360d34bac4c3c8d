"""Lattice design steps on tetrahedral meshes: density matching
(csl_density_match, Sec. 5.5) and vertex re-positioning for self-support
(csl_support_optimize, Sec. 5.3.2). Argument marshalling only; the work runs
in libcslice.so."""
from __future__ import annotations

import ctypes
import math

import numpy as np

from . import _lib
from .slicer import _stream_ptr


def density_match(nodes, tets, grid, *, r_min: float, R: float = 0.0, C: float = 1.0,
                  temperature: float = 0.01, tet_n: int = 8, vox_m: int = 8, max_depth: int = 3,
                  iters: int = 24, stream=None) -> dict:
    """nodes float32 [N, 3], tets int32 [T, 4] (host); grid: dict with origin
    (3,), h, dims (nx, ny, nz) and target float32 [nz, ny, nx]. R = 0 takes
    1.5 x the doubled base radius (6 r_min). Returns numpy arrays: nodes,
    edges, radius, step3_ratio, tets, depth, target, rho_star, tet_ratio,
    voxel_ratio [nz, ny, nx], n_subdivided, host_ms and wall_ms."""
    nodes = np.ascontiguousarray(nodes, dtype=np.float32).reshape(-1, 3)
    tets = np.ascontiguousarray(tets, dtype=np.int32).reshape(-1, 4)
    dims = tuple(int(v) for v in grid["dims"])
    target = np.ascontiguousarray(grid["target"], dtype=np.float32)
    if target.shape != (dims[2], dims[1], dims[0]):
        raise ValueError("target must be [nz, ny, nx]")
    vox = _lib.Voxels((ctypes.c_double * 3)(*[float(v) for v in grid["origin"]]),
                      float(grid["h"]), (ctypes.c_int32 * 3)(*dims),
                      target.ctypes.data_as(ctypes.c_void_p))
    prm = _lib.DmParams(float(r_min), float(R), float(C), float(temperature), int(tet_n),
                        int(vox_m), int(max_depth), int(iters))
    lib = _lib.load()
    out = ctypes.POINTER(_lib.DmResult)()
    _lib.check(lib.csl_density_match(nodes.ctypes.data_as(ctypes.c_void_p), nodes.shape[0],
                                     tets.ctypes.data_as(ctypes.c_void_p), tets.shape[0],
                                     ctypes.byref(vox), ctypes.byref(prm), _stream_ptr(stream),
                                     ctypes.byref(out)))
    try:
        r = out.contents

        def arr(ptr, ctype, n, shape=None):
            if n == 0:
                a = np.zeros(0, dtype=np.dtype(ctype))
            else:
                a = np.ctypeslib.as_array(ctypes.cast(ptr, ctypes.POINTER(ctype)), shape=(n,)).copy()
            return a.reshape(shape) if shape is not None else a

        f32, i32, f64 = ctypes.c_float, ctypes.c_int32, ctypes.c_double
        return dict(
            nodes=arr(r.nodes, f32, 3 * r.n_nodes, (-1, 3)),
            edges=arr(r.edges, i32, 2 * r.n_edges, (-1, 2)),
            radius=arr(r.radius, f32, r.n_edges),
            step3_ratio=arr(r.step3_ratio, f32, r.n_edges),
            tets=arr(r.tets, i32, 4 * r.n_tets, (-1, 4)),
            depth=arr(r.tet_depth, i32, r.n_tets),
            target=arr(r.tet_target, f64, r.n_tets),
            rho_star=arr(r.tet_rho_star, f32, r.n_tets),
            tet_ratio=arr(r.tet_ratio, f32, r.n_tets),
            voxel_ratio=arr(r.voxel_ratio, f32, r.n_voxels, (dims[2], dims[1], dims[0])),
            n_subdivided=int(r.n_subdivided), host_ms=float(r.host_ms),
            wall_ms=float(r.wall_ms))
    finally:
        lib.csl_dm_result_free(out)


PAPER_A = (-0.02, -0.31, 1.44, -1.11, 0.58, -0.16)   # Eq. 12 for alpha = pi / 4


def support_optimize(nodes, tets, radius=None, *, t_p=(0.0, 0.0, 1.0), alpha=math.pi / 4,
                     coeffs=PAPER_A, step=0.25, ball=0.5, min_volume=0.1, backtracks=8,
                     max_rounds=100, stream=None) -> dict:
    """Vertex re-positioning (Eq. 16-17). nodes float32 [N, 3], tets int32
    [T, 4] (host); radius: float per distinct edge in (smaller, larger) order,
    or None. Returns nodes (new float32 array), rounds, moves_per_round,
    n_colours and Gamma / Psi before and after."""
    x = np.array(nodes, dtype=np.float32, copy=True).reshape(-1, 3)
    tets = np.ascontiguousarray(tets, dtype=np.int32).reshape(-1, 4)
    r = None if radius is None else np.ascontiguousarray(radius, dtype=np.float32)
    prm = _lib.PoParams((ctypes.c_double * 3)(*[float(v) for v in t_p]), float(alpha),
                        (ctypes.c_double * 6)(*[float(v) for v in coeffs]), float(step),
                        float(ball), float(min_volume), int(backtracks), int(max_rounds))
    per_round = np.zeros(max(int(max_rounds), 1), dtype=np.int32)
    res = _lib.PoResult()
    _lib.check(_lib.load().csl_support_optimize(
        x.ctypes.data_as(ctypes.c_void_p), x.shape[0], tets.ctypes.data_as(ctypes.c_void_p),
        tets.shape[0], r.ctypes.data_as(ctypes.c_void_p) if r is not None else None,
        ctypes.byref(prm), _stream_ptr(stream), ctypes.byref(res),
        per_round.ctypes.data_as(ctypes.c_void_p)))
    return dict(nodes=x, rounds=int(res.rounds), moves_per_round=per_round[:res.rounds].tolist(),
                moves=int(res.moves), n_colours=int(res.n_colours),
                gamma_before=res.gamma_before, psi_before=res.psi_before,
                gamma_after=res.gamma_after, psi_after=res.psi_after, host_ms=res.host_ms,
                wall_ms=res.wall_ms)
