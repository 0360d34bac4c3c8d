"""Reference for the slab/tile binner (test infrastructure only).

The paper's streaming slicer keeps, per plane, the edges whose swept sphere of
radius R meets the plane (Eq. 8). The GPU build widens that set to a slab of
layers and splits it over square tiles of 16 or 32 pixels; which edges land in which tile
is a rule of the build, not of the paper. This module re-implements that rule
independently, in numpy float32 with the same operation order, so that the
GPU lists can be compared bit for bit, and gives the FP64 set of edges that
really contribute (distance < R) so that the lists can be checked to contain
every contributor.

Bin rule, for a slab with first and last layer planes zf <= zl (each rounded
from double to float) and an edge with exact endpoints (ax, ay, zlo) ->
(bx, by, zhi), zlo <= zhi, margin m (float):
  reject unless (zlo - m) <= zl and (zhi + m) >= zf;
  t0, t1 = 0, 1, or, when zhi - zlo > 0,
  t0 = max(((zf - m) - zlo) / (zhi - zlo), 0), t1 = min(((zl + m) - zlo) / (zhi - zlo), 1);
  x(t) = ax + t (bx - ax), y(t) likewise;
  box = [min(x(t0), x(t1)) - m, max(...) + m] x [same for y];
  tiles floor((box - float(x0)) * float(1 / (T pixel))) clipped to the grid, T the tile side;
  with a one-pixel halo (tiles that also evaluate their next column and row), the
  box's low corner is first lowered by float(pixel).
The margin is float(R + 8e-6 S + 1e-6), S the largest magnitude among the
node bounding box, the grid corners and the first and last layer planes (and
at least 1).
"""
from __future__ import annotations

import numpy as np

TILE = 16


def margin(nodes, R, *, x0, y0, nx, ny, pixel, z0, dz, n_layers):
    n = np.asarray(nodes, dtype=np.float32).reshape(-1, 3)
    s = 1.0
    if n.size:
        s = max(s, float(np.max(np.abs(n.min(axis=0).astype(np.float64)))),
                float(np.max(np.abs(n.max(axis=0).astype(np.float64)))))
    s = max(s, abs(x0), abs(y0), abs(x0 + nx * pixel), abs(y0 + ny * pixel), abs(z0),
            abs(z0 + max(n_layers - 1, 0) * dz))
    return np.float32(R + 8e-6 * s + 1e-6)


def bin_lists_fp32(nodes, edges, R, *, z0, dz, first_layer, n_slab_layers, x0, y0, nx, ny,
                   pixel, tile=TILE, halo=False):
    """Edge ids (ascending) per tile of the slab; returns (tile_off, ids)."""
    f32 = np.float32
    nodes = np.asarray(nodes, dtype=np.float32).reshape(-1, 3)
    edges = np.asarray(edges, dtype=np.int64).reshape(-1, 2)
    m = margin(nodes, R, x0=x0, y0=y0, nx=nx, ny=ny, pixel=pixel, z0=z0, dz=dz,
               n_layers=first_layer + n_slab_layers)
    ntx, nty = -(-nx // tile), -(-ny // tile)
    zf = f32(z0 + first_layer * dz)
    zl = f32(z0 + (first_layer + n_slab_layers - 1) * dz)
    fx0, fy0 = f32(x0), f32(y0)
    inv_tile = f32(1.0 / (tile * pixel))
    a = nodes[edges[:, 0]]
    b = nodes[edges[:, 1]]
    swap = b[:, 2] < a[:, 2]
    lo = np.where(swap[:, None], b, a)
    hi = np.where(swap[:, None], a, b)
    zlo, zhi = lo[:, 2], hi[:, 2]
    keep = ~((zlo - m) > zl) & ~((zhi + m) < zf)
    dzs = zhi - zlo
    t0 = np.zeros_like(dzs)
    t1 = np.ones_like(dzs)
    pos = dzs > 0
    with np.errstate(divide="ignore", invalid="ignore"):
        q0 = ((zf - m) - zlo) / np.where(pos, dzs, f32(1))
        q1 = ((zl + m) - zlo) / np.where(pos, dzs, f32(1))
    t0 = np.where(pos, np.maximum(q0, f32(0)), t0).astype(np.float32)
    t1 = np.where(pos, np.minimum(q1, f32(1)), t1).astype(np.float32)
    ex = hi[:, 0] - lo[:, 0]
    ey = hi[:, 1] - lo[:, 1]
    xa, xb = lo[:, 0] + t0 * ex, lo[:, 0] + t1 * ex
    ya, yb = lo[:, 1] + t0 * ey, lo[:, 1] + t1 * ey
    xmin, xmax = np.minimum(xa, xb) - m, np.maximum(xa, xb) + m
    ymin, ymax = np.minimum(ya, yb) - m, np.maximum(ya, yb) + m
    if halo:
        xmin = xmin - f32(pixel)
        ymin = ymin - f32(pixel)
    gx0 = np.floor((xmin - fx0) * inv_tile)
    gx1 = np.floor((xmax - fx0) * inv_tile)
    gy0 = np.floor((ymin - fy0) * inv_tile)
    gy1 = np.floor((ymax - fy0) * inv_tile)
    keep &= ~((gx1 < 0) | (gy1 < 0) | (gx0 >= ntx) | (gy0 >= nty))
    lists = [[] for _ in range(ntx * nty)]
    for e in np.nonzero(keep)[0]:
        tx0, tx1 = int(max(gx0[e], 0)), int(min(gx1[e], ntx - 1))
        ty0, ty1 = int(max(gy0[e], 0)), int(min(gy1[e], nty - 1))
        for ty in range(ty0, ty1 + 1):
            for tx in range(tx0, tx1 + 1):
                lists[ty * ntx + tx].append(int(e))
    off = np.zeros(len(lists) + 1, np.int64)
    off[1:] = np.cumsum([len(x) for x in lists])
    ids = np.array([e for x in lists for e in x], dtype=np.int64)
    return off, ids


def contributors_fp64(nodes, edges, R, pts):
    """Edge ids whose segment passes within distance < R of any point (FP64):
    exactly the edges with a nonzero Eq. 7 integral at one of the points."""
    nodes = np.asarray(nodes, dtype=np.float64).reshape(-1, 3)
    edges = np.asarray(edges, dtype=np.int64).reshape(-1, 2)
    pts = np.asarray(pts, dtype=np.float64).reshape(-1, 3)
    a = nodes[edges[:, 0]]
    d = nodes[edges[:, 1]] - a
    L2 = np.sum(d * d, axis=1)
    out = set()
    for i in range(0, pts.shape[0], 256):
        p = pts[i:i + 256]
        q = p[:, None, :] - a[None, :, :]
        with np.errstate(divide="ignore", invalid="ignore"):
            t = np.clip(np.sum(q * d[None], axis=2) / np.where(L2 > 0, L2, 1.0), 0.0, 1.0)
        c = q - t[:, :, None] * d[None]
        dist2 = np.sum(c * c, axis=2)
        hit = np.any(dist2 < R * R, axis=0) & (L2 > 0)
        out.update(np.nonzero(hit)[0].tolist())
    return out
