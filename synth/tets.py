"""Seeded tetrahedral meshes and voxel density targets for density matching.

The paper builds its lattices from TetGen meshes of its models and voxel
densities given by the designer; neither is available, so a jittered
Kuhn/Freudenthal tetrahedral mesh of a box (six tetrahedra per cube around
the cube's main diagonal) and a smooth graded target on a voxel grid stand in
for them. No arithmetic of the method lives here.
"""
from __future__ import annotations

import itertools

import numpy as np

from .lattices import SEED_BASE, graded_density, rng


def kuhn_tet_mesh(n_cells, spacing: float, jitter: float = 0.1, seed: int = SEED_BASE + 6,
                  origin=(0.0, 0.0, 0.0)):
    """Nodes (float32 [N, 3]) and tetrahedra (int32 [T, 4]) of a box of
    n_cells = (cx, cy, cz) cubes of edge `spacing`, each cut into the six
    tetrahedra (c, c + e_a, c + e_a + e_b, c + 1) over the permutations
    (a, b, c) of the axes; interior nodes jittered by U(+-jitter * spacing)."""
    cx, cy, cz = (int(v) for v in n_cells)
    gx, gy, gz = np.meshgrid(np.arange(cx + 1), np.arange(cy + 1), np.arange(cz + 1),
                             indexing="ij")
    ijk = np.stack([gx.ravel(), gy.ravel(), gz.ravel()], axis=1)
    pos = ijk * float(spacing) + np.asarray(origin, dtype=np.float64)
    inner = ((ijk > 0) & (ijk < np.array([cx, cy, cz]))).all(1)
    r = rng(seed)
    pos[inner] += r.uniform(-jitter, jitter, size=(int(inner.sum()), 3)) * spacing

    def nid(i, j, k):
        return (i * (cy + 1) + j) * (cz + 1) + k

    tets = []
    for i, j, k in itertools.product(range(cx), range(cy), range(cz)):
        for perm in itertools.permutations(range(3)):
            c = [i, j, k]
            verts = [nid(*c)]
            for ax in perm:
                c[ax] += 1
                verts.append(nid(*c))
            tets.append(verts)
    return pos.astype(np.float32), np.array(tets, dtype=np.int32)


def graded_target_grid(lo, hi, h: float, scale=(0.05, 0.35), period: float = 50.0):
    """Voxels of edge h covering [lo, hi]; target density at each voxel centre
    from the graded field of the adaptive lattice (its period stretched to
    `period` mm), mapped affinely from its range [0.1, 0.4] onto `scale`."""
    lo = np.asarray(lo, dtype=np.float64)
    hi = np.asarray(hi, dtype=np.float64)
    dims = np.maximum(1, np.ceil((hi - lo) / h - 1e-9).astype(int))
    xs = lo[0] + h * (np.arange(dims[0]) + 0.5)
    ys = lo[1] + h * (np.arange(dims[1]) + 0.5)
    f = 50.0 / period
    g = graded_density(f * xs[None, :], f * ys[:, None])    # [ny, nx]
    t = scale[0] + (g - 0.1) / 0.3 * (scale[1] - scale[0])
    target = np.broadcast_to(t[None], (dims[2], dims[1], dims[0])).astype(np.float32).copy()
    # a gentle z ramp so that no two layers of voxels are alike
    ramp = 1.0 + 0.2 * (np.arange(dims[2]) + 0.5) / dims[2]
    target *= ramp[:, None, None].astype(np.float32)
    return dict(origin=(float(lo[0]), float(lo[1]), float(lo[2])), h=float(h),
                dims=(int(dims[0]), int(dims[1]), int(dims[2])), target=target)


def density_config(small: bool = False):
    """Density-matching workload. Full: a 100 mm box of 4 mm cubes (25^3 x 6 =
    93,750 tetrahedra) with 5 mm voxels (20^3), the designer's grid coarser
    than the lattice; small: 2^3 cubes (48 tetrahedra) with 3^3 voxels.
    r_min = 0.1 mm (base radius 0.2 mm)."""
    if small:
        nodes, tets = kuhn_tet_mesh((2, 2, 2), 4.0, 0.1, seed=SEED_BASE + 6)
        grid = graded_target_grid((0.0, 0.0, 0.0), (8.0, 8.0, 8.0), 8.0 / 3.0,
                                  scale=(0.03, 0.9), period=8.0)
        return dict(name="Kuhn tetrahedral mesh 2^3 cubes of 4 mm (48 tetrahedra), 3^3 voxels",
                    nodes=nodes, tets=tets, grid=grid, r_min=0.1, tet_n=4, vox_m=4,
                    max_depth=2, iters=24)
    nodes, tets = kuhn_tet_mesh((25, 25, 25), 4.0, 0.1, seed=SEED_BASE + 6)
    grid = graded_target_grid((0.0, 0.0, 0.0), (100.0, 100.0, 100.0), 5.0)
    return dict(name="Kuhn tetrahedral mesh 25^3 cubes of 4 mm (93,750 tetrahedra), "
                     "20^3 voxels of 5 mm",
                nodes=nodes, tets=tets, grid=grid, r_min=0.1, tet_n=8, vox_m=8, max_depth=3,
                iters=24)
