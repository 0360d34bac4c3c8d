"""Lattice generators and the five workload configurations.

Every function returns (nodes float32 [Nn, 3] in mm, edges int32 [Ne, 2],
radius float32 [Ne] in mm), plus whatever slicing parameters the
configuration fixes.
"""
from __future__ import annotations

import math

import numpy as np

SEED_BASE = 2101050310

# Freudenthal (Kuhn) cube split: from each grid node the edges +x, +y, +z, the
# three face diagonals (1,1,0), (1,0,1), (0,1,1) and the body diagonal (1,1,1).
FREUDENTHAL_DIRS = np.array([[1, 0, 0], [0, 1, 0], [0, 0, 1],
                             [1, 1, 0], [1, 0, 1], [0, 1, 1], [1, 1, 1]], dtype=np.int64)
# Strut length per unit cell volume of a Freudenthal grid of unit spacing.
FREUDENTHAL_LENGTH_DENSITY = 3.0 + 3.0 * math.sqrt(2.0) + math.sqrt(3.0)


def rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.Philox(int(seed)))


def lattice_bbox(nodes):
    n = np.asarray(nodes, dtype=np.float64)
    return n.min(axis=0), n.max(axis=0)


# --------------------------------------------------------------------------
# Regular cubic + BCC lattice (configuration 1)
# --------------------------------------------------------------------------

def cubic_bcc(n_cells: int = 4, cell: float = 5.0, rho: float = 0.5):
    """Cube edges of an n^3 grid of cells plus struts from every body centre
    to its 8 corners. 4^3 cells give 300 + 512 = 812 struts."""
    n = int(n_cells)
    g = np.arange(n + 1)
    I, J, K = np.meshgrid(g, g, g, indexing="ij")
    corners = np.stack([I.ravel(), J.ravel(), K.ravel()], axis=1)

    def cid(i, j, k):
        return (i * (n + 1) + j) * (n + 1) + k

    c = np.arange(n)
    ci, cj, ck = np.meshgrid(c, c, c, indexing="ij")
    ci, cj, ck = ci.ravel(), cj.ravel(), ck.ravel()
    centres = np.stack([ci + 0.5, cj + 0.5, ck + 0.5], axis=1)
    n_corner = corners.shape[0]
    nodes = np.concatenate([corners.astype(np.float64), centres]) * cell

    edges = []
    for d in ((1, 0, 0), (0, 1, 0), (0, 0, 1)):
        m = (I + d[0] <= n) & (J + d[1] <= n) & (K + d[2] <= n)
        a = cid(I[m], J[m], K[m])
        b = cid(I[m] + d[0], J[m] + d[1], K[m] + d[2])
        edges.append(np.stack([a, b], axis=1))
    centre_id = n_corner + np.arange(ci.shape[0])
    for dx in (0, 1):
        for dy in (0, 1):
            for dz in (0, 1):
                b = cid(ci + dx, cj + dy, ck + dz)
                edges.append(np.stack([centre_id, b], axis=1))
    edges = np.concatenate(edges).astype(np.int32)
    radius = np.full(edges.shape[0], rho, dtype=np.float32)
    return nodes.astype(np.float32), edges, radius


# --------------------------------------------------------------------------
# Jittered Freudenthal lattice (configurations 2, 4 and 5)
# --------------------------------------------------------------------------

def freudenthal(n, spacing=1.0, jitter=0.2, rho_range=(0.15, 0.35), seed=SEED_BASE + 2,
                origin=(0.0, 0.0, 0.0)):
    """Nodes on an (nx, ny, nz) grid of the given spacing, each coordinate
    jittered by U(-jitter, +jitter); Freudenthal edges; radii U(rho_range).
    n may be an int (cube) or a 3-tuple. 40^3 nodes give 429,039 struts."""
    if np.isscalar(n):
        n = (int(n),) * 3
    nx, ny, nz = (int(v) for v in n)
    r = rng(seed)
    I, J, K = np.meshgrid(np.arange(nx), np.arange(ny), np.arange(nz), indexing="ij")
    base = np.stack([I.ravel(), J.ravel(), K.ravel()], axis=1).astype(np.float64) * spacing
    base += np.asarray(origin, dtype=np.float64)
    nodes = base + r.uniform(-jitter, jitter, size=base.shape)

    def nid(i, j, k):
        return (i * ny + j) * nz + k

    edges = []
    for d in FREUDENTHAL_DIRS:
        m = (I + d[0] < nx) & (J + d[1] < ny) & (K + d[2] < nz)
        a = nid(I[m], J[m], K[m])
        b = nid(I[m] + d[0], J[m] + d[1], K[m] + d[2])
        edges.append(np.stack([a, b], axis=1))
    edges = np.concatenate(edges).astype(np.int32)
    radius = r.uniform(rho_range[0], rho_range[1], size=edges.shape[0]).astype(np.float32)
    return nodes.astype(np.float32), edges, radius


# --------------------------------------------------------------------------
# Adaptive graded lattice (configuration 3)
# --------------------------------------------------------------------------

def graded_density(x, y):
    """Target density rho(x) = 0.1 + 0.3 (0.5 + 0.5 sin(2 pi x/50) cos(2 pi y/50))."""
    return 0.1 + 0.3 * (0.5 + 0.5 * np.sin(2 * np.pi * x / 50.0) * np.cos(2 * np.pi * y / 50.0))


def _density_estimate(h, r_ref):
    # volume fraction of a Freudenthal grid of spacing h with struts of radius r_ref
    return FREUDENTHAL_LENGTH_DENSITY / (h * h) * math.pi * r_ref * r_ref


def adaptive_graded(box=200.0, level_min=5, level_max=8, threshold=0.165, r_min_frac=0.25):
    """Octree-graded Freudenthal lattice on [0, box]^3.

    A cube of edge h at level l < level_max is split into 8 while the density
    of a Freudenthal grid of spacing h with struts of radius r_ref is below the
    target density at the cube's centre. r_ref is set so that a grid one level
    coarser than level_max reaches ``threshold``; at the defaults this gives
    about 100M struts with levels 7 and 8 (h = 1.5625 and 0.78125 mm). Leaf cubes emit their
    Freudenthal edges; identical edges are kept once, and edges of different
    levels that meet at hanging nodes are all kept. Each strut's radius is
    set from the target density at its midpoint, r = sqrt(rho / (lambda pi))
    with lambda the strut length per volume of its level, clamped to
    [r_min_frac r_ref, r_ref]. Deterministic (no random numbers).
    Returns nodes, edges, radius and r_ref.
    """
    h_ref = box / 2 ** (level_max - 1)
    r_ref = h_ref * math.sqrt(threshold / (FREUDENTHAL_LENGTH_DENSITY * math.pi))
    # leaf[l]: bool [2^l]^3, True where the cube at level l is a leaf
    leaf = {}
    active = np.ones((2 ** level_min,) * 3, dtype=bool)    # cubes that exist at this level
    for lev in range(level_min, level_max + 1):
        n = 2 ** lev
        h = box / n
        if lev == level_max:
            leaf[lev] = active
            break
        c = (np.arange(n) + 0.5) * h
        rho2d = graded_density(c[:, None], c[None, :])       # depends on x, y only
        refine2d = _density_estimate(h, r_ref) < rho2d
        refine = active & refine2d[:, :, None]
        leaf[lev] = active & ~refine
        active = np.repeat(np.repeat(np.repeat(refine, 2, 0), 2, 1), 2, 2)

    nf = 2 ** level_max + 1
    node_map = np.full(nf ** 3, -1, dtype=np.int64)
    per_level_edges = []
    for lev in range(level_min, level_max + 1):
        lf = leaf[lev]
        if not lf.any():
            continue
        n = 2 ** lev
        L = np.zeros((n + 2,) * 3, dtype=bool)                 # leaf flags padded by 1 (offset +1)
        L[1:-1, 1:-1, 1:-1] = lf
        scale = 2 ** (level_max - lev)
        for d in FREUDENTHAL_DIRS:
            # cubes (by min corner) that contain the edge from node (i,j,k) along d
            if d.sum() == 3:
                cubes = [(0, 0, 0)]
            elif d.sum() == 2:
                zero = int(np.where(d == 0)[0][0])
                o = [0, 0, 0]
                o2 = [0, 0, 0]
                o2[zero] = -1
                cubes = [tuple(o), tuple(o2)]
            else:
                ax = int(np.where(d == 1)[0][0])
                others = [a for a in range(3) if a != ax]
                cubes = []
                for s0 in (0, -1):
                    for s1 in (0, -1):
                        o = [0, 0, 0]
                        o[others[0]] = s0
                        o[others[1]] = s1
                        cubes.append(tuple(o))
            m = np.zeros((n + 1,) * 3, dtype=bool)             # over nodes 0..n
            for o in cubes:
                m |= L[1 + o[0]:n + 2 + o[0], 1 + o[1]:n + 2 + o[1], 1 + o[2]:n + 2 + o[2]]
            hi = n + 1 - d                                     # node + d must stay on the grid
            m = m[:hi[0], :hi[1], :hi[2]]
            idx = np.nonzero(m)
            del m
            a = ((idx[0] * scale) * nf + idx[1] * scale) * nf + idx[2] * scale
            b = (((idx[0] + d[0]) * scale) * nf + (idx[1] + d[1]) * scale) * nf + \
                (idx[2] + d[2]) * scale
            del idx
            node_map[a] = 0
            node_map[b] = 0
            per_level_edges.append((lev, a, b))
    used = node_map >= 0
    node_map[used] = np.arange(int(used.sum()))
    fid = np.nonzero(used)[0]
    hf = box / (nf - 1)
    nodes = np.empty((fid.shape[0], 3), dtype=np.float32)
    nodes[:, 0] = (fid // (nf * nf)) * hf
    nodes[:, 1] = ((fid // nf) % nf) * hf
    nodes[:, 2] = (fid % nf) * hf
    del fid, used
    n_edges = sum(e[1].shape[0] for e in per_level_edges)
    edges = np.empty((n_edges, 2), dtype=np.int32)
    radius = np.empty(n_edges, dtype=np.float32)
    pos = 0
    for lev, a, b in per_level_edges:
        k = a.shape[0]
        edges[pos:pos + k, 0] = node_map[a]
        edges[pos:pos + k, 1] = node_map[b]
        h = box / 2 ** lev
        lam_pi = FREUDENTHAL_LENGTH_DENSITY / (h * h) * math.pi
        mid_x = 0.5 * (nodes[edges[pos:pos + k, 0], 0].astype(np.float64)
                       + nodes[edges[pos:pos + k, 1], 0])
        mid_y = 0.5 * (nodes[edges[pos:pos + k, 0], 1].astype(np.float64)
                       + nodes[edges[pos:pos + k, 1], 1])
        r = np.sqrt(graded_density(mid_x, mid_y) / lam_pi)
        radius[pos:pos + k] = np.clip(r, r_min_frac * r_ref, r_ref)
        pos += k
    return nodes, edges, radius, r_ref


# --------------------------------------------------------------------------
# Batched set (configuration 4)
# --------------------------------------------------------------------------

def batched_set(n_lattices=64, ne_range=(1e3, 5e5), extent_range=(10.0, 80.0),
                rho_range=(0.1, 0.5), seed=SEED_BASE + 4):
    """Independent jittered Freudenthal lattices of uneven size: strut count
    log-uniform in ne_range, box extents U(extent_range) per axis, grid spacing
    chosen so the Freudenthal count hits the drawn strut count, jitter of 0.2
    spacing, radii U(rho_range) (clamped below 0.45 spacing)."""
    r = rng(seed)
    out = []
    for i in range(n_lattices):
        ne = math.exp(r.uniform(math.log(ne_range[0]), math.log(ne_range[1])))
        ext = r.uniform(extent_range[0], extent_range[1], size=3)
        # about 7 struts per grid node: solve for spacing s with prod(ext/s) * 7 = ne
        s = (7.0 * float(np.prod(ext)) / ne) ** (1.0 / 3.0)
        n = tuple(max(2, int(round(e / s)) + 1) for e in ext)
        lo = min(rho_range[1], 0.45 * s)
        rr = (min(rho_range[0], 0.5 * lo), lo)
        lat = freudenthal(n, spacing=s, jitter=0.2 * s, rho_range=rr,
                          seed=SEED_BASE + 4 * 1000 + i)
        out.append(lat)
    return out


# --------------------------------------------------------------------------
# The five configurations
# --------------------------------------------------------------------------

def config(index: int, small: bool = False):
    """Inputs and slicing parameters of configuration 1..5.

    Returns a dict with nodes, edges, radius, R, C, and slicing or cell
    parameters. ``small`` shrinks configurations 2-5 to a size the FP64
    oracle finishes in seconds (same recipe, fewer nodes / layers / pixels).
    """
    if index == 1:
        nodes, edges, radius = cubic_bcc(4, 5.0, 0.5)
        return dict(name="cubic+bcc 4^3 cells, 812 struts, 200x200 px x 50 layers",
                    nodes=nodes, edges=edges, radius=radius, R=0.75, C=1.0,
                    x0=0.0, y0=0.0, nx=200, ny=200, pixel=0.1,
                    z0=0.2, dz=0.4, n_layers=50)
    if index == 2:
        n = 10 if small else 40
        nodes, edges, radius = freudenthal(n, 1.0, 0.2, (0.15, 0.35), seed=SEED_BASE + 2)
        lo, hi = lattice_bbox(nodes)
        npx = 300 if small else 2000
        px = 0.02 if not small else 0.04
        cx, cy = 0.5 * (lo[0] + hi[0]), 0.5 * (lo[1] + hi[1])
        nl = 8 if small else 200
        dz = 0.2
        z0 = float(lo[2]) + dz / 2
        return dict(name=f"jittered Freudenthal {n}^3 nodes, {edges.shape[0]} struts, "
                         f"{npx}^2 px x {nl} layers",
                    nodes=nodes, edges=edges, radius=radius, R=0.525, C=1.0,
                    x0=cx - npx * px / 2, y0=cy - npx * px / 2, nx=npx, ny=npx, pixel=px,
                    z0=z0, dz=dz, n_layers=nl)
    if index == 3:
        if small:
            nodes, edges, radius, r_ref = adaptive_graded(box=12.5, level_min=1, level_max=4)
            px, npx, nl, dz = 0.05, 250, 4, 0.2
        else:
            nodes, edges, radius, r_ref = adaptive_graded()
            px, npx, nl, dz = 0.05, 4000, 1000, 0.2
        return dict(name=f"adaptive graded lattice, {edges.shape[0]} struts, "
                         f"{npx}^2 px x {nl} layers",
                    nodes=nodes, edges=edges, radius=radius, R=1.5 * r_ref, C=1.0,
                    x0=0.0, y0=0.0, nx=npx, ny=npx, pixel=px, z0=dz / 2, dz=dz, n_layers=nl)
    if index == 4:
        lats = batched_set(8 if small else 64, ne_range=(1e3, 2e4) if small else (1e3, 5e5))
        jobs = []
        for nodes, edges, radius in lats:
            lo, hi = lattice_bbox(nodes)
            px = 0.05 if not small else 0.1
            pad = 0.75
            nx = int(math.ceil((hi[0] - lo[0] + 2 * pad) / px))
            ny = int(math.ceil((hi[1] - lo[1] + 2 * pad) / px))
            nl = 100 if not small else 4
            dz = (hi[2] - lo[2]) / nl
            jobs.append(dict(nodes=nodes, edges=edges, radius=radius, R=0.75, C=1.0,
                             x0=float(lo[0]) - pad, y0=float(lo[1]) - pad, nx=nx, ny=ny,
                             pixel=px, z0=float(lo[2]) + dz / 2, dz=float(dz), n_layers=nl))
        return dict(name=f"{len(jobs)} Freudenthal lattices, batched", jobs=jobs)
    if index == 5:
        n = 9 if small else 53
        nodes, edges, radius = freudenthal(n, 1.0, 0.2, (0.15, 0.35), seed=SEED_BASE + 5)
        lo, hi = lattice_bbox(nodes)
        dims = 8 if small else 64
        h = float(np.max(hi - lo)) / dims
        return dict(name=f"jittered Freudenthal {n}^3 nodes, {edges.shape[0]} struts, "
                         f"{dims}^3 cells x 8^3 samples",
                    nodes=nodes, edges=edges, radius=radius, R=0.525, C=1.0,
                    cells=dict(origin=(float(lo[0]), float(lo[1]), float(lo[2])), h=h,
                               dims=(dims, dims, dims), m=8, T=0.01))
    raise ValueError(f"unknown configuration {index}")
