"""Density matching of a tetrahedral lattice (Sec. 5.5, the four steps and the
two operators: 1:8 subdivision and radius tuning).

TEST INFRASTRUCTURE ONLY: used by the tests and by bench.py's CPU legs, never
by the product package. Plain numpy in double precision; every step follows
the paper's order: (1) target density per tetrahedron, (2) recursive
subdivision while the doubled-radius density stays below the target, (3)
bisection of the radius per tetrahedron, (4) the per-voxel common ratio with
the smaller ratio kept on every edge.

Readings of the passages the paper leaves open:
  D1 base radius r0 = 2 r_min on every edge; a ratio s scales it, s in
     [1/2, 2] (r_min up to the doubled radius). R = 1.5 x the doubled radius
     unless given.
  D2 the density of a tetrahedron is the mean of the smoothed indicator
     sigma((Sigma - C) / T), T = temperature * C, at the centroids of the n^3
     equal-volume sub-tetrahedra of the n-fold Kuhn subdivision of the
     reference simplex, mapped affinely; Sigma comes from the struts of the
     tetrahedron's own six edges.
  D3 a voxel centre is contained by a tetrahedron when it lies in the closed
     tetrahedron, decided by the signs of four FP64 determinants.
  D4 without a contained centre, the target is the trilinear interpolation of
     the voxel-centre values at the tetrahedron's centroid (clamped).
  D5 subdivision cuts every edge at its midpoint rounded to float32 and the
     inner octahedron along its shortest diagonal (the first on ties); an edge
     split by a neighbour is replaced by its two halves everywhere.
  D6 radius tuning bisects the ratio for every leaf tetrahedron (amplifying
     below the target, reducing above it, bounded by r_min); an edge takes the
     smallest ratio of the leaf tetrahedra containing it.
  D7 the voxel check evaluates the voxel's density with all struts: those
     meeting the voxel at the common ratio, the others at their step-3 ratios;
     every voxel sees the step-3 ratios and the smaller ratios are applied
     after all voxels.
"""
from __future__ import annotations

import itertools

import numpy as np
from scipy.special import expit

LOCAL_EDGES = ((0, 1), (0, 2), (0, 3), (1, 2), (1, 3), (2, 3))


# ---------------------------------------------------------------- sampling
def kuhn_coefficients(n: int) -> np.ndarray:
    """(n^3, 3) coefficients (a1, a2, a3) of the centroids of the n-fold Kuhn
    subdivision of {1 >= x1 >= x2 >= x3 >= 0}. The point of tetrahedron
    (v0, v1, v2, v3) is v0 + a1 (v1 - v0) + a2 (v2 - v1) + a3 (v3 - v2): the
    affine map sending the simplex's corners (0,0,0), (1,0,0), (1,1,0),
    (1,1,1) to v0..v3, so equal volumes stay equal (reading D2)."""
    pts = []
    for perm in itertools.permutations(range(3)):
        for cell in itertools.product(range(n), repeat=3):
            x = np.array(cell, dtype=np.float64)
            x[perm[0]] += 0.75
            x[perm[1]] += 0.5
            x[perm[2]] += 0.25
            if x[0] > x[1] > x[2]:
                pts.append(x / n)
    a = np.array(pts, dtype=np.float64).reshape(-1, 3)
    assert a.shape[0] == n ** 3
    return a


def tet_points(v: np.ndarray, a: np.ndarray) -> np.ndarray:
    v = np.asarray(v, dtype=np.float64)
    return (v[0] + a[:, :1] * (v[1] - v[0]) + a[:, 1:2] * (v[2] - v[1])
            + a[:, 2:3] * (v[3] - v[2]))


def voxel_points(grid, i, j, k, m: int) -> np.ndarray:
    """m^3 stratified samples of voxel (i, j, k): o + h (c + (q + 1/2) / m)."""
    o = np.asarray(grid["origin"], dtype=np.float64)
    h = float(grid["h"])
    q = (np.arange(m) + 0.5) / m
    qz, qy, qx = np.meshgrid(q, q, q, indexing="ij")
    rel = np.stack([qx.ravel(), qy.ravel(), qz.ravel()], axis=1)
    return o + h * (np.array([i, j, k], dtype=np.float64) + rel)


# ---------------------------------------------------------------- the field
def seg_R4I(p, a, b, R: float) -> np.ndarray:
    """R^4 I_j(p) for struts a_j -> b_j: the integral along the edge (arc
    length) of (R^2 - |p - x|^2)_+^2, i.e. Eq. 7 times the chord length, in
    the centred form of Eq. 6 (tau measured from the foot of p). p: (P, 3);
    a, b: (E, 3). Returns (P, E)."""
    p = np.asarray(p, dtype=np.float64).reshape(-1, 3)
    a = np.asarray(a, dtype=np.float64).reshape(-1, 3)
    b = np.asarray(b, dtype=np.float64).reshape(-1, 3)
    d = b - a
    L = np.sqrt((d * d).sum(1))
    u = np.where(L[:, None] > 0, d / np.where(L > 0, L, 1.0)[:, None], 0.0)
    q = p[:, None, :] - a[None, :, :]
    t0 = (q * u[None]).sum(-1)
    e = q - t0[..., None] * u[None]
    h2 = R * R - (e * e).sum(-1)
    w = np.sqrt(np.maximum(h2, 0.0))
    t1 = np.maximum(-t0, -w)
    t2 = np.minimum(L[None, :] - t0, w)

    def F(t):
        return h2 * h2 * t - (2.0 / 3.0) * h2 * t ** 3 + t ** 5 / 5.0

    val = F(t2) - F(t1)
    return np.where((h2 > 0) & (t2 > t1) & (L[None, :] > 0), val, 0.0)


def weight_R4(rho, R: float, C: float):
    """PHYSICAL weight over R^4: Sigma = weight_R4 * R^4 I. An isolated
    infinite strut then has Sigma = C at distance rho (Sec. 3.2)."""
    rho = np.asarray(rho, dtype=np.float64)
    return 15.0 * C / (16.0 * (R * R - rho * rho) ** 2.5)


def smooth_density(sigma, C: float, T: float) -> float:
    """Eq. 9 by sampling, with the smoothed indicator (reading D2)."""
    return float(np.mean(expit((np.asarray(sigma) - C) / T)))


def bisect_ratio(rho, target: float, iters: int) -> float:
    """Ratio s in [1/2, 2] with rho(s) = target for an increasing rho: the end
    points when the target is out of reach, else `iters` halvings."""
    lo, hi = 0.5, 2.0
    if rho(hi) <= target:
        return hi
    if rho(lo) >= target:
        return lo
    for _ in range(iters):
        mid = 0.5 * (lo + hi)
        if rho(mid) < target:
            lo = mid
        else:
            hi = mid
    return 0.5 * (lo + hi)


# ---------------------------------------------------------------- geometry
def orient(a, b, c, d) -> float:
    """Six times the signed volume of (a, b, c, d), in one fixed order of
    FP64 operations (it decides containment, reading D3)."""
    ax = b[0] - a[0]
    ay = b[1] - a[1]
    az = b[2] - a[2]
    bx = c[0] - a[0]
    by = c[1] - a[1]
    bz = c[2] - a[2]
    cx = d[0] - a[0]
    cy = d[1] - a[1]
    cz = d[2] - a[2]
    return ax * (by * cz - bz * cy) - ay * (bx * cz - bz * cx) + az * (bx * cy - by * cx)


def point_in_tet(p, v) -> bool:
    v = [np.asarray(x, dtype=np.float64) for x in v]
    D = orient(v[0], v[1], v[2], v[3])
    if D == 0.0:
        return False
    Ds = (orient(p, v[1], v[2], v[3]), orient(v[0], p, v[2], v[3]),
          orient(v[0], v[1], p, v[3]), orient(v[0], v[1], v[2], p))
    if D > 0.0:
        return all(x >= 0.0 for x in Ds)
    return all(x <= 0.0 for x in Ds)


def seg_meets_box(a, b, lo, hi) -> bool:
    """Closed segment a-b against the closed box [lo, hi] (slab test, FP64)."""
    t0, t1 = 0.0, 1.0
    for k in range(3):
        d = b[k] - a[k]
        if d == 0.0:
            if a[k] < lo[k] or a[k] > hi[k]:
                return False
        else:
            ta = (lo[k] - a[k]) / d
            tb = (hi[k] - a[k]) / d
            if ta > tb:
                ta, tb = tb, ta
            if ta > t0:
                t0 = ta
            if tb < t1:
                t1 = tb
            if t0 > t1:
                return False
    return True


def trilinear(grid, p) -> float:
    """Trilinear interpolation of the voxel-centre values at p (clamped)."""
    o = grid["origin"]
    h = float(grid["h"])
    dims = grid["dims"]
    tgt = grid["target"]
    idx, frac = [], []
    for ax in range(3):
        n = int(dims[ax])
        g = (float(p[ax]) - float(o[ax])) / h - 0.5
        if n == 1:
            idx.append(0)
            frac.append(0.0)
            continue
        g = min(max(g, 0.0), float(n - 1))
        i0 = min(int(np.floor(g)), n - 2)
        idx.append(i0)
        frac.append(g - i0)
    val = 0.0
    for cz in (0, 1):
        for cy in (0, 1):
            for cx in (0, 1):
                wgt = ((frac[0] if cx else 1.0 - frac[0]) * (frac[1] if cy else 1.0 - frac[1])
                       * (frac[2] if cz else 1.0 - frac[2]))
                if wgt == 0.0:
                    continue
                i = min(idx[0] + cx, int(dims[0]) - 1)
                j = min(idx[1] + cy, int(dims[1]) - 1)
                k = min(idx[2] + cz, int(dims[2]) - 1)
                val += wgt * float(tgt[k, j, i])
    return val


def voxel_centre(grid, i, j, k):
    o = grid["origin"]
    h = float(grid["h"])
    return (float(o[0]) + h * (i + 0.5), float(o[1]) + h * (j + 0.5), float(o[2]) + h * (k + 0.5))


def tet_target(grid, v) -> float:
    """Step 1: the largest target of the voxels whose centres the tetrahedron
    contains (D3), else the interpolated target at its centroid (D4). Only
    centres inside the tetrahedron's bounding box can be contained, so the
    others are not tested."""
    dims = grid["dims"]
    vv = np.asarray(v, dtype=np.float64)
    lo, hi = vv.min(0), vv.max(0)
    o = np.asarray(grid["origin"], dtype=np.float64)
    h = float(grid["h"])
    rng = []
    for ax in range(3):
        c = o[ax] + h * (np.arange(int(dims[ax])) + 0.5)
        rng.append(np.nonzero((c >= lo[ax]) & (c <= hi[ax]))[0])
    best = None
    for k in rng[2]:
        for j in rng[1]:
            for i in rng[0]:
                if point_in_tet(voxel_centre(grid, int(i), int(j), int(k)), v):
                    t = float(grid["target"][k, j, i])
                    best = t if best is None else max(best, t)
    if best is not None:
        return best
    v = np.asarray(v, dtype=np.float64)
    c = (v[0] + v[1] + v[2] + v[3]) * 0.25
    return trilinear(grid, c)


# ---------------------------------------------------------------- the mesh
class TetLattice:
    """Nodes (float32), edges keyed by their node pair, tetrahedra with their
    six edge ids; subdivision appends nodes, edges and tetrahedra in a fixed
    order (reading D5)."""

    def __init__(self, nodes, tets):
        self.nodes = [tuple(np.float32(c) for c in row) for row in np.asarray(nodes, np.float32)]
        keys = set()
        for t in np.asarray(tets, dtype=np.int64):
            for p, q in LOCAL_EDGES:
                a, b = int(t[p]), int(t[q])
                keys.add((min(a, b), max(a, b)))
        self.edges = sorted(keys)
        self.edge_id = {k: i for i, k in enumerate(self.edges)}
        self.children = [None] * len(self.edges)   # (half id, half id) once split
        self.mid = [None] * len(self.edges)        # midpoint node id once split
        self.tets = [tuple(int(x) for x in t) for t in np.asarray(tets, dtype=np.int64)]
        self.tet_edges = [self._tet_edge_ids(t) for t in self.tets]
        self.depth = [0] * len(self.tets)
        self.leaf = [True] * len(self.tets)

    def _edge(self, a, b):
        k = (min(a, b), max(a, b))
        e = self.edge_id.get(k)
        if e is None:
            e = len(self.edges)
            self.edges.append(k)
            self.edge_id[k] = e
            self.children.append(None)
            self.mid.append(None)
        return e

    def _tet_edge_ids(self, t):
        return [self._edge(t[p], t[q]) for p, q in LOCAL_EDGES]

    def coords(self, i):
        return np.array(self.nodes[i], dtype=np.float64)

    def _split(self, e):
        if self.mid[e] is None:
            a, b = self.edges[e]
            pa, pb = self.nodes[a], self.nodes[b]
            m = tuple(np.float32((np.float64(pa[k]) + np.float64(pb[k])) * 0.5) for k in range(3))
            mid = len(self.nodes)
            self.nodes.append(m)
            self.mid[e] = mid
            h0 = self._edge(a, mid)
            h1 = self._edge(mid, b)
            self.children[e] = (h0, h1)
        return self.mid[e]

    def _len2(self, i, j):
        pi, pj = self.nodes[i], self.nodes[j]
        dx = np.float64(pi[0]) - np.float64(pj[0])
        dy = np.float64(pi[1]) - np.float64(pj[1])
        dz = np.float64(pi[2]) - np.float64(pj[2])
        return float(dx * dx + dy * dy + dz * dz)

    def subdivide(self, t):
        """1:8 subdivision (Sec. 5.5, subdivision operator): four corner
        tetrahedra and four around the octahedron's shortest diagonal."""
        v = self.tets[t]
        m = {}
        for k, (p, q) in enumerate(LOCAL_EDGES):
            m[(p, q)] = self._split(self.tet_edges[t][k])
        m01, m02, m03 = m[(0, 1)], m[(0, 2)], m[(0, 3)]
        m12, m13, m23 = m[(1, 2)], m[(1, 3)], m[(2, 3)]
        kids = [(v[0], m01, m02, m03), (m01, v[1], m12, m13), (m02, m12, v[2], m23),
                (m03, m13, m23, v[3])]
        options = (((m01, m23), (m02, m03, m13, m12)), ((m02, m13), (m01, m03, m23, m12)),
                   ((m03, m12), (m01, m02, m23, m13)))
        best = 0
        best_l2 = self._len2(*options[0][0])
        for i in (1, 2):
            l2 = self._len2(*options[i][0])
            if l2 < best_l2:
                best, best_l2 = i, l2
        (p, q), cyc = options[best]
        for i in range(4):
            kids.append((p, q, cyc[i], cyc[(i + 1) % 4]))
        self.leaf[t] = False
        ids = []
        for kt in kids:
            self.tets.append(kt)
            self.tet_edges.append(self._tet_edge_ids(kt))
            self.depth.append(self.depth[t] + 1)
            self.leaf.append(True)
            ids.append(len(self.tets) - 1)
        return ids

    def leaf_segments(self, e):
        if self.children[e] is None:
            return [e]
        a, b = self.children[e]
        return self.leaf_segments(a) + self.leaf_segments(b)

    def tet_vertices(self, t):
        return np.array([self.nodes[i] for i in self.tets[t]], dtype=np.float64)


def tet_density_fn(v, A, r0: float, R: float, C: float, T: float):
    """rho_T(s): density of tetrahedron v with its six struts at radius r0 s
    (reading D2)."""
    pts = tet_points(v, A)
    a = np.array([v[p] for p, _ in LOCAL_EDGES])
    b = np.array([v[q] for _, q in LOCAL_EDGES])
    J = seg_R4I(pts, a, b, R).sum(1)
    return lambda s: smooth_density(weight_R4(r0 * s, R, C) * J, C, T)


def voxel_density_fn(grid, i, j, k, seg_a, seg_b, seg_ratio, r0: float, R: float, C: float,
                     T: float, m: int):
    """(rho_V(s), meets) of voxel (i, j, k) (reading D7): the struts meeting the
    voxel at radius r0 s, the others at r0 * seg_ratio. Struts whose support
    box misses the voxel contribute nothing at its samples and are skipped."""
    o = [float(x) for x in grid["origin"]]
    h = float(grid["h"])
    lo = (o[0] + h * i, o[1] + h * j, o[2] + h * k)
    hi = (o[0] + h * (i + 1), o[1] + h * (j + 1), o[2] + h * (k + 1))
    seg_a = np.asarray(seg_a, dtype=np.float64).reshape(-1, 3)
    seg_b = np.asarray(seg_b, dtype=np.float64).reshape(-1, 3)
    near = np.all((np.minimum(seg_a, seg_b) - R <= np.array(hi))
                  & (np.maximum(seg_a, seg_b) + R >= np.array(lo)), axis=1)
    idx = np.nonzero(near)[0]
    meets = np.zeros(seg_a.shape[0], dtype=bool)
    for s in idx:
        meets[s] = seg_meets_box(seg_a[s], seg_b[s], lo, hi)
    pts = voxel_points(grid, i, j, k, m)
    M = seg_R4I(pts, seg_a[idx], seg_b[idx], R)
    mi = meets[idx]
    F = (M[:, ~mi] * weight_R4(r0 * np.asarray(seg_ratio)[idx][~mi], R, C)[None, :]).sum(1)
    J = M[:, mi].sum(1)
    return (lambda s: smooth_density(F + weight_R4(r0 * s, R, C) * J, C, T)), meets


def density_match(nodes, tets, grid, *, r_min: float, R: float | None = None, C: float = 1.0,
                  temperature: float = 0.01, tet_n: int = 8, vox_m: int = 8, max_depth: int = 3,
                  iters: int = 24):
    """The four steps of Sec. 5.5 on a tetrahedral lattice. grid: dict with
    origin (3,), h, dims (nx, ny, nz) and target [nz, ny, nx].

    Returns a dict: nodes (float32 [N, 3]), edges (int32 [E, 2], the unsplit
    edges in creation order), radius (float64 [E]), tets / depth / target /
    rho_star / ratio of the leaf tetrahedra (in creation order), voxel_ratio
    (float64 [nz, ny, nx], NaN where no edge meets the voxel) and flags (the
    subdivision decisions with their margins rho* - target)."""
    r0 = 2.0 * float(r_min)
    R = 1.5 * 2.0 * r0 if R is None else float(R)
    if not 2.0 * r0 < R:
        raise ValueError("the doubled radius must stay below R")
    T = temperature * C
    A = kuhn_coefficients(tet_n)
    lat = TetLattice(nodes, tets)
    target, rho_star, ratio = {}, {}, {}
    decisions = []
    cand = list(range(len(lat.tets)))
    for d in range(max_depth + 1):
        nxt = []
        for t in cand:
            v = lat.tet_vertices(t)
            target[t] = tet_target(grid, v)
            rho = tet_density_fn(v, A, r0, R, C, T)
            rho_star[t] = rho(2.0)
            split = d < max_depth and rho_star[t] < target[t]
            decisions.append((t, rho_star[t] - target[t], split))
            if split:
                nxt.extend(lat.subdivide(t))
            else:
                ratio[t] = bisect_ratio(rho, target[t], iters)     # step 3
        cand = nxt
    leaves = [t for t in range(len(lat.tets)) if lat.leaf[t]]

    # step 3: every edge takes the smallest ratio of the leaf tetrahedra containing it
    n_e = len(lat.edges)
    e_ratio = np.full(n_e, np.inf)
    for t in leaves:
        for e in lat.tet_edges[t]:
            for s in lat.leaf_segments(e):
                e_ratio[s] = min(e_ratio[s], ratio[t])
    segs = [e for e in range(n_e) if lat.children[e] is None]
    e_ratio[np.isinf(e_ratio)] = 1.0
    seg_a = np.array([lat.coords(lat.edges[e][0]) for e in segs]).reshape(-1, 3)
    seg_b = np.array([lat.coords(lat.edges[e][1]) for e in segs]).reshape(-1, 3)
    seg_r = e_ratio[segs]

    # step 4: the common ratio of each voxel, against the step-3 ratios
    dims = [int(x) for x in grid["dims"]]
    vox = np.full((dims[2], dims[1], dims[0]), np.nan)
    new_r = seg_r.copy()
    for k in range(dims[2]):
        for j in range(dims[1]):
            for i in range(dims[0]):
                rho, meets = voxel_density_fn(grid, i, j, k, seg_a, seg_b, seg_r, r0, R, C, T,
                                              vox_m)
                if not meets.any():
                    continue
                s_v = bisect_ratio(rho, float(grid["target"][k, j, i]), iters)
                vox[k, j, i] = s_v
                new_r[meets] = np.minimum(new_r[meets], s_v)
    nodes_out = np.array(lat.nodes, dtype=np.float32).reshape(-1, 3)
    edges_out = np.array([lat.edges[e] for e in segs], dtype=np.int32).reshape(-1, 2)
    return dict(
        nodes=nodes_out, edges=edges_out, radius=r0 * new_r, ratio=new_r, step3_ratio=seg_r,
        tets=np.array([lat.tets[t] for t in leaves], dtype=np.int32).reshape(-1, 4),
        depth=np.array([lat.depth[t] for t in leaves], dtype=np.int32),
        target=np.array([target[t] for t in leaves]),
        rho_star=np.array([rho_star[t] for t in leaves]),
        tet_ratio=np.array([ratio[t] for t in leaves]),
        voxel_ratio=vox, decisions=decisions, r0=r0, R=R, lattice=lat)
