"""Pins of the density-matching oracle (Sec. 5.5) to facts it does not
compute itself: quadrature, closed forms, the subdivision identities the paper
states, exact volumes, brute-force containment, and the C oracle's field."""
import itertools

import numpy as np
import pytest
from scipy import integrate

import oracle
import synth
from oracle import density as D


def _tet_volume(v):
    v = np.asarray(v, dtype=np.float64)
    return abs(np.linalg.det(np.stack([v[1] - v[0], v[2] - v[0], v[3] - v[0]]))) / 6.0


RANDOM_TET = np.array([[0.3, -0.2, 0.1], [4.1, 0.4, -0.3], [1.2, 3.7, 0.5], [0.9, 1.1, 3.3]])


@pytest.mark.parametrize("n", [1, 2, 3, 5])
def test_kuhn_samples_are_equal_volume_centroids(n):
    a = D.kuhn_coefficients(n)
    assert a.shape == (n ** 3, 3)
    assert np.all(a[:, 0] < 1) and np.all(a[:, 0] > a[:, 1]) and np.all(a[:, 1] > a[:, 2])
    assert np.all(a[:, 2] > 0)
    # centroid of {1 >= x1 >= x2 >= x3 >= 0}
    assert np.allclose(a.mean(0), [0.75, 0.5, 0.25], atol=1e-14)
    p = D.tet_points(RANDOM_TET, a)
    # the centroid rule on equal-volume pieces integrates linear functions exactly
    assert np.allclose(p.mean(0), RANDOM_TET.mean(0), atol=1e-12)
    # second moments of a tetrahedron: (sum v_i v_j^T + s s^T) / 20, s = sum of vertices
    s = RANDOM_TET.sum(0)
    exact = (RANDOM_TET.T @ RANDOM_TET + np.outer(s, s)) / 20.0
    got = p.T @ p / p.shape[0]
    scale = np.abs(exact).max()
    assert np.abs(got - exact).max() <= 0.2 * scale / n ** 2 + 1e-12
    if n >= 3:
        assert np.abs(got - exact).max() > 0     # not a tautology: the rule is only O(1/n^2)


def test_segment_integral_against_quadrature():
    R = 0.6
    r = synth.rng(7)
    a = np.array([[0.1, 0.2, -0.1]])
    b = np.array([[1.3, -0.4, 0.9]])
    L = np.linalg.norm(b - a)
    u = (b - a)[0] / L
    pts = a + r.uniform(-0.8, 1.8, size=(40, 1)) * (b - a) + r.uniform(-0.6, 0.6, size=(40, 3))
    got = D.seg_R4I(pts, a, b, R)[:, 0]
    for p, g in zip(pts, got):
        def f(t):
            x = a[0] + t * u
            q = R * R - np.sum((p - x) ** 2)
            return q * q if q > 0 else 0.0
        ref, _ = integrate.quad(f, 0.0, L, epsabs=1e-14, epsrel=1e-12, limit=200)
        assert abs(g - ref) <= 1e-10 * max(abs(ref), 1e-6), (g, ref)
    # the C oracle's segment integral (Eq. 7 x l) agrees too
    for p, g in zip(pts[:10], got[:10]):
        assert abs(g - R ** 4 * oracle.segment_integral(p, a[0], b[0], R)) <= 1e-12 * R ** 4


def test_isolated_long_strut_surface_at_its_radius():
    """PHYSICAL weights: a long strut's field equals C at distance r (Sec. 3.2),
    the infinite-line integral being 16 (R^2 - d^2)^(5/2) / 15."""
    R, C = 0.6, 1.0
    a = np.array([[0.0, 0.0, -10.0]])
    b = np.array([[0.0, 0.0, 10.0]])
    for r in (0.1, 0.2, 0.35):
        d = np.array([[r, 0.0, 0.3]])
        J = D.seg_R4I(d, a, b, R)[0, 0]
        assert abs(J - 16.0 * (R * R - r * r) ** 2.5 / 15.0) <= 1e-12
        assert abs(D.weight_R4(r, R, C) * J - C) <= 1e-12


def test_one_subdivision_matches_the_paper_identities():
    """Sec. 5.5: eight children of equal volume; the total edge length grows
    from sum l_i to l_r + 2 sum l_i; the new edges other than the octahedron's
    diagonal are parallel to an edge of the parent."""
    v = RANDOM_TET.astype(np.float32)
    lat = D.TetLattice(v, np.array([[0, 1, 2, 3]]))
    parent_len = [np.linalg.norm(v[q].astype(float) - v[p].astype(float)) for p, q in D.LOCAL_EDGES]
    kids = lat.subdivide(0)
    assert len(kids) == 8 and len(lat.nodes) == 10
    V = _tet_volume(v)
    for t in kids:
        assert abs(_tet_volume(lat.tet_vertices(t)) - V / 8) <= 1e-6 * V
    leaf = [e for e in range(len(lat.edges)) if lat.children[e] is None]
    assert len(leaf) == 6 * 2 + 12 + 1
    length = lambda e: np.linalg.norm(lat.coords(lat.edges[e][1]) - lat.coords(lat.edges[e][0]))
    mids = set(range(4, 10))
    diag = [e for e in leaf if set(lat.edges[e]) <= mids and
            not any(np.linalg.norm(np.cross(lat.coords(lat.edges[e][1]) - lat.coords(lat.edges[e][0]),
                                            v[q].astype(float) - v[p].astype(float))) < 1e-5
                    for p, q in D.LOCAL_EDGES)]
    assert len(diag) == 1
    l_r = length(diag[0])
    assert abs(sum(length(e) for e in leaf) - (l_r + 2 * sum(parent_len))) <= 1e-5
    # the diagonal is the shortest of the octahedron's three
    m = [lat.mid[lat.edge_id[(min(v0, v1), max(v0, v1))]] for v0, v1 in D.LOCAL_EDGES]
    cands = [np.linalg.norm(lat.coords(m[0]) - lat.coords(m[5])),
             np.linalg.norm(lat.coords(m[1]) - lat.coords(m[4])),
             np.linalg.norm(lat.coords(m[2]) - lat.coords(m[3]))]
    assert abs(l_r - min(cands)) <= 1e-6


def test_shared_faces_and_hanging_nodes():
    nodes = np.array([[0, 0, 0], [4, 0, 0], [0, 4, 0], [0, 0, 4], [3, 3, 3]], np.float32)
    tets = np.array([[0, 1, 2, 3], [1, 2, 3, 4]])
    both = D.TetLattice(nodes, tets)
    both.subdivide(0)
    both.subdivide(1)
    assert len(both.nodes) == 5 + 9
    leaf = [e for e in range(len(both.edges)) if both.children[e] is None]
    assert len(leaf) == 9 * 2 + (12 + 12 - 3) + 2
    assert len(set(both.edges)) == len(both.edges)
    # one side only: the other tetrahedron keeps its shared edges, now as halves
    one = D.TetLattice(nodes, tets)
    one.subdivide(0)
    shared = [one.edge_id[k] for k in ((1, 2), (1, 3), (2, 3))]
    for e in shared:
        assert e in one.tet_edges[1] and one.children[e] is not None
        segs = one.leaf_segments(e)
        assert len(segs) == 2
        tot = sum(np.linalg.norm(one.coords(one.edges[s][1]) - one.coords(one.edges[s][0]))
                  for s in segs)
        a, b = one.edges[e]
        assert abs(tot - np.linalg.norm(one.coords(b) - one.coords(a))) <= 1e-5


def test_containment_is_exact_and_kuhn_cells_tile_the_cube():
    # dyadic points on the boundary of an integer tetrahedron: exact determinants
    w = np.array([[0, 0, 0], [4, 0, 0], [1, 4, 0], [1, 1, 4]], np.float64)
    for p in list(w) + [w.mean(0), (w[0] + w[1] + 2 * w[2]) / 4, 0.5 * (w[1] + w[3])]:
        assert D.point_in_tet(p, w)
    v = RANDOM_TET
    c = v.mean(0)
    for k in range(4):
        assert not D.point_in_tet(v[k] + 0.01 * (v[k] - c), v)
    # the six tetrahedra of a cube: every interior point in exactly one
    tets = []
    for perm in itertools.permutations(range(3)):
        cc = np.zeros(3)
        vs = [cc.copy()]
        for ax in perm:
            cc[ax] += 1
            vs.append(cc.copy())
        tets.append(np.array(vs))
    r = synth.rng(3)
    for p in r.uniform(0, 1, size=(300, 3)):
        assert sum(D.point_in_tet(p, t) for t in tets) == 1
    # against barycentric coordinates from a linear solve
    for p in r.uniform(-1, 4, size=(300, 3)):
        lam = np.linalg.solve(np.vstack([v.T, np.ones(4)]), np.append(p, 1.0))
        if np.abs(lam).min() > 1e-9:
            assert D.point_in_tet(p, v) == bool(np.all(lam > 0))


def test_trilinear_reproduces_linear_fields_and_targets():
    grid = dict(origin=(0.5, -1.0, 2.0), h=1.5, dims=(4, 3, 5))
    nx, ny, nz = grid["dims"]
    xs = 0.5 + 1.5 * (np.arange(nx) + 0.5)
    ys = -1.0 + 1.5 * (np.arange(ny) + 0.5)
    zs = 2.0 + 1.5 * (np.arange(nz) + 0.5)
    lin = lambda x, y, z: 0.1 + 0.02 * x - 0.03 * y + 0.05 * z
    grid["target"] = lin(xs[None, None, :], ys[None, :, None], zs[:, None, None])
    r = synth.rng(5)
    for p in r.uniform([xs[0], ys[0], zs[0]], [xs[-1], ys[-1], zs[-1]], size=(50, 3)):
        assert abs(D.trilinear(grid, p) - lin(*p)) <= 1e-12
    # a tetrahedron containing voxel centres takes their largest target
    v = np.array([[0.0, -2.0, 1.0], [8.0, -2.0, 1.0], [0.0, 4.0, 1.0], [0.0, -2.0, 11.0]])
    inside = [(i, j, k) for k in range(nz) for j in range(ny) for i in range(nx)
              if np.all(np.linalg.solve(np.vstack([v.T, np.ones(4)]),
                                        np.array([xs[i], ys[j], zs[k], 1.0])) > 1e-9)]
    assert inside
    assert D.tet_target(grid, v) == max(grid["target"][k, j, i] for i, j, k in inside)
    # a small one with no centre inside interpolates at its centroid
    w = np.array([[1.6, 0.1, 3.1], [1.8, 0.1, 3.1], [1.6, 0.3, 3.1], [1.6, 0.1, 3.3]])
    assert abs(D.tet_target(grid, w) - lin(*w.mean(0))) <= 1e-12


def test_segment_box_test_against_dense_sampling():
    r = synth.rng(11)
    lo, hi = np.array([0.0, 0.0, 0.0]), np.array([1.0, 1.5, 2.0])
    for _ in range(300):
        a, b = r.uniform(-1.5, 3.0, size=(2, 3))
        t = np.linspace(0, 1, 20001)[:, None]
        x = a + t * (b - a)
        inside = np.all((x >= lo) & (x <= hi), axis=1)
        got = D.seg_meets_box(a, b, lo, hi)
        if inside.any():
            assert got
        elif got:
            # a hit the sampling missed must be a sliver: the segment comes within 1e-3
            d = np.max(np.maximum(lo - x, x - hi), axis=1).min()
            assert d < 1e-3


def _tet_density_c_oracle(v, s, r0, R, C, T, n):
    """rho_T(s) with the field of the C oracle (sigma_points) instead of seg_R4I."""
    pts = D.tet_points(v, D.kuhn_coefficients(n))
    nodes = np.asarray(v, np.float32)
    edges = np.array(D.LOCAL_EDGES, np.int32)
    sig = oracle.sigma_points(nodes, edges, np.full(6, r0 * s, np.float32), pts, R=R, C=C)
    return float(np.mean(1.0 / (1.0 + np.exp(-(sig - C) / T))))


def test_bisection_recovers_a_known_ratio():
    v = RANDOM_TET.astype(np.float32).astype(np.float64) * 0.5
    r0, R, C, T = 0.2, 0.6, 1.0, 0.01
    rho = D.tet_density_fn(v, D.kuhn_coefficients(6), r0, R, C, T)
    ss = np.linspace(0.5, 2.0, 16)
    vals = [rho(s) for s in ss]
    assert all(b > a for a, b in zip(vals, vals[1:]))        # increasing in the ratio
    for s0 in (0.73, 1.37, 1.9):
        s = D.bisect_ratio(rho, rho(s0), 30)
        assert abs(s - s0) <= 1e-6
        # and the density it solves for is the C oracle's field at that ratio
        # (whose radii are float32: the density moves by its slope x 6e-8)
        assert abs(_tet_density_c_oracle(v, s, r0, R, C, T, 6) - rho(s0)) <= 1e-7
    assert D.bisect_ratio(rho, 2.0, 30) == 2.0 and D.bisect_ratio(rho, -1.0, 30) == 0.5


def test_thin_struts_fill_their_wedges():
    """Far from the joints a strut of radius r is a cylinder (Sec. 3.2), so the
    density of a large tetrahedron with thin struts approaches the wedges'
    share sum_e theta_e r^2 l_e / (2 V) (theta_e the dihedral angle at e)."""
    v = np.array([[0, 0, 0], [10, 0, 0], [5, 8.66, 0], [5, 2.89, 8.16]], np.float64)
    r0, R, C, T = 0.25, 0.6, 1.0, 0.002
    rho = D.tet_density_fn(v, D.kuhn_coefficients(40), r0, R, C, T)(1.0)
    V = _tet_volume(v)
    est = 0.0
    for p, q in D.LOCAL_EDGES:
        o = [k for k in range(4) if k not in (p, q)]
        e = v[q] - v[p]
        e /= np.linalg.norm(e)
        n1 = (v[o[0]] - v[p]) - np.dot(v[o[0]] - v[p], e) * e
        n2 = (v[o[1]] - v[p]) - np.dot(v[o[1]] - v[p], e) * e
        theta = np.arccos(np.dot(n1, n2) / np.linalg.norm(n1) / np.linalg.norm(n2))
        est += theta * r0 * r0 * np.linalg.norm(v[q] - v[p]) / 2.0
    est /= V
    assert abs(rho - est) <= 0.25 * est, (rho, est)


@pytest.fixture(scope="module")
def small_result():
    cfg = synth.density_config(small=True)
    res = D.density_match(cfg["nodes"], cfg["tets"], cfg["grid"], r_min=cfg["r_min"],
                          tet_n=cfg["tet_n"], vox_m=cfg["vox_m"], max_depth=cfg["max_depth"],
                          iters=cfg["iters"])
    return cfg, res


def test_density_match_invariants(small_result):
    cfg, res = small_result
    lat = res["lattice"]
    # subdivision keeps the volume
    V0 = sum(_tet_volume(cfg["nodes"][t]) for t in cfg["tets"])
    V1 = sum(_tet_volume(res["nodes"][t]) for t in res["tets"])
    assert abs(V1 - V0) <= 1e-5 * V0
    # every leaf above the depth limit stopped because rho* reached its target
    for d, rs, tg in zip(res["depth"], res["rho_star"], res["target"]):
        if d < cfg["max_depth"]:
            assert rs >= tg
    assert 0 < res["depth"].min() or res["depth"].max() <= cfg["max_depth"]
    # radii between r_min and the doubled base radius; edges unique and unsplit
    r0 = res["r0"]
    assert np.all(res["radius"] >= 0.5 * r0 - 1e-12) and np.all(res["radius"] <= 2 * r0 + 1e-12)
    keys = set(map(tuple, res["edges"]))
    assert len(keys) == res["edges"].shape[0]
    # every leaf tetrahedron's edges are covered by final segments
    for t in range(len(lat.tets)):
        if lat.leaf[t]:
            for e in lat.tet_edges[t]:
                for s in lat.leaf_segments(e):
                    assert lat.edges[s] in keys
    # voxel ratios only lower the step-3 ratios
    assert np.all(res["ratio"] <= res["step3_ratio"] + 1e-15)


def test_step3_and_step4_ratios_solve_their_densities(small_result):
    """Re-evaluate the densities with the C oracle's field at the returned
    ratios: a tetrahedron at an interior ratio has its target density, and so
    has a voxel (with the other struts at their step-3 radii)."""
    cfg, res = small_result
    r0, R, C, T = res["r0"], res["R"], 1.0, 0.01
    n_checked = 0
    for k, t in enumerate(res["tets"][:40]):
        s = res["tet_ratio"][k]
        if 0.5 < s < 2.0:
            rho = _tet_density_c_oracle(res["nodes"][t].astype(np.float64), s, r0, R, C, T,
                                        cfg["tet_n"])
            assert abs(rho - res["target"][k]) <= 1e-5
            n_checked += 1
    assert n_checked >= 10
    grid = cfg["grid"]
    nodes, edges = res["nodes"], res["edges"]
    a = nodes[edges[:, 0]].astype(np.float64)
    b = nodes[edges[:, 1]].astype(np.float64)
    o, h = grid["origin"], grid["h"]
    n_vox = 0
    nx, ny, nz = grid["dims"]
    for k, j, i in itertools.product(range(nz), range(ny), range(nx)):
        s = res["voxel_ratio"][k, j, i]
        if not (0.5 < s < 2.0):
            continue
        lo = (o[0] + h * i, o[1] + h * j, o[2] + h * k)
        hi = (o[0] + h * (i + 1), o[1] + h * (j + 1), o[2] + h * (k + 1))
        meets = np.array([D.seg_meets_box(a[e], b[e], lo, hi) for e in range(len(edges))])
        rad = np.where(meets, r0 * s, r0 * res["step3_ratio"]).astype(np.float32)
        pts = D.voxel_points(grid, i, j, k, cfg["vox_m"])
        sig = oracle.sigma_points(nodes, edges, rad, pts, R=R, C=C)
        rho = float(np.mean(1.0 / (1.0 + np.exp(-(sig - C) / T))))
        # float32 radii in the C oracle: the density moves by its slope x 1e-7
        assert abs(rho - grid["target"][k, j, i]) <= 2e-5
        n_vox += 1
    assert n_vox >= 5
