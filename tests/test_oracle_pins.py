"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Nothing here compares the oracle with itself: each check uses an independent
library routine (scipy quadrature), a closed form, a hand-derived marching-
squares case, a symmetry of a regular lattice, or brute force.
"""
import math

import numpy as np
import pytest
from scipy import integrate

import oracle
import synth

R_DEF = 0.75


def quad_segment(p, a, b, R):
    """Eq. 6 integrand (Eq. 5 kernel) integrated by arc length with scipy."""
    p, a, b = (np.asarray(x, dtype=np.float64) for x in (p, a, b))
    L = float(np.linalg.norm(b - a))
    if L == 0.0:
        return 0.0
    u = (b - a) / L

    def f(t):
        d2 = float(np.sum((p - a - t * u) ** 2))
        return (1.0 - d2 / R ** 2) ** 2 if d2 < R ** 2 else 0.0

    # the support along the line is where the distance is below R
    t0 = float(np.dot(p - a, u))
    e2 = float(np.sum((p - a - t0 * u) ** 2))
    if e2 >= R * R:
        return 0.0
    w = math.sqrt(R * R - e2)
    lo, hi = max(0.0, t0 - w), min(L, t0 + w)
    if lo >= hi:
        return 0.0
    val, _ = integrate.quad(f, lo, hi, epsabs=1e-15, epsrel=1e-13, limit=200)
    return val


# ---------------------------------------------------------------- Eq. 5 ----

def test_kernel_values():
    assert oracle.kernel(0.0, 2.0) == 1.0
    assert oracle.kernel(4.0, 2.0) == 0.0
    assert oracle.kernel(5.0, 2.0) == 0.0
    assert oracle.kernel(1.0, 2.0) == pytest.approx(0.5625, abs=0)   # (1 - 1/4)^2


# ---------------------------------------------------------------- Eq. 7 ----

def _random_cases(n, seed):
    r = np.random.default_rng(seed)
    cases = []
    for _ in range(n):
        R = r.uniform(0.3, 1.2)
        a = r.uniform(-1, 1, 3)
        b = a + r.normal(size=3) * r.uniform(0.05, 2.5)
        # a point near the segment so that most cases intersect the support
        t = r.uniform(-0.3, 1.3)
        p = a + t * (b - a) + r.normal(size=3) * R * 0.6
        cases.append((p, a, b, R))
    return cases


def test_segment_integral_matches_quadrature():
    hits = 0
    for p, a, b, R in _random_cases(400, 1):
        ref = quad_segment(p, a, b, R)
        got = oracle.segment_integral(p, a, b, R)
        assert got == pytest.approx(ref, rel=1e-9, abs=1e-14)
        hits += ref > 0
    assert hits > 200


def test_three_point_gauss_legendre_is_exact_on_the_clipped_interval():
    """The GPU evaluates Eq. 7 by 3-point Gauss-Legendre on the clipped
    interval [tau1, tau2]: in the edge's frame the kernel is (w^2 - tau^2)^2 / R^4,
    a polynomial of degree 4, which the rule integrates exactly. Written
    here in FP64 from the rule's nodes (0, +-sqrt(3/5)) and weights (8/9,
    5/9), it must equal the oracle's closed form to rounding. A dropped or
    wrongly weighted node, or a midpoint/half-width mix-up, is off by far
    more."""
    g = math.sqrt(0.6)
    hits = 0
    for p, a, b, R in _random_cases(400, 7):
        u = b - a
        L = float(np.linalg.norm(u))
        u = u / L
        t0 = float(np.dot(p - a, u))
        e = p - a - t0 * u
        h2 = R * R - float(np.dot(e, e))
        gl = 0.0
        if h2 > 0.0:
            w = math.sqrt(h2)
            t1, t2 = max(-t0, -w), min(L - t0, w)
            if t2 > t1:
                m, h = 0.5 * (t1 + t2), 0.5 * (t2 - t1)
                f = lambda tau: (h2 - tau * tau) ** 2 / R ** 4
                gl = h * (5.0 / 9.0 * (f(m - g * h) + f(m + g * h)) + 8.0 / 9.0 * f(m))
        ref = oracle.segment_integral(p, a, b, R)
        # to rounding of integrals of order 1 (the closed form subtracts quintics,
        # so near the support's edge it carries ~1e-15 absolute)
        assert gl == pytest.approx(ref, rel=1e-11, abs=1e-14)
        hits += ref > 0
    assert hits > 200


def test_segment_integral_clip_cases():
    R = 1.0
    a, b = np.array([0.0, 0, 0]), np.array([0.0, 0, 3.0])
    # sphere wholly inside the edge, end inside the sphere, start inside, miss
    for p in ([0.3, 0, 1.5], [0.2, 0.1, 2.7], [0.1, 0.3, 0.2], [1.2, 0, 1.0], [0, 0, -0.5],
              [0, 0, 3.9], [0.999, 0, 1.0]):
        assert oracle.segment_integral(p, a, b, R) == pytest.approx(quad_segment(p, a, b, R),
                                                                    rel=1e-9, abs=1e-15)
    # zero-length edge contributes 0; symmetric in the endpoints
    assert oracle.segment_integral([0, 0, 0], a, a, R) == 0.0
    p = np.array([0.2, 0.3, 2.9])
    assert oracle.segment_integral(p, a, b, R) == pytest.approx(
        oracle.segment_integral(p, b, a, R), rel=1e-12)


def test_infinite_strut_closed_form():
    # integral over the whole chord: 16 (R^2 - d^2)^(5/2) / (15 R^4)
    R = 0.75
    a, b = np.array([0.0, 0, -10]), np.array([0.0, 0, 10])
    for d in (0.0, 0.1, 0.3, 0.5, 0.7, 0.7499):
        closed = 16.0 * (R * R - d * d) ** 2.5 / (15.0 * R ** 4)
        assert oracle.segment_integral([d, 0, 0.37], a, b, R) == pytest.approx(closed, rel=1e-11)


def test_physical_weight_puts_isosurface_at_radius():
    # an isolated long strut with the PHYSICAL weight has Sigma = C at distance rho
    R, C = 0.75, 2.5
    a, b = np.array([0.0, 0, -10]), np.array([0.0, 0, 10])
    for rho in (0.1, 0.3, 0.5, 0.6):
        w = oracle.weight(rho, R, C, oracle.PHYSICAL)
        val = w * quad_segment([rho, 0, 0.1], a, b, R)
        assert val == pytest.approx(C, rel=1e-10)
    assert oracle.weight(0.37, R, C, oracle.RAW) == pytest.approx(0.37)
    # dw/drho by central differences
    for rho in (0.2, 0.45):
        h = 1e-6
        fd = (oracle.weight(rho + h, R, C) - oracle.weight(rho - h, R, C)) / (2 * h)
        assert oracle.weight_drho(rho, R, C) == pytest.approx(fd, rel=1e-7)


def test_strut_radius_monotone_in_weight():
    # Sec. 3.2: a smaller r_i moves the iso-surface towards the edge (RAW mode:
    # the radius argument is the paper's r_i itself)
    R, C = 0.75, 1.0
    nodes = np.array([[0, 0, -10], [0, 0, 10]], dtype=np.float32)
    edges = np.array([[0, 1]], dtype=np.int32)
    radii = []
    for w in (1.5, 2.0, 4.0, 8.0, 16.0):
        lo, hi = 0.0, R
        for _ in range(50):
            mid = 0.5 * (lo + hi)
            s = oracle.sigma_points(nodes, edges, np.array([w], np.float32), [[mid, 0, 0]],
                                    R=R, C=C, mode=oracle.RAW)[0]
            if s >= C:
                lo = mid
            else:
                hi = mid
        radii.append(lo)
    assert all(0 < x < y < R for x, y in zip(radii, radii[1:]))


# ------------------------------------------------- Steps 1-6 (sweep) -------

def test_sweep_equals_brute_force_quadrature():
    r = np.random.default_rng(7)
    nodes = r.uniform(0, 3, size=(30, 3)).astype(np.float32)
    edges = r.integers(0, 30, size=(45, 2)).astype(np.int32)
    radius = r.uniform(0.1, 0.4, size=45).astype(np.float32)
    R = 0.6
    sig = oracle.slice_sigma(nodes, edges, radius, R=R, C=1.0, z0=0.3, dz=0.9, n_layers=3,
                             x0=0.0, y0=0.0, nx=6, ny=5, pixel=0.5)
    for k in range(3):
        for j in range(5):
            for i in range(6):
                p = np.array([(i + 0.5) * 0.5, (j + 0.5) * 0.5, 0.3 + 0.9 * k])
                ref = 0.0
                for e in range(45):
                    a = nodes[edges[e, 0]].astype(np.float64)
                    b = nodes[edges[e, 1]].astype(np.float64)
                    w = oracle.weight(float(radius[e]), R, 1.0)
                    ref += w * quad_segment(p, a, b, R)
                assert sig[k, j, i] == pytest.approx(ref, rel=1e-9, abs=1e-12)


def test_sigma_points_equals_slice():
    nodes, edges, radius = synth.cubic_bcc(2, 5.0, 0.5)
    sig = oracle.slice_sigma(nodes, edges, radius, R=0.75, z0=0.3, dz=1.1, n_layers=4,
                             x0=0.0, y0=0.0, nx=9, ny=7, pixel=1.1)
    pts = []
    for k in range(4):
        for j in range(7):
            for i in range(9):
                pts.append(((i + 0.5) * 1.1, (j + 0.5) * 1.1, 0.3 + 1.1 * k))
    pts = np.array(pts)[::-1]   # reversed order: the sweep must sort them
    got = oracle.sigma_points(nodes, edges, radius, pts, R=0.75)[::-1]
    np.testing.assert_allclose(got, sig.ravel(), rtol=0, atol=0)


def test_active_set_contains_every_contributor():
    nodes, edges, radius, _ = synth.adaptive_graded(box=6.25, level_min=0, level_max=3)
    R = 0.2
    r = np.random.default_rng(3)
    for z in (0.3, 2.0, 4.41):
        act = set(oracle.active_set(nodes, edges, R, z).tolist())
        for _ in range(200):
            p = np.array([r.uniform(0, 6.25), r.uniform(0, 6.25), z])
            for e in range(edges.shape[0]):
                a = nodes[edges[e, 0]].astype(np.float64)
                b = nodes[edges[e, 1]].astype(np.float64)
                if abs(a[2] - z) > 2 and abs(b[2] - z) > 2:
                    continue
                if oracle.segment_integral(p, a, b, R) > 0:
                    assert e in act


# ------------------------------------------------- symmetry, C1 lattice ----

@pytest.fixture(scope="module")
def c1_layers():
    c = synth.config(1)
    sig = oracle.slice_sigma(c["nodes"], c["edges"], c["radius"], R=c["R"], z0=1.25, dz=5.0,
                             n_layers=2, x0=0.0, y0=0.0, nx=200, ny=200, pixel=0.1)
    return c, sig


def test_c1_symmetry(c1_layers):
    c, sig = c1_layers
    s = sig[0]
    np.testing.assert_allclose(s, s.T, rtol=1e-12, atol=1e-13)            # x <-> y
    np.testing.assert_allclose(s, s[:, ::-1], rtol=1e-12, atol=1e-13)     # x -> 20 - x
    np.testing.assert_allclose(s, s[::-1, :], rtol=1e-12, atol=1e-13)     # y -> 20 - y
    np.testing.assert_allclose(sig[0], sig[1], rtol=1e-12, atol=1e-13)    # one period in z


def test_c1_loop_count(c1_layers):
    # z = 1.25 meets the 25 vertical cube edges and 4 body diagonals per cell
    c, sig = c1_layers
    off, eid, xy = oracle.marching_squares(sig[0], x0=0.0, y0=0.0, pixel=0.1, C=1.0)
    assert len(off) - 1 == 25 + 4 * 16


# ------------------------------------------------- marching squares --------

def _area(xy):
    x, y = xy[:, 0], xy[:, 1]
    return 0.5 * float(np.sum(x * np.roll(y, -1) - np.roll(x, -1) * y))


def test_ms_single_pixel_loop():
    # one inside pixel, value 3, C = 1: t = (3 - 1) / (3 - 0) = 2/3 from the centre
    off, eid, xy = oracle.marching_squares(np.array([[3.0]]), x0=0.0, y0=0.0, pixel=1.0, C=1.0)
    assert off.tolist() == [0, 4]
    # padded width 3: bottom vertical edge 2*(0*3+1)+1 = 3, right horizontal 2*(1*3+1) = 8,
    # top vertical 2*(1*3+1)+1 = 9, left horizontal 2*(1*3+0) = 6; counter-clockwise
    assert eid.tolist() == [3, 8, 9, 6]
    t = 2.0 / 3.0
    np.testing.assert_allclose(xy, [[0.5, 0.5 - t], [0.5 + t, 0.5], [0.5, 0.5 + t],
                                    [0.5 - t, 0.5]], atol=1e-15)
    assert _area(xy) > 0


def test_ms_saddle_rule():
    # diagonal inside pixels; the mean of the four decides joined / separated
    sep = np.array([[1.5, 0.2], [0.2, 1.5]])
    joined = np.array([[1.9, 0.3], [0.3, 1.9]])
    off, _, _ = oracle.marching_squares(sep, x0=0, y0=0, pixel=1.0, C=1.0)
    assert np.diff(off).tolist() == [4, 4]
    off, eid, xy = oracle.marching_squares(joined, x0=0, y0=0, pixel=1.0, C=1.0)
    assert np.diff(off).tolist() == [8]
    assert _area(xy) > 0


def test_ms_annulus_orientation():
    f = np.full((5, 5), 2.0)
    f[2, 2] = 0.5
    off, eid, xy = oracle.marching_squares(f, x0=0, y0=0, pixel=1.0, C=1.0)
    lens = np.diff(off).tolist()
    assert sorted(lens) == [4, 20]
    areas = [_area(xy[off[i]:off[i + 1]]) for i in range(2)]
    outer = int(np.argmax(lens))
    assert areas[outer] > 0 and areas[1 - outer] < 0
    # loops are listed by their smallest edge id and start there
    for i in range(2):
        seg = eid[off[i]:off[i + 1]]
        assert seg[0] == seg.min()
    assert eid[off[0]] < eid[off[1]]


def test_ms_empty_and_full():
    off, eid, xy = oracle.marching_squares(np.zeros((4, 3)), x0=0, y0=0, pixel=1.0, C=1.0)
    assert off.tolist() == [0] and eid.size == 0
    off, eid, xy = oracle.marching_squares(np.full((4, 3), 5.0), x0=0, y0=0, pixel=1.0, C=1.0)
    assert off.tolist() == [0, 14] and _area(xy) > 0


def test_isolated_strut_circle():
    rho, R = 0.5, 0.75
    nodes = np.array([[0, 0, -10], [0, 0, 10]], dtype=np.float32)
    edges = np.array([[0, 1]], dtype=np.int32)
    radius = np.array([rho], dtype=np.float32)
    px = 0.02
    sig = oracle.slice_sigma(nodes, edges, radius, R=R, z0=0.0, dz=1.0, n_layers=1,
                             x0=-1.0, y0=-1.0, nx=100, ny=100, pixel=px)
    off, eid, xy = oracle.marching_squares(sig[0], x0=-1.0, y0=-1.0, pixel=px, C=1.0)
    assert len(off) == 2
    r = np.hypot(xy[:, 0], xy[:, 1])
    assert np.max(np.abs(r - rho)) < 0.01 * px
    assert _area(xy) == pytest.approx(math.pi * rho * rho, rel=2e-3)


def test_slanted_strut_ellipse():
    rho, R, phi = 0.4, 0.6, math.radians(40)
    u = np.array([math.sin(phi), 0.0, math.cos(phi)])
    nodes = np.array([-12 * u, 12 * u], dtype=np.float32)
    edges = np.array([[0, 1]], dtype=np.int32)
    radius = np.array([rho], dtype=np.float32)
    px = 0.02
    sig = oracle.slice_sigma(nodes, edges, radius, R=R, z0=0.0, dz=1.0, n_layers=1,
                             x0=-1.0, y0=-1.0, nx=100, ny=100, pixel=px)
    off, eid, xy = oracle.marching_squares(sig[0], x0=-1.0, y0=-1.0, pixel=px, C=1.0)
    assert len(off) == 2
    # nodes are float32: use the stored direction for the analytic ellipse
    a, b = nodes.astype(np.float64)
    uu = (b - a) / np.linalg.norm(b - a)
    p = np.concatenate([xy, np.zeros((xy.shape[0], 1))], axis=1) - a
    d = np.linalg.norm(p - np.outer(p @ uu, uu), axis=1)
    assert np.max(np.abs(d - rho)) < 0.01 * px
    assert _area(xy) == pytest.approx(math.pi * rho * rho / math.cos(phi), rel=2e-3)


# ------------------------------------------------- volume fraction ---------

def test_vf_hard_limit_isolated_strut():
    # a long vertical strut through one cell, T -> 0: vf is the share of the
    # 8x8 sample columns inside the circle of radius rho
    rho, R, m, h = 0.3, 0.45, 8, 1.0
    nodes = np.array([[0.5, 0.5, -5], [0.5, 0.5, 5]], dtype=np.float32)
    edges = np.array([[0, 1]], dtype=np.int32)
    radius = np.array([rho], dtype=np.float32)
    cells = dict(origin=(0.0, 0.0, 0.0), h=h, dims=(1, 1, 1), m=m, T=1e-5)
    vf = oracle.volume_fraction(nodes, edges, radius, cells, R=R)
    k = (np.arange(m) + 0.5) / m
    X, Y = np.meshgrid(k, k)
    d = np.hypot(X - 0.5, Y - 0.5)
    assert np.min(np.abs(d - rho)) > 0.01          # no sample on the boundary
    assert vf[0] == pytest.approx(float(np.mean(d < rho)), abs=1e-12)
    # and approximately pi rho^2 l / h^3
    assert vf[0] == pytest.approx(math.pi * rho * rho, abs=0.05)


def test_vf_soft_values_in_range():
    nodes, edges, radius = synth.cubic_bcc(1, 2.0, 0.3)
    cells = dict(origin=(0.0, 0.0, 0.0), h=1.0, dims=(2, 2, 2), m=4, T=0.01)
    vf = oracle.volume_fraction(nodes, edges, radius, cells, R=0.45)
    assert np.all(vf > 0) and np.all(vf < 1)
    # the cube is symmetric under the 8 octant reflections: all cells equal
    np.testing.assert_allclose(vf, vf[0], rtol=1e-12)


# ------------------------------------------------- gradients ---------------

def test_segment_gradient_against_finite_differences():
    h = 1e-6
    n_checked = 0
    for p, a, b, R in _random_cases(150, 11):
        I, ga, gb = oracle.segment_integral_grad(p, a, b, R)
        assert I == pytest.approx(oracle.segment_integral(p, a, b, R), rel=1e-9, abs=1e-14)
        if I < 1e-6:
            continue
        n_checked += 1
        for k in range(3):
            e = np.zeros(3)
            e[k] = h
            fa = (oracle.segment_integral(p, a + e, b, R) - oracle.segment_integral(p, a - e, b, R)) / (2 * h)
            fb = (oracle.segment_integral(p, a, b + e, R) - oracle.segment_integral(p, a, b - e, R)) / (2 * h)
            fp = (oracle.segment_integral(p + e, a, b, R) - oracle.segment_integral(p - e, a, b, R)) / (2 * h)
            scale = max(abs(fa), abs(fb), abs(fp), 1e-3)
            assert ga[k] == pytest.approx(fa, abs=2e-7 * scale + 1e-9)
            assert gb[k] == pytest.approx(fb, abs=2e-7 * scale + 1e-9)
            # translation invariance: d/da + d/db = -d/dp
            assert ga[k] + gb[k] == pytest.approx(-fp, abs=2e-7 * scale + 1e-9)
    assert n_checked > 60


def _richardson(fd_fn, h):
    # central differences have an h^2 error term; two steps cancel it
    return (4.0 * fd_fn(h / 2) - fd_fn(h)) / 3.0


def test_vf_gradient_against_finite_differences():
    # With T = 0.01 C the sigmoid is sharp: a radius step of 1e-4 mm moves
    # (Sigma - C) / T by ~0.06, so a plain central difference carries an
    # O(h^2) error of ~1e-4 relative. The pin uses the Richardson-extrapolated
    # difference (error O(h^4)); the plain h = 1e-4 difference is checked at
    # its own truncation level.
    nodes, edges, radius = synth.freudenthal(3, 1.0, 0.2, (0.15, 0.35), seed=99)
    cells = dict(origin=(0.0, 0.0, 0.0), h=0.75, dims=(3, 3, 3), m=4, T=0.01)
    R = 0.525
    r = np.random.default_rng(5)
    g = r.normal(size=27)
    gr, gn = oracle.vf_backward(nodes, edges, radius, cells, g, R=R)
    je = r.choice(edges.shape[0], 12, replace=False)

    def fd_r(h):
        return oracle.vf_fd(nodes, edges, radius, cells, g, np.zeros(12), je, R=R, h=h)

    scale = np.max(np.abs(gr))
    np.testing.assert_allclose(gr[je], _richardson(fd_r, 1e-4), rtol=1e-6, atol=1e-8 * scale)
    np.testing.assert_allclose(gr[je], fd_r(1e-4), rtol=1e-3, atol=1e-6 * scale)
    jn = r.choice(nodes.shape[0], 6, replace=False)
    kind = np.repeat([1, 2, 3], 6)
    idx = np.tile(jn, 3)

    def fd_n(h):
        return oracle.vf_fd(nodes, edges, radius, cells, g, kind, idx, R=R, h=h)

    an = gn[idx, kind - 1]
    scale = np.max(np.abs(gn))
    np.testing.assert_allclose(an, _richardson(fd_n, 1e-4), rtol=1e-6, atol=1e-8 * scale)
    np.testing.assert_allclose(an, fd_n(1e-4), rtol=1e-3, atol=1e-6 * scale)
