"""Pins of the contour smoothing oracle: the closed-form shrinking of a
single-pixel diamond toward its sample, edge midpoints at margin 1/2 (the
binary-image marching squares), the straight side of a rectangle as a fixed
point, identities, and, on marching squares' own loops of the cubic+BCC
lattice (also after simplification), vertices kept on their edges inside the
margin and no crossing, by brute force over all segment pairs."""
import numpy as np
import pytest

import oracle
import synth
from oracle import simplify as Z
from oracle import smooth as M
from tests.test_oracle_simplify import _crossings, _segments


def _one_layer(s, pixel=1.0):
    return oracle.marching_squares(s, x0=0.0, y0=0.0, pixel=pixel, C=1.0)


@pytest.mark.parametrize("lam,mu,K", [(0.5, 0.05, 3), (0.5, 0.1, 3), (0.25, 0.02, 5)])
def test_single_pixel_diamond_closed_form(lam, mu, K):
    """One inside sample (Sigma = 2, C = 1) among outside ones (0): four
    vertices at half a pixel from it. Each vertex's neighbours lie on the
    other axis' edges through the sample, so its offset t from the sample
    shrinks as t_k = max(t_(k-1) (1 - lam), mu) from t_0 = 1/2."""
    s = np.zeros((3, 3))
    s[1, 1] = 2.0
    off, eid, xy = _one_layer(s)
    assert len(off) == 2 and int(off[1]) == 4
    xy32 = xy.astype(np.float32)
    out = M.smooth_loops(off, eid, xy32, x0=0.0, y0=0.0, pixel=1.0, nx=3, lam=lam, margin=mu,
                         iterations=K)
    t = 0.5
    for _ in range(K):
        t = max(t * (1.0 - lam), mu)
    cx = cy = 1.5                                  # the sample's centre
    for v in range(4):
        axis, _ = M.edge_axis_and_lo(int(eid[v]), 5, 0.0, 0.0, 1.0)
        other = 1 - axis
        assert out[v, other] == xy32[v, other]     # the fixed coordinate
        c = (cx, cy)[axis]
        side = np.sign(float(xy32[v, axis]) - c)
        assert abs(float(out[v, axis]) - (c + side * t)) <= 1e-6, (v, out[v], t)


def test_margin_one_half_gives_edge_midpoints():
    cfg = synth.config(1)
    sig = oracle.slice_sigma(cfg["nodes"], cfg["edges"], cfg["radius"], R=cfg["R"], C=cfg["C"],
                             z0=cfg["z0"] + 5 * cfg["dz"], dz=cfg["dz"], n_layers=1,
                             x0=cfg["x0"], y0=cfg["y0"], nx=cfg["nx"], ny=cfg["ny"],
                             pixel=cfg["pixel"])[0]
    off, eid, xy = oracle.marching_squares(sig, x0=cfg["x0"], y0=cfg["y0"], pixel=cfg["pixel"],
                                           C=cfg["C"])
    xy32 = xy.astype(np.float32)
    out = M.smooth_loops(off, eid, xy32, x0=cfg["x0"], y0=cfg["y0"], pixel=cfg["pixel"],
                         nx=cfg["nx"], lam=0.3, margin=0.5, iterations=1)
    W = cfg["nx"] + 2
    for v in range(len(eid)):
        axis, lo = M.edge_axis_and_lo(int(eid[v]), W, cfg["x0"], cfg["y0"], cfg["pixel"])
        mid = lo + 0.5 * cfg["pixel"]
        # the midpoint in FP64, up to the float32 roundings of the bound (c0, the
        # product, two sums: at most 2 ulp of the coordinate)
        ulp = float(np.spacing(np.float32(abs(mid) + cfg["pixel"])))
        assert abs(float(out[v, axis]) - mid) <= 2.0 * ulp
        assert out[v, 1 - axis] == xy32[v, 1 - axis]


def test_straight_side_is_a_fixed_point():
    """An inside rectangle of 6 columns and 40 rows: its right side crosses
    the row edges at their midpoints (x = 6). Both neighbours of such a vertex
    sit on the same vertical line, so it stays put until the moves that start
    at the corners reach it, one vertex per Jacobi iteration: after K = 6
    iterations the side's vertices 7 or more rows from either end are
    unchanged, whatever lam."""
    ny, nx = 40, 10
    s = np.zeros((ny, nx))
    s[:, :6] = 2.0
    off, eid, xy = _one_layer(s)
    xy32 = xy.astype(np.float32)
    out = M.smooth_loops(off, eid, xy32, x0=0.0, y0=0.0, pixel=1.0, nx=nx, lam=0.7, margin=0.05,
                         iterations=6)
    side = np.isclose(xy32[:, 0], 6.0)
    assert side.sum() == ny
    far = np.nonzero(side & (xy32[:, 1] > 7.0) & (xy32[:, 1] < ny - 7.0))[0]
    assert len(far) == ny - 14
    assert np.array_equal(out[far], xy32[far])
    near = np.nonzero(side & (xy32[:, 1] < 1.0))[0]
    assert len(near) == 1 and out[near[0], 0] < 6.0   # the corner's neighbour moved inwards
    assert out[near[0], 1] == xy32[near[0], 1]
    # one iteration by hand: its neighbours are the side's next vertex (x = 6)
    # and the bottom side's first one, on the vertical edge at x = 5.5, so
    # x becomes 6 + 0.7 (5.75 - 6)
    one = M.smooth_loops(off, eid, xy32, x0=0.0, y0=0.0, pixel=1.0, nx=nx, lam=0.7, margin=0.05,
                         iterations=1)
    assert one[near[0], 0] == np.float32(6.0 + 0.7 * (5.75 - 6.0))


def test_identities():
    s = np.zeros((6, 6))
    s[1:4, 2:5] = [[1.5, 2.0, 1.2], [2.5, 3.0, 1.7], [1.1, 1.9, 1.4]]
    off, eid, xy = _one_layer(s)
    xy32 = xy.astype(np.float32)
    kw = dict(x0=0.0, y0=0.0, pixel=1.0, nx=6)
    assert np.array_equal(M.smooth_loops(off, eid, xy32, lam=0.5, margin=0.05, iterations=0,
                                         **kw), xy32)
    # lam = 0 leaves every vertex that already lies inside the margin
    out = M.smooth_loops(off, eid, xy32, lam=0.0, margin=1e-3, iterations=4, **kw)
    assert np.array_equal(out, xy32)


@pytest.mark.parametrize("k,simplify", [(3, False), (11, False), (11, True)])
def test_loops_stay_on_their_edges_and_do_not_cross(k, simplify):
    cfg = synth.config(1)
    sig = oracle.slice_sigma(cfg["nodes"], cfg["edges"], cfg["radius"], R=cfg["R"], C=cfg["C"],
                             z0=cfg["z0"] + k * cfg["dz"], dz=cfg["dz"], n_layers=1,
                             x0=cfg["x0"], y0=cfg["y0"], nx=cfg["nx"], ny=cfg["ny"],
                             pixel=cfg["pixel"])[0]
    off, eid, xy = oracle.marching_squares(sig, x0=cfg["x0"], y0=cfg["y0"], pixel=cfg["pixel"],
                                           C=cfg["C"])
    xy32 = xy.astype(np.float32)
    if simplify:
        off, eid, xy32, _ = Z.simplify_layer(off, eid, xy32, cfg["nx"], 0.3 * cfg["pixel"])
    mu = 0.05
    out = M.smooth_loops(off, eid, xy32, x0=cfg["x0"], y0=cfg["y0"], pixel=cfg["pixel"],
                         nx=cfg["nx"], lam=0.5, margin=mu, iterations=10)
    W = cfg["nx"] + 2
    for v in range(len(eid)):
        axis, lo = M.edge_axis_and_lo(int(eid[v]), W, cfg["x0"], cfg["y0"], cfg["pixel"])
        assert out[v, 1 - axis] == xy32[v, 1 - axis]
        # inside the margin up to the float32 roundings of the bounds (2 ulp),
        # strictly inside the edge (what keeps every segment in its cell)
        a = float(out[v, axis])
        ulp = float(np.spacing(np.float32(abs(lo) + cfg["pixel"])))
        assert lo + mu * cfg["pixel"] - 2.0 * ulp <= a <= lo + (1.0 - mu) * cfg["pixel"] + 2.0 * ulp
        assert lo < a < lo + cfg["pixel"]
    moved = np.any(out != xy32, axis=1)
    assert moved.sum() > 0.5 * len(eid)
    assert _crossings(*_segments(off, out)) == 0
