"""Pins of the contour simplification oracle: on real marching-squares loops,
no two segments of the simplified layer cross (checked by brute force over
all segment pairs), the loops keep their order, heads and at least three
vertices, removed vertices lie within the tolerance of their chord, an
isolated disc loses exactly every other vertex, and vertices beside a saddle
cell stay."""
import numpy as np
import pytest

import oracle
import synth
from oracle import simplify as Z


def _segments(loop_off, xy):
    a, b = [], []
    for L in range(len(loop_off) - 1):
        s, e = int(loop_off[L]), int(loop_off[L + 1])
        pts = xy[s:e]
        a.append(pts)
        b.append(np.roll(pts, -1, axis=0))
    return np.concatenate(a), np.concatenate(b)


def _crossings(p, q):
    """Pairs of segments that properly cross (shared end points excluded)."""
    p = p.astype(np.float64)
    q = q.astype(np.float64)

    def orient(a, b, c):
        return (b[..., 0] - a[..., 0]) * (c[..., 1] - a[..., 1]) - \
               (b[..., 1] - a[..., 1]) * (c[..., 0] - a[..., 0])

    P1, P2 = p[:, None, :], q[:, None, :]
    Q1, Q2 = p[None, :, :], q[None, :, :]
    d1, d2 = orient(P1, P2, Q1), orient(P1, P2, Q2)
    d3, d4 = orient(Q1, Q2, P1), orient(Q1, Q2, P2)
    cross = (d1 * d2 < 0) & (d3 * d4 < 0)
    return int(np.triu(cross, 1).sum())


def _layer(cfg, k):
    s = oracle.slice_sigma(cfg["nodes"], cfg["edges"], cfg["radius"], R=cfg["R"], C=cfg["C"],
                           z0=cfg["z0"] + k * cfg["dz"], dz=cfg["dz"], n_layers=1, x0=cfg["x0"],
                           y0=cfg["y0"], nx=cfg["nx"], ny=cfg["ny"], pixel=cfg["pixel"])[0]
    return oracle.marching_squares(s, x0=cfg["x0"], y0=cfg["y0"], pixel=cfg["pixel"], C=cfg["C"])


@pytest.mark.parametrize("k", [3, 11])
def test_simplified_layers_do_not_cross(k):
    cfg = synth.config(1)
    off, eid, xy = _layer(cfg, k)
    tol = 0.3 * cfg["pixel"]
    noff, neid, nxy, keep = Z.simplify_layer(off, eid, xy, cfg["nx"], tol)
    assert len(noff) == len(off)
    assert _crossings(*_segments(off, xy)) == 0          # marching squares' own loops
    assert _crossings(*_segments(noff, nxy)) == 0
    removed = int((~keep).sum())
    assert removed > 0.1 * len(eid)
    for L in range(len(off) - 1):
        a, b = int(off[L]), int(off[L + 1])
        assert keep[a]                                     # the head stays
        assert int(noff[L + 1] - noff[L]) >= min(3, b - a)
        # removed vertices lie within tol of the chord of their kept neighbours
        idx = np.arange(a, b)
        for q in np.nonzero(~keep[a:b])[0]:
            p0, p1 = xy[idx[q - 1]], xy[idx[(q + 1) % (b - a)]]
            v = xy[idx[q]]
            d = p1 - p0
            dist = abs((v[0] - p0[0]) * d[1] - (v[1] - p0[1]) * d[0]) / np.hypot(*d)
            assert dist <= tol * (1 + 1e-12)
            assert keep[idx[q - 1]] and keep[idx[(q + 1) % (b - a)]]


def test_isolated_disc_loses_every_other_vertex():
    rho, R = 0.6, 0.9
    nodes = np.array([[5, 5, -20], [5, 5, 20]], np.float32)
    s = oracle.slice_sigma(nodes, np.array([[0, 1]], np.int32), np.array([rho], np.float32),
                           R=R, C=1.0, z0=0.0, dz=1.0, n_layers=1, x0=0.0, y0=0.0, nx=100, ny=100,
                           pixel=0.1)[0]
    off, eid, xy = oracle.marching_squares(s, x0=0.0, y0=0.0, pixel=0.1, C=1.0)
    assert len(off) == 2
    n = int(off[1])
    noff, _, _, _ = Z.simplify_layer(off, eid, xy, 100, 1e9)
    assert int(noff[1]) == n - n // 2
    noff, _, _, _ = Z.simplify_layer(off, eid, xy, 100, 0.0)
    assert int(noff[1]) == n                               # a circle has no collinear triple


def test_saddle_neighbours_stay():
    """Two touching squares whose corners meet in a saddle cell (the saddle
    joins them, so it is one loop): the two vertices on the saddle cell's
    edges are never dropped, however large the tolerance."""
    s = np.zeros((12, 12))
    s[2:6, 2:6] = 2.0
    s[6:10, 6:10] = 2.0
    s[5, 6] = s[6, 5] = 0.2                   # the saddle cell (5..6, 5..6): diagonal inside corners
    off, eid, xy = oracle.marching_squares(s, x0=0.0, y0=0.0, pixel=1.0, C=1.0)
    noff, neid, nxy, keep = Z.simplify_layer(off, eid, xy, 12, 1e9)
    W = 14
    saddle_edges = set(Z.cell_edges(6, 6, W))            # padded cell of samples (5..6, 5..6)
    on_saddle = [i for i, e in enumerate(eid) if int(e) in saddle_edges]
    assert len(on_saddle) == 4
    for i in on_saddle:
        assert keep[i]
    assert _crossings(*_segments(noff, nxy)) == 0
