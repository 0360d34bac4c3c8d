"""Contour simplification on the GPU (csl_simplify_contours) against the
oracle's rule applied to the same input loops: the same vertices kept (the
decisions are FP64 on the same float inputs), and no crossings."""
import numpy as np
import pytest

import synth
from oracle import simplify as Z
from tests.helpers import oracle_contour_set
from tests.test_oracle_simplify import _crossings, _segments

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _layer_arrays(cset, k):
    l0, l1 = int(cset.layer_loop_off[k]), int(cset.layer_loop_off[k + 1])
    v0, v1 = int(cset.loop_vert_off[l0]), int(cset.loop_vert_off[l1])
    return cset.loop_vert_off[l0:l1 + 1] - v0, cset.edge_id[v0:v1], cset.xy[v0:v1]


def test_simplify_matches_the_oracle_rule():
    """The input is the oracle's own marching-squares contours of 12 layers
    (float32), uploaded with csl_contours_create."""
    import paper_2101_05031_gb300 as cs
    cfg = synth.config(1)
    n = 12
    lo, vo, xy_all, eid_all = oracle_contour_set(cfg, range(n))
    src = cs.ContourSet(lo, vo, xy_all, eid_all)
    dev = cs.DeviceContours.from_host(lo, vo, xy_all, eid_all)
    tol = 0.3 * cfg["pixel"]
    out = dev.simplify(cfg["nx"], cfg["ny"], tol).to_host()
    assert np.array_equal(out.layer_loop_off, src.layer_loop_off)
    total_in = total_out = 0
    for k in range(n):
        off, eid, xy = _layer_arrays(src, k)
        goff, geid, gxy = _layer_arrays(out, k)
        roff, reid, rxy, _ = Z.simplify_layer(off, eid, xy, cfg["nx"], tol)
        assert np.array_equal(goff, roff), k
        assert np.array_equal(geid, reid), k
        assert np.array_equal(gxy, rxy), k
        total_in += len(eid)
        total_out += len(reid)
        if k in (3, 9):
            assert _crossings(*_segments(goff, gxy)) == 0
    assert total_out < 0.9 * total_in


def test_simplify_arguments_and_empty_input():
    import paper_2101_05031_gb300 as cs
    cfg = synth.config(1)
    lat = cs.Lattice(cfg["nodes"], cfg["edges"], cfg["radius"], R=cfg["R"])
    kw = dict(z0=cfg["z0"], dz=cfg["dz"], x0=cfg["x0"], y0=cfg["y0"], nx=cfg["nx"], ny=cfg["ny"],
              pixel=cfg["pixel"], on_device=True)
    no_ids = lat.slice(n_layers=2, **kw)
    with pytest.raises(cs.CslError):
        no_ids.simplify(cfg["nx"], cfg["ny"], 0.01)
    empty = lat.slice(n_layers=0, edge_ids=True, **kw)
    out = empty.simplify(cfg["nx"], cfg["ny"], 0.01)
    assert out.n_loops == 0 and out.n_verts == 0


def _check_rule_properties(off, eid, xy, goff, geid, gxy, tol):
    """What the rule implies for one layer, from its input and output alone:
    the kept vertices are a subsequence with the loop heads, every loop keeps
    at least 3 (or all) vertices, and every dropped vertex sat at an odd
    position of a loop of at least 5, between two kept vertices, within tol of
    their chord."""
    assert len(goff) == len(off)
    keep = np.isin(eid, geid)            # one crossing per grid edge in a layer
    assert keep.sum() == len(geid)
    assert np.array_equal(eid[keep], geid) and np.array_equal(xy[keep], gxy)
    n = np.diff(off)
    assert np.array_equal(np.diff(goff), [k.sum() for k in np.split(keep, off[1:-1])])
    assert np.all(keep[off[:-1][n > 0]])
    assert np.all(np.diff(goff) >= np.minimum(n, 3))
    loop = np.repeat(np.arange(len(n)), n)
    q = np.arange(len(eid)) - off[:-1][loop]
    drop = np.nonzero(~keep)[0]
    assert np.all(q[drop] % 2 == 1) and np.all(n[loop[drop]] >= 5)
    prv = off[:-1][loop[drop]] + (q[drop] - 1)
    nxt = off[:-1][loop[drop]] + (q[drop] + 1) % n[loop[drop]]
    assert np.all(keep[prv]) and np.all(keep[nxt])
    a, b, v = (xy[prv].astype(np.float64), xy[nxt].astype(np.float64),
               xy[drop].astype(np.float64))
    d = b - a
    cross = (v[:, 0] - a[:, 0]) * d[:, 1] - (v[:, 1] - a[:, 1]) * d[:, 0]
    assert np.all(np.abs(cross) <= tol * np.hypot(d[:, 0], d[:, 1]) * (1 + 1e-12))


def test_full_grid_layers_of_the_10M_workload():
    """20 layers of the 10M-strut graded lattice at its full 2000 x 2000 grid,
    simplified as the benchmark does (0.25 px): on two sampled layers, what
    the rule implies, checked from the input and the output alone."""
    import paper_2101_05031_gb300 as cs
    nodes, edges, radius, r_ref = synth.adaptive_graded(box=100.0, level_min=4, level_max=7)
    lat = cs.Lattice(nodes, edges, radius, R=1.5 * r_ref, C=1.0)
    nx = ny = 2000
    pixel = 0.05
    dev = lat.slice(z0=40.1, dz=0.2, n_layers=20, x0=0.0, y0=0.0, nx=nx, ny=ny, pixel=pixel,
                    on_device=True, edge_ids=True)
    src = dev.to_host()
    out = dev.simplify(nx, ny, 0.25 * pixel).to_host()
    for k in (4, 17):
        off, eid, xy = _layer_arrays(src, k)
        goff, geid, gxy = _layer_arrays(out, k)
        _check_rule_properties(off, eid, xy, goff, geid, gxy, 0.25 * pixel)
        assert len(geid) < 0.8 * len(eid)
