"""Contour simplification on the GPU (csl_simplify_contours) against the
oracle's rule applied to the same input loops: the same vertices kept (the
decisions are FP64 on the same float inputs), and no crossings."""
import numpy as np
import pytest

import synth
from oracle import simplify as Z
from tests.test_oracle_simplify import _crossings, _segments

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _layer_arrays(cset, k):
    l0, l1 = int(cset.layer_loop_off[k]), int(cset.layer_loop_off[k + 1])
    v0, v1 = int(cset.loop_vert_off[l0]), int(cset.loop_vert_off[l1])
    return cset.loop_vert_off[l0:l1 + 1] - v0, cset.edge_id[v0:v1], cset.xy[v0:v1]


def test_simplify_matches_the_oracle_rule():
    import paper_2101_05031_gb300 as cs
    cfg = synth.config(1)
    lat = cs.Lattice(cfg["nodes"], cfg["edges"], cfg["radius"], R=cfg["R"])
    n = 12
    dev = lat.slice(z0=cfg["z0"], dz=cfg["dz"], n_layers=n, x0=cfg["x0"], y0=cfg["y0"],
                    nx=cfg["nx"], ny=cfg["ny"], pixel=cfg["pixel"], on_device=True, edge_ids=True)
    src = dev.to_host()
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


def test_full_grid_layers_of_the_10M_workload():
    """20 layers of the 10M-strut graded lattice at its full 2000 x 2000 grid,
    simplified as the benchmark does (0.25 px): two sampled layers against the
    oracle's rule, one of them checked for crossings."""
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
        roff, reid, rxy, _ = Z.simplify_layer(off, eid, xy, nx, 0.25 * pixel)
        assert np.array_equal(goff, roff) and np.array_equal(geid, reid)
        assert np.array_equal(gxy, rxy)
        assert len(reid) < 0.8 * len(eid)
