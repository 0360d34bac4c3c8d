"""Contour smoothing on the GPU (csl_smooth_contours) against the oracle's
operator on the same input: the oracle's own marching-squares contours of the
cubic+BCC lattice (float32), uploaded with csl_contours_create. Both sides do
the arithmetic in float32, each operation rounded on its own in one fixed
order, so the vertices agree bit for bit.
At full size (the 10M-strut workload's contours) the properties that make
the operator topology-preserving are checked on every vertex."""
import numpy as np
import pytest

import synth
from oracle import simplify as Z
from oracle import smooth as M
from tests.helpers import layer_arrays, oracle_contour_set
from tests.test_oracle_simplify import _crossings, _segments

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

LAYERS = (2, 5, 11, 17)


@pytest.fixture(scope="module")
def c1_set():
    cfg = synth.config(1)
    return cfg, oracle_contour_set(cfg, LAYERS)


def _geom(cfg):
    return dict(x0=cfg["x0"], y0=cfg["y0"], pixel=cfg["pixel"], nx=cfg["nx"])


def test_smooth_matches_the_oracle(c1_set):
    import paper_2101_05031_gb300 as cs
    cfg, (lo, vo, xy, eid) = c1_set
    dev = cs.DeviceContours.from_host(lo, vo, xy, eid)
    dev.smooth(cfg["x0"], cfg["y0"], cfg["pixel"], cfg["nx"], cfg["ny"], lam=0.5, margin=0.05,
               iterations=7)
    out = dev.to_host()
    assert np.array_equal(out.layer_loop_off, lo) and np.array_equal(out.loop_vert_off, vo)
    assert np.array_equal(out.edge_id, eid)
    ref = M.smooth_loops(vo, eid, xy, lam=0.5, margin=0.05, iterations=7, **_geom(cfg))
    assert np.array_equal(out.xy, ref)
    assert np.sum(np.any(out.xy != xy, axis=1)) > 0.5 * len(eid)
    for k in range(len(LAYERS)):
        off, _, lxy = layer_arrays(lo, vo, out.xy, eid, k)
        assert _crossings(*_segments(off, lxy)) == 0


def test_simplify_then_smooth_matches_the_oracle(c1_set):
    import paper_2101_05031_gb300 as cs
    cfg, (lo, vo, xy, eid) = c1_set
    tol = 0.3 * cfg["pixel"]
    dev = cs.DeviceContours.from_host(lo, vo, xy, eid)
    simp = dev.simplify(cfg["nx"], cfg["ny"], tol)
    simp.smooth(cfg["x0"], cfg["y0"], cfg["pixel"], cfg["nx"], cfg["ny"], lam=0.3, margin=0.1,
                iterations=5)
    out = simp.to_host()
    for k in range(len(LAYERS)):
        off, leid, lxy = layer_arrays(lo, vo, xy, eid, k)
        roff, reid, rxy, _ = Z.simplify_layer(off, leid, lxy, cfg["nx"], tol)
        ref = M.smooth_loops(roff, reid, rxy, lam=0.3, margin=0.1, iterations=5, **_geom(cfg))
        goff, geid, gxy = layer_arrays(out.layer_loop_off, out.loop_vert_off, out.xy,
                                       out.edge_id, k)
        assert np.array_equal(goff, roff) and np.array_equal(geid, reid)
        assert np.array_equal(gxy, ref), k
        assert _crossings(*_segments(goff, gxy)) == 0


def test_identities_edge_cases_and_errors(c1_set):
    import paper_2101_05031_gb300 as cs
    cfg, (lo, vo, xy, eid) = c1_set
    dev = cs.DeviceContours.from_host(lo, vo, xy, eid)
    dev.smooth(cfg["x0"], cfg["y0"], cfg["pixel"], cfg["nx"], cfg["ny"], iterations=0)
    assert np.array_equal(dev.to_host().xy, xy)
    # margin 1/2: every vertex at its edge's midpoint (binary-image marching squares)
    dev.smooth(cfg["x0"], cfg["y0"], cfg["pixel"], cfg["nx"], cfg["ny"], lam=0.2, margin=0.5,
               iterations=1)
    ref = M.smooth_loops(vo, eid, xy, lam=0.2, margin=0.5, iterations=1, **_geom(cfg))
    assert np.array_equal(dev.to_host().xy, ref)
    # edge ids of a larger grid than the one given: rejected, nothing changed
    fresh = cs.DeviceContours.from_host(lo, vo, xy, eid)
    with pytest.raises(cs.CslError) as err:
        fresh.smooth(cfg["x0"], cfg["y0"], cfg["pixel"], 20, 20)
    assert err.value.code == 1
    assert np.array_equal(fresh.to_host().xy, xy)
    with pytest.raises(cs.CslError) as err:
        fresh.simplify(20, 20, 0.01)
    assert err.value.code == 1
    # contours without edge ids, and empty ones
    with pytest.raises(cs.CslError):
        cs.DeviceContours.from_host(lo, vo, xy).smooth(0.0, 0.0, 0.1, cfg["nx"], cfg["ny"])
    empty = cs.DeviceContours.from_host(np.zeros(3, np.int64), np.zeros(1, np.int64),
                                        np.zeros((0, 2), np.float32), np.zeros(0, np.int32))
    empty.smooth(0.0, 0.0, 0.1, 10, 10)
    assert empty.n_verts == 0 and len(empty.to_host().xy) == 0
    assert empty.simplify(10, 10, 0.01).n_loops == 0


def _edge_geometry(eid, nx, x0, y0, px):
    e = np.asarray(eid, dtype=np.int64)
    base, vert = e >> 1, (e & 1).astype(bool)
    W = nx + 2
    J, I = base // W, base % W
    lo = np.where(vert, y0 + (J.astype(np.float64) - 0.5) * px,
                  x0 + (I.astype(np.float64) - 0.5) * px)
    return vert, lo


def test_full_grid_layers_of_the_10M_workload():
    """20 layers of the 10M-strut graded lattice at its full 2000 x 2000
    grid, smoothed as the benchmark does: every vertex keeps its fixed
    coordinate and its free one stays inside its edge's margin, edge ids and
    offsets are untouched, and a window of one layer has no crossing."""
    import paper_2101_05031_gb300 as cs
    nodes, edges, radius, r_ref = synth.adaptive_graded(box=100.0, level_min=4, level_max=7)
    lat = cs.Lattice(nodes, edges, radius, R=1.5 * r_ref, C=1.0)
    nx = ny = 2000
    pixel, mu = 0.05, 0.05
    dev = lat.slice(z0=40.1, dz=0.2, n_layers=20, x0=0.0, y0=0.0, nx=nx, ny=ny, pixel=pixel,
                    on_device=True, edge_ids=True)
    src = dev.to_host()
    dev.smooth(0.0, 0.0, pixel, nx, ny, lam=0.5, margin=mu, iterations=4)
    out = dev.to_host()
    assert np.array_equal(out.loop_vert_off, src.loop_vert_off)
    assert np.array_equal(out.edge_id, src.edge_id)
    vert, lo = _edge_geometry(src.edge_id, nx, 0.0, 0.0, pixel)
    free = np.where(vert, out.xy[:, 1], out.xy[:, 0])
    fixed_in = np.where(vert, src.xy[:, 0], src.xy[:, 1])
    fixed_out = np.where(vert, out.xy[:, 0], out.xy[:, 1])
    assert np.array_equal(fixed_in, fixed_out)
    # inside the margin up to the float32 roundings of the bounds; strictly
    # inside the edge
    ulp = np.spacing((np.abs(lo) + pixel).astype(np.float32)).astype(np.float64)
    f64 = free.astype(np.float64)
    assert np.all(f64 >= lo + mu * pixel - 2.0 * ulp)
    assert np.all(f64 <= lo + (1.0 - mu) * pixel + 2.0 * ulp)
    assert np.all((f64 > lo) & (f64 < lo + pixel))
    assert np.mean(np.any(out.xy != src.xy, axis=1)) > 0.5
    # a 3 x 3 mm window of layer 9: the loops that lie wholly inside it
    k = 9
    off, _, lxy = layer_arrays(out.layer_loop_off, out.loop_vert_off, out.xy, out.edge_id, k)
    keep = []
    for L in range(len(off) - 1):
        pts = lxy[off[L]:off[L + 1]]
        if np.all((pts >= 40.0) & (pts <= 43.0)):
            keep.append(L)
    assert len(keep) > 5
    woff = np.concatenate([[0], np.cumsum([off[L + 1] - off[L] for L in keep])])
    wxy = np.concatenate([lxy[off[L]:off[L + 1]] for L in keep])
    assert _crossings(*_segments(woff, wxy)) == 0
