"""Zigzag infill on the GPU (csl_hatch_layers) against the reference hatcher
applied to the same contours (the oracle's own, uploaded), and, on the GPU's
slices, against the oracle's field."""
import numpy as np
import pytest

import oracle
import synth
from oracle import hatch
from tests.helpers import oracle_contour_set

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _c1_contours(n_layers=50):
    import paper_2101_05031_gb300 as cs
    cfg = synth.config(1)
    lat = cs.Lattice(cfg["nodes"], cfg["edges"], cfg["radius"], R=cfg["R"], C=cfg["C"])
    dev = lat.slice(z0=cfg["z0"], dz=cfg["dz"], n_layers=n_layers, x0=cfg["x0"], y0=cfg["y0"],
                    nx=cfg["nx"], ny=cfg["ny"], pixel=cfg["pixel"], on_device=True,
                    chunk_layers=16, slab=8)
    return cfg, lat, dev


def test_hatch_matches_reference_on_the_same_contours():
    """The input is the oracle's own marching-squares contours of 50 layers
    (float32), uploaded with csl_contours_create."""
    import paper_2101_05031_gb300 as cs
    cfg = synth.config(1)
    lo, vo, xy, eid = oracle_contour_set(cfg, range(50))
    dev = cs.DeviceContours.from_host(lo, vo, xy, eid)
    y0, sp, n_lines = cfg["y0"] + 0.025, 0.25, 80
    off, seg = dev.hatch(y0, sp, n_lines)
    roff, rseg = hatch.hatch_contours(lo, vo, xy, y0, sp, n_lines)
    assert np.array_equal(off, roff)
    assert seg.shape == rseg.shape and len(seg) > 1000
    assert np.array_equal(seg[:, 2].astype(np.float64), rseg[:, 2])   # the same float32 lines
    assert np.max(np.abs(seg[:, :2] - rseg[:, :2])) <= 1e-4          # FP32 vs FP64 abscissae


def test_hatch_segments_lie_inside_the_solid():
    """Midpoints of the segments longer than two pixels have Sigma >= C by the
    oracle's field (up to the contour tolerance)."""
    cfg, lat, dev = _c1_contours(n_layers=10)
    y0, sp, n_lines = cfg["y0"] + 0.025, 0.5, 40
    off, seg = dev.hatch(y0, sp, n_lines)
    r = np.random.default_rng(5)
    pts = []
    for k in range(10):
        z = cfg["z0"] + k * cfg["dz"]
        s = seg[off[k]:off[k + 1]]
        s = s[np.abs(s[:, 1] - s[:, 0]) > 2 * cfg["pixel"]]
        pick = s[r.choice(len(s), min(20, len(s)), replace=False)]
        for x0_, x1_, y in pick:
            pts.append((0.5 * (x0_ + x1_), y, z))
    pts = np.array(pts, np.float64)
    sig = oracle.sigma_points(cfg["nodes"], cfg["edges"], cfg["radius"], pts, R=cfg["R"],
                              C=cfg["C"])
    assert np.all(sig >= cfg["C"] * (1 - 1e-3))


def test_hatch_empty_and_errors():
    import paper_2101_05031_gb300 as cs
    cfg, lat, dev = _c1_contours(n_layers=2)
    off, seg = dev.hatch(-100.0, 1.0, 3)   # lines below the part
    assert list(off) == [0, 0, 0] and seg.shape == (0, 3)
    with pytest.raises(cs.CslError):
        dev.hatch(0.0, 0.0, 3)
    with pytest.raises(cs.CslError):
        dev.hatch(float("nan"), 1.0, 3)
