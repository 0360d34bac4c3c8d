"""Depth images of the implicit solid (csl_render_depth) against the FP64
ray-casting oracle, and against the exact cylinder of an isolated strut."""
import math

import numpy as np
import pytest

import synth
from oracle import render as V

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_isolated_strut_cylinder():
    import paper_2101_05031_gb300 as cs
    rho, R = 0.3, 0.45
    nodes = np.array([[0, 0, -20], [0, 0, 20]], np.float32)
    lat = cs.Lattice(nodes, np.array([[0, 1]], np.int32), np.array([rho], np.float32), R=R)
    # looking along -y from y = 5 at the axis: the centre column's rays hit x^2 + y^2 = rho^2
    w, h = 9, 7
    depth = lat.render_depth(eye=(0.0, 5.0, 1.0), target=(0.0, 0.0, 1.0), up=(0.0, 0.0, 1.0),
                             fov_y=0.2, width=w, height=h, step=0.01, refine=24).cpu().numpy()
    o, d = V.camera_rays((0.0, 5.0, 1.0), (0.0, 0.0, 1.0), (0.0, 0.0, 1.0), 0.2, w, h)
    r32 = float(np.float32(rho))
    for j in range(h):
        for i in range(w):
            ray = d[j, i]
            # distance to the axis along the ray: solve |(o + t d)_xy| = rho
            a = ray[0] ** 2 + ray[1] ** 2
            b = 2 * (o[0] * ray[0] + o[1] * ray[1])
            c = o[0] ** 2 + o[1] ** 2 - r32 ** 2
            disc = b * b - 4 * a * c
            if disc > 0.05:
                t = (-b - math.sqrt(disc)) / (2 * a)
                assert abs(depth[j, i] - t) <= 2e-4, (j, i, depth[j, i], t)
            elif disc < -0.05:
                assert np.isinf(depth[j, i])


def test_cubic_bcc_against_the_oracle():
    import paper_2101_05031_gb300 as cs
    cfg = synth.config(1)
    lat = cs.Lattice(cfg["nodes"], cfg["edges"], cfg["radius"], R=cfg["R"])
    cam = dict(eye=(31.0, -17.0, 24.0), target=(10.0, 10.0, 9.0), up=(0.0, 0.0, 1.0),
               fov_y=0.9, width=32, height=24)
    step = 0.05
    depth = lat.render_depth(**cam, step=step, refine=20).cpu().numpy()
    ref = V.render(cfg["nodes"], cfg["edges"], cfg["radius"], R=cfg["R"], C=1.0, step=step,
                   refine=20, **cam)
    n_hit = n_bad = 0
    for (j, i), t in ref.items():
        g = depth[j, i]
        if np.isinf(t) and np.isinf(g):
            continue
        n_hit += not np.isinf(t)
        # a sample whose field sits at C within rounding can decide the other way
        if not (abs(g - t) <= 2e-3):
            n_bad += 1
    assert n_hit > 100
    assert n_bad <= 0.01 * len(ref), n_bad


def test_full_workload_sampled_rays():
    """The bench's image (430k-strut Freudenthal lattice, 1920 x 1080, step
    R/8): 40 sampled pixels against the oracle, ray by ray."""
    import paper_2101_05031_gb300 as cs
    cfg = synth.config(2)
    lat = cs.Lattice(cfg["nodes"], cfg["edges"], cfg["radius"], R=cfg["R"], C=cfg["C"])
    lo, hi = synth.lattice_bbox(cfg["nodes"])
    c = 0.5 * (lo + hi)
    ext = float(np.max(hi - lo))
    cam = dict(eye=(float(c[0] + 1.1 * ext), float(c[1] - 0.8 * ext), float(c[2] + 0.7 * ext)),
               target=(float(c[0]), float(c[1]), float(c[2])), up=(0.0, 0.0, 1.0), fov_y=0.6,
               width=1920, height=1080)
    step = cfg["R"] / 8
    depth = lat.render_depth(**cam, step=step, refine=20).cpu().numpy()
    r = synth.rng(29)
    pix = [(int(r.integers(1080)), int(r.integers(1920))) for _ in range(40)]
    ref = V.render(cfg["nodes"], cfg["edges"], cfg["radius"], R=cfg["R"], step=step, refine=20,
                   pixels=pix, **cam)
    n_hit = n_bad = 0
    for (j, i), t in ref.items():
        g = depth[j, i]
        if np.isinf(t) and np.isinf(g):
            continue
        n_hit += 1
        n_bad += not (abs(g - t) <= 2e-3)
    assert n_hit >= 20
    assert n_bad <= 1, n_bad


def test_edge_cases_of_the_ray_march():
    """Rays that point away from the lattice miss; rays that start inside the
    solid stop at their first sample (depth 0, reading V2 with t_in = 0); a
    lattice without struts gives +inf everywhere; a step that would need more
    than 2^24 samples across the box is rejected before any launch."""
    import paper_2101_05031_gb300 as cs
    rho, R = 0.3, 0.45
    nodes = np.array([[0, 0, -20], [0, 0, 20]], np.float32)
    lat = cs.Lattice(nodes, np.array([[0, 1]], np.int32), np.array([rho], np.float32), R=R)
    away = lat.render_depth(eye=(0.0, 5.0, 1.0), target=(0.0, 10.0, 1.0), up=(0.0, 0.0, 1.0),
                            fov_y=0.2, width=5, height=3, step=0.01).cpu().numpy()
    assert np.all(np.isinf(away))
    inside = lat.render_depth(eye=(0.0, 0.0, 1.0), target=(1.0, 0.0, 1.0), up=(0.0, 0.0, 1.0),
                              fov_y=0.5, width=4, height=4, step=0.01).cpu().numpy()
    assert np.all(inside == 0.0)
    ref = V.render(nodes, np.array([[0, 1]], np.int32), np.array([rho], np.float32), R=R,
                   eye=(0.0, 0.0, 1.0), target=(1.0, 0.0, 1.0), up=(0.0, 0.0, 1.0), fov_y=0.5,
                   width=4, height=4, step=0.01, pixels=[(0, 0), (2, 1)])
    assert all(t == 0.0 for t in ref.values())
    empty = cs.Lattice(nodes, np.zeros((0, 2), np.int32), np.zeros(0, np.float32), R=R)
    e = empty.render_depth(eye=(0.0, 5.0, 1.0), target=(0.0, 0.0, 1.0), width=3, height=2,
                           step=0.01).cpu().numpy()
    assert np.all(np.isinf(e))
    with pytest.raises(cs.CslError) as err:
        lat.render_depth(eye=(0.0, 5.0, 1.0), target=(0.0, 0.0, 1.0), width=3, height=2,
                         step=1e-7)
    assert err.value.code == 1
