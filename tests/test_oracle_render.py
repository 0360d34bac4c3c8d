"""Pins of the ray-casting oracle: camera geometry, the box interval, and the
exact cylinder an isolated long strut's surface forms (PHYSICAL weights put
it at the strut radius, Sec. 3.2)."""
import math

import numpy as np

from oracle import render as V


def test_camera_rays_are_unit_and_centred():
    o, d = V.camera_rays((0, 0, 10), (0, 0, 0), (0, 1, 0), math.radians(40), 5, 3)
    assert np.allclose(np.linalg.norm(d, axis=2), 1.0)
    assert np.allclose(d[1, 2], [0, 0, -1])                     # the centre pixel
    # the top row's vertical angle: (1 - 0.5 / 3 * 2) of tan(fov / 2)
    y = d[0, 2, 1] / -d[0, 2, 2]
    assert abs(y - (1 - 1.0 / 3) * math.tan(math.radians(20))) <= 1e-12
    x = d[1, 4, 0] / -d[1, 4, 2]
    assert abs(x - (0.8 * math.tan(math.radians(20)) * 5 / 3)) <= 1e-12


def test_box_interval():
    lo, hi = np.array([0.0, 0.0, 0.0]), np.array([1.0, 2.0, 3.0])
    t = V.box_interval(np.array([-1.0, 1.0, 1.0]), np.array([1.0, 0.0, 0.0]), lo, hi)
    assert t == (1.0, 2.0)
    assert V.box_interval(np.array([-1.0, 3.0, 1.0]), np.array([1.0, 0.0, 0.0]), lo, hi) is None
    t = V.box_interval(np.array([0.5, 1.0, 1.0]), np.array([0.0, 0.0, 1.0]), lo, hi)
    assert t == (0.0, 2.0)


def test_isolated_strut_is_hit_on_its_cylinder():
    rho, R = 0.3, 0.45
    nodes = np.array([[0, 0, -20], [0, 0, 20]], np.float32)
    edges = np.array([[0, 1]], np.int32)
    radius = np.array([rho], np.float32)
    lo = nodes.min(0).astype(np.float64) - R
    hi = nodes.max(0).astype(np.float64) + R
    d = np.array([1.0, 0.0, 0.0])
    for b in (0.0, 0.1, 0.2, 0.28):
        o = np.array([-5.0, b, 1.0])
        t = V.cast(nodes, edges, radius, o, d, R=R, step=0.02, refine=30, lo=lo, hi=hi)
        assert abs(t - (5.0 - math.sqrt(float(np.float32(rho)) ** 2 - b * b))) <= 1e-6, b
    o = np.array([-5.0, 0.31, 1.0])
    assert V.cast(nodes, edges, radius, o, d, R=R, step=0.02, lo=lo, hi=hi) == math.inf
    # a ray along the axis from above enters the rounded end cap first
    t = V.cast(nodes, edges, radius, np.array([0.0, 0.0, 25.0]), np.array([0.0, 0.0, -1.0]),
               R=R, step=0.01, lo=lo, hi=hi)
    assert 5.0 - R < t < 5.0


def test_near_ray_filter_drops_no_contributor(monkeypatch):
    """The filter keeps every strut that can reach the ray's line: 24 random
    rays through the cubic+BCC lattice give the same depths as a brute-force
    cast over all struts."""
    import synth
    cfg = synth.config(1)
    nodes, edges, radius, R = cfg["nodes"], cfg["edges"], cfg["radius"], cfg["R"]
    lo = np.asarray(nodes, np.float32).min(0).astype(np.float64) - R
    hi = np.asarray(nodes, np.float32).max(0).astype(np.float64) + R
    r = synth.rng(31)
    rays = []
    for _ in range(24):
        o = r.uniform(lo - 5.0, hi + 5.0)
        tgt = r.uniform(lo, hi)
        d = (tgt - o) / np.linalg.norm(tgt - o)
        rays.append((o, d))
    kw = dict(R=R, C=1.0, step=0.05, refine=12, lo=lo, hi=hi)
    filtered = [V.cast(nodes, edges, radius, o, d, **kw) for o, d in rays]
    monkeypatch.setattr(V, "near_ray", lambda nodes_, edges_, o_, d_, R_: np.arange(len(edges_)))
    brute = [V.cast(nodes, edges, radius, o, d, **kw) for o, d in rays]
    assert filtered == brute
    assert sum(not math.isinf(t) for t in brute) >= 8
