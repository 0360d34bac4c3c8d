"""Ray casting of the implicit solid {Sigma >= C} (the paper renders its
lattices by ray tracing the implicit function directly, without a mesh; Sec.
5.5's result figures and Sec. 3's convolution surface, Eq. 5-7).

TEST INFRASTRUCTURE ONLY: used by the tests, never by the product package.
Plain numpy in double precision, with the field of the C oracle.

Readings:
  V1 camera: pinhole at `eye` looking at `target`, `up` fixing the roll,
     vertical field of view `fov_y` (radians); pixel (i, j) (j = row from the
     top) has its ray through the image-plane point of its centre.
  V2 a ray is sampled at t_k = t_in + k * step, k = 0, 1, ..., from where it
     enters the lattice's box grown by R (t_in >= 0) to where it leaves; the
     hit is the first sample with Sigma >= C, refined by `refine` halvings of
     [t_{k-1}, t_k] (from t_in itself when k = 0); no sample inside: a miss
     (depth +inf). Features thinner than a step can be missed, as in any
     sampled ray march.
"""
from __future__ import annotations

import math

import numpy as np

from . import sigma_points


def camera_rays(eye, target, up, fov_y: float, width: int, height: int):
    """Ray origins (the eye) and unit directions [height, width, 3] (V1)."""
    eye = np.asarray(eye, dtype=np.float64)
    f = np.asarray(target, dtype=np.float64) - eye
    f /= np.linalg.norm(f)
    r = np.cross(f, np.asarray(up, dtype=np.float64))
    r /= np.linalg.norm(r)
    u = np.cross(r, f)
    half_h = math.tan(0.5 * fov_y)
    half_w = half_h * width / height
    jj, ii = np.meshgrid(np.arange(height), np.arange(width), indexing="ij")
    x = ((ii + 0.5) / width * 2.0 - 1.0) * half_w
    y = (1.0 - (jj + 0.5) / height * 2.0) * half_h
    d = f[None, None, :] + x[..., None] * r[None, None, :] + y[..., None] * u[None, None, :]
    d /= np.linalg.norm(d, axis=2, keepdims=True)
    return eye, d


def box_interval(o, d, lo, hi):
    """[t0, t1] of the ray o + t d inside the box (t0 clamped at 0), or None."""
    t0, t1 = 0.0, math.inf
    for k in range(3):
        if d[k] == 0.0:
            if o[k] < lo[k] or o[k] > hi[k]:
                return None
            continue
        a = (lo[k] - o[k]) / d[k]
        b = (hi[k] - o[k]) / d[k]
        if a > b:
            a, b = b, a
        t0 = max(t0, a)
        t1 = min(t1, b)
        if t0 > t1:
            return None
    return t0, t1


def near_ray(nodes, edges, o, d, R):
    """Indices of the struts that can reach the ray's line: a strut whose
    midpoint lies farther than R + half its length from the line contributes
    nothing anywhere on it."""
    nodes = np.asarray(nodes, dtype=np.float64)
    a = nodes[edges[:, 0]]
    b = nodes[edges[:, 1]]
    m = 0.5 * (a + b)
    half = 0.5 * np.linalg.norm(b - a, axis=1)
    q = m - o[None, :]
    t = q @ d
    dist = np.linalg.norm(q - t[:, None] * d[None, :], axis=1)
    return np.nonzero(dist <= R + half)[0]


def cast(nodes, edges, radius, o, d, *, R, C=1.0, step, refine=24, lo, hi):
    """Depth of the first hit of one ray (V2), +inf for a miss."""
    iv = box_interval(o, d, lo, hi)
    if iv is None:
        return math.inf
    keep = near_ray(nodes, np.asarray(edges), o, d, R)
    edges = np.asarray(edges)[keep]
    radius = np.asarray(radius)[keep]
    if edges.shape[0] == 0:
        return math.inf
    t_in, t_out = iv
    n = int(math.floor((t_out - t_in) / step)) + 1
    ts = t_in + step * np.arange(n)
    pts = o[None, :] + ts[:, None] * d[None, :]
    sig = sigma_points(nodes, edges, radius, pts, R=R, C=C)
    inside = np.nonzero(sig >= C)[0]
    if inside.size == 0:
        return math.inf
    k = int(inside[0])
    if k == 0:
        return float(ts[0])
    a, b = float(ts[k - 1]), float(ts[k])
    for _ in range(refine):
        m = 0.5 * (a + b)
        s = sigma_points(nodes, edges, radius, (o + m * d)[None, :], R=R, C=C)[0]
        if s >= C:
            b = m
        else:
            a = m
    return 0.5 * (a + b)


def render(nodes, edges, radius, *, R, C=1.0, eye, target, up, fov_y, width, height, step,
           refine=24, pixels=None):
    """Depth image [height, width] (or the listed (j, i) pixels)."""
    nodes = np.asarray(nodes, dtype=np.float32)
    lo = nodes.min(0).astype(np.float64) - R
    hi = nodes.max(0).astype(np.float64) + R
    o, dirs = camera_rays(eye, target, up, fov_y, width, height)
    if pixels is None:
        pixels = [(j, i) for j in range(height) for i in range(width)]
    out = {}
    for j, i in pixels:
        out[(j, i)] = cast(nodes, edges, radius, o, dirs[j, i], R=R, C=C, step=step,
                           refine=refine, lo=lo, hi=hi)
    return out
