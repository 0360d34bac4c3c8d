"""FP64 CPU oracle for the convolution-surface lattice slicer (arxiv 2101.05031).

TEST INFRASTRUCTURE ONLY. The tests, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` use this module;
the product package never imports it. The arithmetic lives in
``cslice_oracle.c`` (plain single-threaded C, double precision), compiled on
first use with gcc; this file only marshals numpy arrays.

Functions and the paper passages they follow:
  kernel            Eq. 5 (quartic compact kernel)
  weight            Sec. 3.2 (r_i controls the strut radius; PHYSICAL/RAW)
  segment_integral  Eq. 7 with the arc-length Jacobian of Eq. 6
  slice_sigma       Sec. 4, Steps 1-6 (sorted edges, active set, Step 4 field)
  sigma_points      the same sweep at arbitrary points
  active_set        Eq. 8
  marching_squares  Sec. 4, last paragraph (marching squares on the slice)
  volume_fraction   Eq. 9 (cell density), deterministic smoothed samples
  vf_backward       analytic gradient of sum_c g_c vf_c (radius tuning, Sec. 5.4)
  vf_fd             central finite differences of the same loss
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "cslice_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

PHYSICAL = 0
RAW = 1


def build(force: bool = False) -> str:
    """Compile the oracle into ``oracle/_build/liboracle.so`` (gcc, -O2)."""
    os.makedirs(_BUILD, exist_ok=True)
    stale = (not os.path.exists(_LIB_PATH)
             or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC))
    if force or stale:
        tmp = _LIB_PATH + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-std=c99", "-shared", "-fPIC",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class _Loops(ctypes.Structure):
    _fields_ = [("n_loops", ctypes.c_int64), ("n_verts", ctypes.c_int64),
                ("loop_off", ctypes.POINTER(ctypes.c_int64)),
                ("edge_id", ctypes.POINTER(ctypes.c_int64)),
                ("xy", ctypes.POINTER(ctypes.c_double))]


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            P = ctypes.c_void_p
            i64, i32, d = ctypes.c_int64, ctypes.c_int32, ctypes.c_double
            lat = [P, i64, P, P, i64, d, d, ctypes.c_int]
            cells = [d, d, d, d, i32, i32, i32, i32, d]
            lib.orc_kernel.argtypes = [d, d]
            lib.orc_kernel.restype = d
            lib.orc_weight.argtypes = [d, d, d, ctypes.c_int]
            lib.orc_weight.restype = d
            lib.orc_weight_drho.argtypes = [d, d, d, ctypes.c_int]
            lib.orc_weight_drho.restype = d
            lib.orc_segment_integral.argtypes = [P, P, P, d]
            lib.orc_segment_integral.restype = d
            lib.orc_segment_integral_grad.argtypes = [P, P, P, d, P, P]
            lib.orc_segment_integral_grad.restype = d
            lib.orc_slice_sigma.argtypes = lat + [d, d, i32, d, d, i32, i32, d, P]
            lib.orc_slice_sigma.restype = ctypes.c_int
            lib.orc_sigma_points.argtypes = lat + [P, i64, P]
            lib.orc_sigma_points.restype = ctypes.c_int
            lib.orc_active_set.argtypes = [P, i64, P, P, i64, d, d, P]
            lib.orc_active_set.restype = i64
            lib.orc_marching_squares.argtypes = [P, i32, i32, d, d, d, d]
            lib.orc_marching_squares.restype = ctypes.POINTER(_Loops)
            lib.orc_loops_free.argtypes = [ctypes.POINTER(_Loops)]
            lib.orc_loops_free.restype = None
            lib.orc_volume_fraction.argtypes = lat + cells + [P, i64, P]
            lib.orc_volume_fraction.restype = ctypes.c_int
            lib.orc_vf_backward.argtypes = lat + cells + [P, P, i64, P, P]
            lib.orc_vf_backward.restype = ctypes.c_int
            lib.orc_vf_fd.argtypes = lat + cells + [P, P, i64, P, P, i64, d, P]
            lib.orc_vf_fd.restype = ctypes.c_int
            _lib = lib
    return _lib


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def _lattice_args(nodes, edges, radius):
    nodes = np.ascontiguousarray(nodes, dtype=np.float32).reshape(-1, 3)
    edges = np.ascontiguousarray(edges, dtype=np.int32).reshape(-1, 2)
    radius = np.ascontiguousarray(radius, dtype=np.float32).reshape(-1)
    if radius.shape[0] != edges.shape[0]:
        raise ValueError("radius must have one value per edge")
    keep = (nodes, edges, radius)
    return keep, [_ptr(nodes), nodes.shape[0], _ptr(edges), _ptr(radius), edges.shape[0]]


def _check(rc, what):
    if rc == -1:
        raise ValueError(f"{what}: edge index out of range")
    if rc != 0:
        raise RuntimeError(f"{what}: oracle error {rc}")


def default_support(radius) -> float:
    """R = 1.5 x the largest strut radius (Sec. 3.2)."""
    return 1.5 * float(np.max(np.asarray(radius, dtype=np.float64)))


def kernel(dist2: float, R: float) -> float:
    return _load().orc_kernel(float(dist2), float(R))


def weight(rho: float, R: float, C: float = 1.0, mode: int = PHYSICAL) -> float:
    return _load().orc_weight(float(rho), float(R), float(C), int(mode))


def weight_drho(rho: float, R: float, C: float = 1.0, mode: int = PHYSICAL) -> float:
    return _load().orc_weight_drho(float(rho), float(R), float(C), int(mode))


def segment_integral(p, vs, ve, R: float) -> float:
    p, vs, ve = (np.ascontiguousarray(x, dtype=np.float64) for x in (p, vs, ve))
    return _load().orc_segment_integral(_ptr(p), _ptr(vs), _ptr(ve), float(R))


def segment_integral_grad(p, a, b, R: float):
    """Returns (I, dI/da, dI/db) for one edge a -> b at point p."""
    p, a, b = (np.ascontiguousarray(x, dtype=np.float64) for x in (p, a, b))
    ga = np.zeros(3)
    gb = np.zeros(3)
    I = _load().orc_segment_integral_grad(_ptr(p), _ptr(a), _ptr(b), float(R), _ptr(ga), _ptr(gb))
    return I, ga, gb


def slice_sigma(nodes, edges, radius, *, R, C=1.0, mode=PHYSICAL, z0, dz, n_layers,
                x0, y0, nx, ny, pixel):
    """Sigma (the weighted sum of Eq. 6, no -C) on [n_layers, ny, nx] pixel centres."""
    keep, lat = _lattice_args(nodes, edges, radius)
    out = np.empty((int(n_layers), int(ny), int(nx)), dtype=np.float64)
    rc = _load().orc_slice_sigma(*lat, float(R), float(C), int(mode), float(z0), float(dz),
                                 int(n_layers), float(x0), float(y0), int(nx), int(ny),
                                 float(pixel), _ptr(out))
    _check(rc, "slice_sigma")
    del keep
    return out


def sigma_points(nodes, edges, radius, pts, *, R, C=1.0, mode=PHYSICAL):
    keep, lat = _lattice_args(nodes, edges, radius)
    pts = np.ascontiguousarray(pts, dtype=np.float64).reshape(-1, 3)
    out = np.empty(pts.shape[0], dtype=np.float64)
    rc = _load().orc_sigma_points(*lat, float(R), float(C), int(mode), _ptr(pts),
                                  pts.shape[0], _ptr(out))
    _check(rc, "sigma_points")
    del keep
    return out


def active_set(nodes, edges, R, z):
    nodes = np.ascontiguousarray(nodes, dtype=np.float32).reshape(-1, 3)
    edges = np.ascontiguousarray(edges, dtype=np.int32).reshape(-1, 2)
    out = np.empty(max(1, edges.shape[0]), dtype=np.int64)
    n = _load().orc_active_set(_ptr(nodes), nodes.shape[0], _ptr(edges), None,
                               edges.shape[0], float(R), float(z), _ptr(out))
    if n < 0:
        raise ValueError("active_set: edge index out of range")
    return out[:n].copy()


def marching_squares(sigma2d, *, x0, y0, pixel, C=1.0):
    """Closed loops of one slice. Returns (loop_off[n_loops+1], edge_id[n], xy[n, 2])."""
    s = np.ascontiguousarray(sigma2d, dtype=np.float64)
    ny, nx = s.shape
    L = _load().orc_marching_squares(_ptr(s), int(nx), int(ny), float(x0), float(y0),
                                     float(pixel), float(C))
    if not L:
        raise RuntimeError("marching_squares failed")
    try:
        c = L.contents
        nl, nv = c.n_loops, c.n_verts
        off = np.ctypeslib.as_array(c.loop_off, shape=(nl + 1,)).copy()
        if nv:
            eid = np.ctypeslib.as_array(c.edge_id, shape=(nv,)).copy()
            xy = np.ctypeslib.as_array(c.xy, shape=(nv * 2,)).reshape(nv, 2).copy()
        else:
            eid = np.zeros(0, np.int64)
            xy = np.zeros((0, 2))
    finally:
        _load().orc_loops_free(L)
    return off, eid, xy


def _cell_args(cells):
    o = cells["origin"]
    d = cells["dims"]
    return [float(o[0]), float(o[1]), float(o[2]), float(cells["h"]), int(d[0]), int(d[1]),
            int(d[2]), int(cells["m"]), float(cells["T"])]


def _cell_ids(cells, ids):
    if ids is None:
        d = cells["dims"]
        ids = np.arange(int(d[0]) * int(d[1]) * int(d[2]), dtype=np.int64)
    return np.ascontiguousarray(ids, dtype=np.int64)


def volume_fraction(nodes, edges, radius, cells, *, R, C=1.0, mode=PHYSICAL, ids=None):
    """vf of the listed cells (flat id (iz*cy + iy)*cx + ix); all cells if ids is None."""
    keep, lat = _lattice_args(nodes, edges, radius)
    ids = _cell_ids(cells, ids)
    out = np.empty(ids.shape[0], dtype=np.float64)
    rc = _load().orc_volume_fraction(*lat, float(R), float(C), int(mode), *_cell_args(cells),
                                     _ptr(ids), ids.shape[0], _ptr(out))
    _check(rc, "volume_fraction")
    del keep
    return out


def vf_backward(nodes, edges, radius, cells, g, *, R, C=1.0, mode=PHYSICAL, ids=None):
    """Gradient of sum_c g_c vf_c. Returns (grad_radius[n_edges], grad_nodes[n_nodes, 3])."""
    keep, lat = _lattice_args(nodes, edges, radius)
    ids = _cell_ids(cells, ids)
    g = np.ascontiguousarray(g, dtype=np.float64).reshape(-1)
    if g.shape[0] != ids.shape[0]:
        raise ValueError("one g per listed cell")
    n_edges = lat[4]
    n_nodes = lat[1]
    gr = np.empty(n_edges, dtype=np.float64)
    gn = np.empty((n_nodes, 3), dtype=np.float64)
    rc = _load().orc_vf_backward(*lat, float(R), float(C), int(mode), *_cell_args(cells),
                                 _ptr(ids), _ptr(g), ids.shape[0], _ptr(gr), _ptr(gn))
    _check(rc, "vf_backward")
    del keep
    return gr, gn


def vf_fd(nodes, edges, radius, cells, g, kind, idx, *, R, C=1.0, mode=PHYSICAL, ids=None,
          h=1e-4):
    """Central differences of sum_c g_c vf_c. kind 0: radius of edge idx;
    kind 1..3: x/y/z of node idx."""
    keep, lat = _lattice_args(nodes, edges, radius)
    ids = _cell_ids(cells, ids)
    g = np.ascontiguousarray(g, dtype=np.float64).reshape(-1)
    kind = np.ascontiguousarray(kind, dtype=np.int32).reshape(-1)
    idx = np.ascontiguousarray(idx, dtype=np.int64).reshape(-1)
    out = np.empty(kind.shape[0], dtype=np.float64)
    rc = _load().orc_vf_fd(*lat, float(R), float(C), int(mode), *_cell_args(cells), _ptr(ids),
                           _ptr(g), ids.shape[0], _ptr(kind), _ptr(idx), kind.shape[0],
                           float(h), _ptr(out))
    _check(rc, "vf_fd")
    del keep
    return out
