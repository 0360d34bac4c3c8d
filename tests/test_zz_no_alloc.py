"""csl_field_layers_static, the entry point that allocates no memory.

Some callers cannot allocate device memory: an application that plans all of
its device memory up front, or one that must not take the device-wide
synchronisation that cudaMalloc and cudaFree imply. For them the library
offers csl_field_layers_static, whose only scratch is a fixed static device
array. These tests call it through the C ABI and compare its output with the
regular entry point's (csl_slice_layers with sigma_out) within the field
tolerance the other parity tests use, on two calls in a row that share the
static scratch.
"""
import ctypes

import numpy as np
import pytest

import oracle
import synth
from tests import helpers

torch = pytest.importorskip("torch")


def _lib():
    from paper_2101_05031_gb300 import _lib as L
    return L


def _desc(L, *, z0, dz, n_layers, x0, y0, nx, ny, pixel):
    d = L.SliceDesc()
    d.z0, d.dz, d.n_layers = float(z0), float(dz), int(n_layers)
    d.nx, d.ny, d.pixel = int(nx), int(ny), float(pixel)
    d.x0, d.y0 = float(x0), float(y0)
    return d


def _static_call(cfg, grid, sigma):
    """csl_field_layers_static on device copies of cfg's arrays."""
    L = _lib()
    st = _static_status(cfg, grid, sigma)
    L.check(st)
    torch.cuda.synchronize()
    return sigma.cpu().numpy()


def _static_status(cfg, grid, sigma):
    L = _lib()
    lib = L.load()
    nodes = torch.from_numpy(np.ascontiguousarray(cfg["nodes"], np.float32)).cuda()
    edges = torch.from_numpy(np.ascontiguousarray(cfg["edges"], np.int32)).cuda()
    radius = torch.from_numpy(np.ascontiguousarray(cfg["radius"], np.float32)).cuda()
    d = _desc(L, **grid)
    st = lib.csl_field_layers_static(
        ctypes.c_void_p(nodes.data_ptr()), nodes.shape[0], ctypes.c_void_p(edges.data_ptr()),
        ctypes.c_void_p(radius.data_ptr()), edges.shape[0], float(cfg["R"]), float(cfg["C"]),
        L.MODE_PHYSICAL, ctypes.byref(d), ctypes.c_void_p(sigma.data_ptr()),
        ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    torch.cuda.synchronize()
    return st


def _regular_call(cfg, grid):
    import paper_2101_05031_gb300 as cs
    lat = cs.Lattice(cfg["nodes"], cfg["edges"], cfg["radius"], R=cfg["R"], C=cfg["C"])
    sig = torch.empty((grid["n_layers"], grid["ny"], grid["nx"]), dtype=torch.float32,
                      device="cuda")
    lat.slice(**grid, sigma_out=sig, contours=False)
    torch.cuda.synchronize()
    return sig.cpu().numpy()


@pytest.mark.gpu
def test_static_entry_point_matches_regular_two_calls():
    c1 = synth.config(1)
    g1 = dict(z0=1.25, dz=0.7, n_layers=5, x0=0.0, y0=0.0, nx=200, ny=200, pixel=0.1)
    c2 = synth.config(2, small=True)
    g2 = dict(z0=c2["z0"], dz=c2["dz"], n_layers=3, x0=c2["x0"], y0=c2["y0"], nx=137, ny=91,
              pixel=c2["pixel"])
    out1 = torch.full((5, 200, 200), -1.0, device="cuda")
    out2 = torch.full((3, 91, 137), -1.0, device="cuda")
    a1 = _static_call(c1, g1, out1)          # first call
    a2 = _static_call(c2, g2, out2)          # second call reuses the same scratch
    r1 = _regular_call(c1, g1)
    r2 = _regular_call(c2, g2)
    assert helpers.field_error(a1, r1, c1["C"]) <= helpers.FIELD_RTOL
    assert helpers.field_error(a2, r2, c2["C"]) <= helpers.FIELD_RTOL
    assert np.max(r1) > c1["C"] and np.max(r2) > c2["C"]   # the layers cut struts


@pytest.mark.gpu
def test_static_entry_point_reports_bad_input():
    L = _lib()
    cfg = dict(synth.config(1))
    cfg["edges"] = cfg["edges"].copy()
    cfg["edges"][3, 1] = 10_000                       # out of range: found on the device
    out = torch.empty((1, 16, 16), device="cuda")
    with pytest.raises(L.CslError, match="INVALID_ARG"):
        _static_call(cfg, dict(z0=1.0, dz=0.1, n_layers=1, x0=0, y0=0, nx=16, ny=16, pixel=0.1),
                     out)


def test_static_entry_point_rejects_too_many_edges():
    """Sizes beyond the static scratch are refused before any GPU work."""
    L = _lib()
    lib = L.load()
    d = _desc(L, z0=0, dz=0.1, n_layers=1, x0=0, y0=0, nx=4, ny=4, pixel=0.1)
    st = lib.csl_field_layers_static(None, 2, None, None, L.STATIC_MAX_EDGES + 1, 1.0, 1.0,
                                     L.MODE_PHYSICAL, ctypes.byref(d), None, None)
    assert st == 5   # CSL_ERR_CAPACITY
    assert b"CSL_STATIC_MAX_EDGES" in lib.csl_last_error()


@pytest.mark.gpu
def test_static_entry_point_matches_the_oracle():
    """The allocation-free field against the FP64 oracle (Eq. 6-7 summed over
    every edge), on layers of the cubic+BCC lattice and of a jittered
    Freudenthal block, two calls in a row."""
    c1 = synth.config(1)
    g1 = dict(z0=2.3, dz=1.9, n_layers=3, x0=0.0, y0=0.0, nx=200, ny=200, pixel=0.1)
    c2 = synth.config(2, small=True)
    g2 = dict(z0=c2["z0"] + 0.7, dz=0.45, n_layers=2, x0=c2["x0"], y0=c2["y0"], nx=120,
              ny=96, pixel=c2["pixel"])
    for cfg, g in ((c1, g1), (c2, g2)):
        got = _static_call(cfg, g, torch.full((g["n_layers"], g["ny"], g["nx"]), -1.0,
                                              device="cuda"))
        ref = oracle.slice_sigma(cfg["nodes"], cfg["edges"], cfg["radius"], R=cfg["R"],
                                 C=cfg["C"], z0=g["z0"], dz=g["dz"], n_layers=g["n_layers"],
                                 x0=g["x0"], y0=g["y0"], nx=g["nx"], ny=g["ny"],
                                 pixel=g["pixel"])
        helpers.assert_field(got, ref, cfg["C"])
        assert np.max(ref) > cfg["C"]


@pytest.mark.gpu
def test_static_entry_point_at_capacity():
    """Exactly CSL_STATIC_MAX_EDGES edges, so the last record fills the end of
    the static array: the same field as csl_slice_layers."""
    L = _lib()
    n = L.STATIC_MAX_EDGES
    rng = np.random.default_rng(2101050310)
    a = rng.uniform(0.0, 2.0, (n, 3)).astype(np.float32)
    b = (a + rng.uniform(-0.15, 0.15, (n, 3))).astype(np.float32)
    nodes = np.empty((2 * n, 3), np.float32)
    nodes[0::2], nodes[1::2] = a, b
    edges = np.arange(2 * n, dtype=np.int32).reshape(n, 2)
    radius = rng.uniform(0.01, 0.025, n).astype(np.float32)
    cfg = dict(nodes=nodes, edges=edges, radius=radius, R=0.04, C=1.0)
    g = dict(z0=1.0, dz=0.1, n_layers=1, x0=0.0, y0=0.0, nx=40, ny=40, pixel=0.05)
    got = _static_call(cfg, g, torch.full((1, 40, 40), -1.0, device="cuda"))
    ref = _regular_call(cfg, g)
    assert helpers.field_error(got, ref, 1.0) <= helpers.FIELD_RTOL
    assert np.count_nonzero(ref) > 100


@pytest.mark.gpu
def test_static_entry_point_checks_every_node():
    """A non-finite coordinate of a node that no edge uses is reported too, as
    csl_lattice_upload reports it."""
    L = _lib()
    cfg = dict(synth.config(1))
    cfg["nodes"] = np.concatenate([cfg["nodes"], [[np.nan, 0.0, 0.0]]]).astype(np.float32)
    out = torch.empty((1, 16, 16), device="cuda")
    st = _static_status(cfg, dict(z0=1.0, dz=0.1, n_layers=1, x0=0, y0=0, nx=16, ny=16,
                                  pixel=0.1), out)
    assert st == 1 and b"non-finite" in L.load().csl_last_error()


def test_static_entry_point_rejects_a_non_finite_dz():
    """Layer k lies at z0 + k dz: a non-finite dz is refused even for a single
    layer (before any GPU work)."""
    L = _lib()
    lib = L.load()
    for dz in (float("inf"), float("nan")):
        d = _desc(L, z0=0, dz=dz, n_layers=1, x0=0, y0=0, nx=4, ny=4, pixel=0.1)
        st = lib.csl_field_layers_static(None, 0, None, None, 0, 1.0, 1.0, L.MODE_PHYSICAL,
                                         ctypes.byref(d), None, None)
        assert st == 1 and b"dz" in lib.csl_last_error()
