"""Host-side checks of the C ABI (no GPU needed)."""
import ctypes
import os
import re
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(csl_[a-z0-9_]+)\s*\(", src))
    return names


def test_header_declares_entry_points():
    names = declared_functions()
    for n in ("csl_lattice_upload", "csl_slice_layers", "csl_last_error", "csl_contours_free"):
        assert n in names


def test_library_exports_every_declared_symbol():
    from paper_2101_05031_gb300 import _lib
    lib = _lib.load()
    missing = [n for n in sorted(declared_functions()) if not hasattr(lib, n)]
    assert not missing, f"not exported: {missing}"
    # the binding declares a signature for each one
    bound = {n for n, _, _ in _lib.SIGNATURES}
    assert declared_functions() <= bound


def test_structs_match_header_layout(tmp_path):
    """ctypes mirrors of the ABI structs have the header's size and offsets."""
    from paper_2101_05031_gb300 import _lib
    mirrors = {"csl_params": _lib.Params, "csl_lattice_info": _lib.LatticeInfo,
               "csl_slice_desc": _lib.SliceDesc, "csl_contours": _lib.Contours,
               "csl_stats": _lib.Stats, "csl_batch_opts": _lib.BatchOpts,
               "csl_batch_info": _lib.BatchInfo, "csl_hatches": _lib.Hatches,
               "csl_cells": _lib.CellsDesc, "csl_voxels": _lib.Voxels,
               "csl_dm_params": _lib.DmParams, "csl_dm_result": _lib.DmResult,
               "csl_po_params": _lib.PoParams, "csl_po_result": _lib.PoResult,
               "csl_camera": _lib.Camera}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "cslice.h"', 'int main(void){']
    for cname, py in mirrors.items():
        lines.append(f'printf("{cname} %zu\\n", sizeof({cname}));')
        for fname, _ in py._fields_:
            lines.append(f'printf("{cname}.{fname} %zu\\n", offsetof({cname}, {fname}));')
    lines.append("return 0;}")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)])
    got = dict(l.split() for l in subprocess.check_output([str(exe)]).decode().splitlines())
    for cname, py in mirrors.items():
        assert int(got[cname]) == ctypes.sizeof(py), cname
        for fname, _ in py._fields_:
            assert int(got[f"{cname}.{fname}"]) == getattr(py, fname).offset, (cname, fname)


def test_errors_cross_the_abi_as_codes():
    """Host-side validation runs before any device work."""
    from paper_2101_05031_gb300 import _lib
    lib = _lib.load()
    out = ctypes.c_void_p()
    st = lib.csl_lattice_upload(None, -1, None, None, 0, None, None, ctypes.byref(out))
    assert st == 1 and b"negative" in lib.csl_last_error()
    st = lib.csl_lattice_upload(None, 0, None, None, 0, None, None, None)
    assert st == 1
    d = _lib.SliceDesc()
    d.nx = d.ny = 10
    d.pixel = 0.1
    d.n_layers = 1
    st = lib.csl_slice_layers(None, ctypes.byref(d), None, None)
    assert st == 1 and b"NULL" in lib.csl_last_error()
    # batches: argument checks come before any device call
    descs = (_lib.SliceDesc * 1)()
    lats = (ctypes.c_void_p * 1)()
    st = lib.csl_batch_create(lats, descs, 0, None, None, ctypes.byref(out))
    assert st == 1 and b"n_jobs" in lib.csl_last_error()
    bad = _lib.BatchOpts(0, 3, 0, 0)
    st = lib.csl_batch_create(lats, descs, 1, ctypes.byref(bad), None, ctypes.byref(out))
    assert st == 1 and b"slab" in lib.csl_last_error()
    st = lib.csl_batch_run(None, None)
    assert st == 1
    info = _lib.BatchInfo()
    assert lib.csl_batch_get_info(None, ctypes.byref(info)) == 1
    # density matching: parameters and indices are checked before any device call
    vox = _lib.Voxels((ctypes.c_double * 3)(0, 0, 0), 1.0, (ctypes.c_int32 * 3)(1, 1, 1), None)
    prm = _lib.DmParams(0.1, 0.0, 1.0, 0.01, 4, 4, 2, 24)
    res = ctypes.POINTER(_lib.DmResult)()
    st = lib.csl_density_match(None, 0, None, 0, ctypes.byref(vox), ctypes.byref(prm), None,
                               ctypes.byref(res))
    assert st == 1 and b"target" in lib.csl_last_error()
    tgt = np.zeros(1, np.float32)
    vox.target = tgt.ctypes.data_as(ctypes.c_void_p)
    for field, bad, word in (("R", 0.3, b"R must"), ("tet_n", 17, b"tet_n"), ("max_depth", 9, b"max_depth"),
                             ("iters", 0, b"iters"), ("r_min", -1.0, b"r_min")):
        p2 = _lib.DmParams(0.1, 0.0, 1.0, 0.01, 4, 4, 2, 24)
        setattr(p2, field, bad)
        st = lib.csl_density_match(None, 0, None, 0, ctypes.byref(vox), ctypes.byref(p2), None,
                                   ctypes.byref(res))
        assert st == 1 and word in lib.csl_last_error(), field
    nodes = np.zeros((4, 3), np.float32)
    tets = np.array([[0, 1, 2, 4]], np.int32)
    st = lib.csl_density_match(nodes.ctypes.data_as(ctypes.c_void_p), 4,
                               tets.ctypes.data_as(ctypes.c_void_p), 1, ctypes.byref(vox),
                               ctypes.byref(prm), None, ctypes.byref(res))
    assert st == 1 and b"out of range" in lib.csl_last_error()
    # vertex re-positioning: parameters and indices before any device call
    po = _lib.PoParams((ctypes.c_double * 3)(0, 0, 1), 0.785, (ctypes.c_double * 6)(), 0.25, 0.5,
                       0.1, 8, 10)
    pr = _lib.PoResult()
    for field, bad, word in (("step", 0.0, b"step"), ("min_volume", 1.0, b"min_volume"),
                             ("backtracks", -1, b"backtracks"), ("alpha", 2.0, b"alpha")):
        p2 = _lib.PoParams.from_buffer_copy(po)
        setattr(p2, field, bad)
        st = lib.csl_support_optimize(None, 0, None, 0, None, ctypes.byref(p2), None,
                                      ctypes.byref(pr), None)
        assert st == 1 and word in lib.csl_last_error(), field
    st = lib.csl_support_optimize(nodes.ctypes.data_as(ctypes.c_void_p), 4,
                                  tets.ctypes.data_as(ctypes.c_void_p), 1, None, ctypes.byref(po),
                                  None, ctypes.byref(pr), None)
    assert st == 1 and b"out of range" in lib.csl_last_error()
    # depth images, simplification and streamed uploads check their arguments first
    cam = _lib.Camera((ctypes.c_double * 3)(0, 0, 10), (ctypes.c_double * 3)(0, 0, 0),
                      (ctypes.c_double * 3)(0, 1, 0), 0.5, 16, 16, 0.1, 10, 0)
    assert lib.csl_render_depth(None, ctypes.byref(cam), None, None) == 1
    host = _lib.Contours()
    res_c = ctypes.POINTER(_lib.Contours)()
    st = lib.csl_simplify_contours(ctypes.byref(host), 10, 10, 0.1, None, ctypes.byref(res_c))
    assert st == 1 and b"device" in lib.csl_last_error()
    host.on_device = 1
    st = lib.csl_simplify_contours(ctypes.byref(host), 10, 10, 0.1, None, ctypes.byref(res_c))
    assert st == 1 and b"edge ids" in lib.csl_last_error()
    prm_dev = _lib.Params(0.0, 1.0, 0, 1)
    lat_out = ctypes.c_void_p()
    st = lib.csl_lattice_upload_streamed(nodes.ctypes.data_as(ctypes.c_void_p), 4, None, None, 0,
                                         ctypes.byref(prm_dev), 0, None, ctypes.byref(lat_out))
    assert st == 1 and b"host arrays" in lib.csl_last_error()
    st = lib.csl_lattice_upload_streamed(nodes.ctypes.data_as(ctypes.c_void_p), 4, None, None, 0,
                                         None, -1, None, ctypes.byref(lat_out))
    assert st == 1 and b"batch_edges" in lib.csl_last_error()
    # smoothing and contours from host arrays check their arguments first
    st = lib.csl_smooth_contours(ctypes.byref(host), 0.0, 0.0, 0.1, 10, 10, 0.5, 0.05, 4, None)
    assert st == 1 and b"edge ids" in lib.csl_last_error()
    host.on_device = 0
    st = lib.csl_smooth_contours(ctypes.byref(host), 0.0, 0.0, 0.1, 10, 10, 0.5, 0.05, 4, None)
    assert st == 1 and b"device" in lib.csl_last_error()
    host.on_device = 1
    host.edge_id = 16   # never read: every call below fails its argument checks first
    for args, word in (((0.1, 10, 10, 1.5, 0.05, 4), b"lambda"), ((0.1, 10, 10, 0.5, 0.0, 4), b"margin"),
                       ((0.1, 10, 10, 0.5, 0.6, 4), b"margin"), ((0.0, 10, 10, 0.5, 0.05, 4), b"pixel"),
                       ((0.1, 0, 10, 0.5, 0.05, 4), b"nx"), ((0.1, 10, 10, 0.5, 0.05, -1), b"iterations")):
        st = lib.csl_smooth_contours(ctypes.byref(host), 0.0, 0.0, *args, None)
        assert st == 1 and word in lib.csl_last_error(), word
    lo = np.array([0, 1], np.int64)
    xy = np.zeros((4, 2), np.float32)
    p = lambda a: a.ctypes.data_as(ctypes.c_void_p)
    for vo, word in ((np.array([0, 5], np.int64), b"loop_vert_off"),
                     (np.array([1, 4], np.int64), b"loop_vert_off")):
        st = lib.csl_contours_create(1, 1, 4, p(lo), p(vo), p(xy), None, None, ctypes.byref(res_c))
        assert st == 1 and word in lib.csl_last_error()
    st = lib.csl_contours_create(1, 2, 4, p(lo), p(np.array([0, 3, 4], np.int64)), p(xy), None,
                                 None, ctypes.byref(res_c))
    assert st == 1 and b"layer_loop_off" in lib.csl_last_error()
    st = lib.csl_contours_create(1, 2, 4, p(np.array([0, 2], np.int64)),
                                 p(np.array([0, 5, 4], np.int64)), p(xy), None, None,
                                 ctypes.byref(res_c))
    assert st == 1 and b"decreases" in lib.csl_last_error()
    bad_xy = xy.copy()
    bad_xy[2, 1] = np.nan
    st = lib.csl_contours_create(1, 1, 4, p(lo), p(np.array([0, 4], np.int64)), p(bad_xy), None,
                                 None, ctypes.byref(res_c))
    assert st == 1 and b"non-finite" in lib.csl_last_error()
    st = lib.csl_contours_create(1, 1, 4, p(lo), p(np.array([0, 4], np.int64)), p(xy),
                                 p(np.array([0, 2, -4, 6], np.int32)), None, ctypes.byref(res_c))
    assert st == 1 and b"negative edge id" in lib.csl_last_error()
    # the wait test's poll count is checked before any device call
    assert lib.csl_debug_wait_timeout(0, None) == 1
    assert lib.csl_debug_wait_timeout(1 << 23, None) == 1


def test_no_gpu_reports_not_ready():
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    import paper_2101_05031_gb300 as cs
    with pytest.raises(cs.CslError) as e:
        cs.Lattice(np.zeros((2, 3), np.float32), np.array([[0, 1]], np.int32),
                   np.array([0.1], np.float32))
    assert e.value.code in (3, 6)


def test_product_path_does_not_use_the_oracle():
    pkg = os.path.join(ROOT, "paper_2101_05031_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                src = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in src and "from oracle" not in src, f
                assert "cslice_oracle" not in src and "liboracle" not in src, f
