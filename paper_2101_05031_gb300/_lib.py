"""ctypes declarations for libcslice.so (see include/cslice.h).

The library is built in-tree by ``paper_2101_05031_gb300.build``; loading
fails loudly when it is missing. There is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

from . import build as _build

c_i32, c_i64, c_f32, c_f64, c_vp = (ctypes.c_int32, ctypes.c_int64, ctypes.c_float,
                                    ctypes.c_double, ctypes.c_void_p)

CSL_OK = 0
STATUS_NAMES = {0: "OK", 1: "INVALID_ARG", 2: "OOM", 3: "CUDA", 4: "TIMEOUT", 5: "CAPACITY",
                6: "NOT_READY"}
MODE_PHYSICAL = 0
MODE_RAW = 1
SLICE_CONTOURS_ON_DEVICE = 1
SLICE_EDGE_IDS = 2
SLICE_NO_CONTOURS = 4
SLICE_TIME_KERNELS = 8
SLICE_COUNT_PAIRS = 16
SLICE_FUSED = 32
STATIC_MAX_EDGES = 262144
FIELD_KERNELS = {"auto": 0, "block": 1, "footprint": 2}   # csl_slice_desc.field_kernel
BATCH_MAX_CANDIDATES = 16


class Params(ctypes.Structure):
    _fields_ = [("R", c_f64), ("C", c_f64), ("mode", c_i32), ("input_on_device", c_i32)]


class LatticeInfo(ctypes.Structure):
    _fields_ = [("n_nodes", c_i64), ("n_edges", c_i64), ("R", c_f64), ("C", c_f64),
                ("mode", c_i32), ("pad_", c_i32), ("bbox_lo", c_f32 * 3), ("bbox_hi", c_f32 * 3),
                ("max_dz", c_f32), ("max_radius", c_f32)]


class SliceDesc(ctypes.Structure):
    _fields_ = [("z0", c_f64), ("dz", c_f64), ("n_layers", c_i32), ("nx", c_i32), ("ny", c_i32),
                ("flags", c_i32), ("x0", c_f64), ("y0", c_f64), ("pixel", c_f64),
                ("sigma_out", c_vp), ("tile", c_i32), ("slab", c_i32), ("chunk_layers", c_i32),
                ("field_kernel", ctypes.c_int16), ("stage_records", ctypes.c_int16),
                ("mask_out", c_vp), ("workspace_budget", c_i64)]


class Contours(ctypes.Structure):
    _fields_ = [("n_layers", c_i32), ("on_device", c_i32), ("n_loops", c_i64), ("n_verts", c_i64),
                ("layer_loop_off", c_vp), ("loop_vert_off", c_vp), ("xy", c_vp),
                ("edge_id", c_vp)]


class Hatches(ctypes.Structure):
    _fields_ = [("n_layers", c_i32), ("on_device", c_i32), ("n_segments", c_i64),
                ("layer_seg_off", c_vp), ("seg", c_vp)]


class Stats(ctypes.Structure):
    _fields_ = [("candidate_pairs", c_i64), ("crossings", c_i64), ("loops", c_i64),
                ("chunks", c_i64), ("device_bytes_peak", c_i64), ("kernel_launches", c_i64),
                ("field_launches", c_i64), ("field_ms", c_f64), ("contributing_pairs", c_i64),
                ("bin_ms", c_f64), ("contour_ms", c_f64), ("output_ms", c_f64),
                ("evaluated_terms", c_i64), ("window_records", c_i64),
                ("field_kernel", c_i32), ("tile", c_i32), ("slab", c_i32),
                ("stage_records", c_i32), ("fused", c_i32), ("reserved_", c_i32)]


class Voxels(ctypes.Structure):
    _fields_ = [("origin", c_f64 * 3), ("h", c_f64), ("dims", c_i32 * 3), ("target", c_vp)]


class DmParams(ctypes.Structure):
    _fields_ = [("r_min", ctypes.c_float), ("R", ctypes.c_float), ("C", ctypes.c_float),
                ("temperature", ctypes.c_float), ("tet_n", c_i32), ("vox_m", c_i32),
                ("max_depth", c_i32), ("iters", c_i32)]


class Camera(ctypes.Structure):
    _fields_ = [("eye", c_f64 * 3), ("target", c_f64 * 3), ("up", c_f64 * 3), ("fov_y", c_f64),
                ("width", c_i32), ("height", c_i32), ("step", c_f64), ("refine", c_i32),
                ("reserved", c_i32)]


class PoParams(ctypes.Structure):
    _fields_ = [("t_p", c_f64 * 3), ("alpha", c_f64), ("a", c_f64 * 6), ("step", c_f64),
                ("ball", c_f64), ("min_volume", c_f64), ("backtracks", c_i32),
                ("max_rounds", c_i32)]


class PoResult(ctypes.Structure):
    _fields_ = [("rounds", c_i32), ("n_colours", c_i32), ("moves", c_i64),
                ("gamma_before", c_f64), ("psi_before", c_f64), ("gamma_after", c_f64),
                ("psi_after", c_f64), ("host_ms", c_f64), ("wall_ms", c_f64)]


class DmResult(ctypes.Structure):
    _fields_ = [("n_nodes", c_i64), ("nodes", c_vp), ("n_edges", c_i64), ("edges", c_vp),
                ("radius", c_vp), ("step3_ratio", c_vp), ("n_tets", c_i64), ("tets", c_vp),
                ("tet_depth", c_vp), ("tet_target", c_vp), ("tet_rho_star", c_vp),
                ("tet_ratio", c_vp), ("n_voxels", c_i64), ("voxel_ratio", c_vp),
                ("n_subdivided", c_i64), ("host_ms", c_f64), ("wall_ms", c_f64)]


class CellsDesc(ctypes.Structure):
    _fields_ = [("origin", c_f64 * 3), ("h", c_f64), ("dims", c_i32 * 3), ("m", c_i32),
                ("temperature", c_f64)]


class BatchOpts(ctypes.Structure):
    _fields_ = [("autotune", c_i32), ("slab", c_i32), ("ctas_per_sm", c_i32), ("branches", c_i32),
                ("field_kernel", c_i32), ("tile", c_i32), ("stage_records", c_i32),
                ("reserved_", c_i32)]


class BatchInfo(ctypes.Structure):
    _fields_ = [("n_jobs", c_i32), ("slab", c_i32), ("ctas_per_sm", c_i32), ("from_cache", c_i32),
                ("n_items", c_i64), ("n_pairs", c_i64), ("n_crossings", c_i64), ("n_loops", c_i64),
                ("graph_nodes", c_i64), ("pixel_evals", c_i64), ("plan_ms", c_f64),
                ("tune_ms", c_f64), ("n_candidates", c_i32),
                ("cand_slab", c_i32 * BATCH_MAX_CANDIDATES),
                ("cand_ctas", c_i32 * BATCH_MAX_CANDIDATES),
                ("cand_ms", c_f32 * BATCH_MAX_CANDIDATES),
                ("cand_kernel", c_i32 * BATCH_MAX_CANDIDATES),
                ("cand_tile", c_i32 * BATCH_MAX_CANDIDATES),
                ("cand_stage", c_i32 * BATCH_MAX_CANDIDATES),
                ("field_kernel", c_i32), ("tile", c_i32), ("stage_records", c_i32),
                ("reserved_", c_i32)]


class CslError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{STATUS_NAMES.get(code, code)}: {msg}")
        self.code = code


_lib = None

# (name, restype, argtypes); every entry point the header declares
SIGNATURES = [
    ("csl_last_error", ctypes.c_char_p, []),
    ("csl_version", ctypes.c_char_p, []),
    ("csl_last_stats", c_i32, [ctypes.POINTER(Stats)]),
    ("csl_lattice_upload", c_i32, [c_vp, c_i64, c_vp, c_vp, c_i64, ctypes.POINTER(Params), c_vp,
                                   ctypes.POINTER(c_vp)]),
    ("csl_lattice_upload_streamed", c_i32, [c_vp, c_i64, c_vp, c_vp, c_i64, ctypes.POINTER(Params),
                                            c_i64, c_vp, ctypes.POINTER(c_vp)]),
    ("csl_lattice_update", c_i32, [c_vp, c_vp, c_vp, c_vp]),
    ("csl_lattice_get_info", c_i32, [c_vp, ctypes.POINTER(LatticeInfo)]),
    ("csl_lattice_free", None, [c_vp]),
    ("csl_slice_layers", c_i32, [c_vp, ctypes.POINTER(SliceDesc), c_vp,
                                 ctypes.POINTER(ctypes.POINTER(Contours))]),
    ("csl_contours_free", None, [ctypes.POINTER(Contours)]),
    ("csl_contours_copy", c_i32, [ctypes.POINTER(Contours), c_vp, c_vp, c_vp, c_vp, c_i32, c_vp]),
    ("csl_debug_slab_bins", c_i32, [c_vp, ctypes.POINTER(SliceDesc), c_i32, c_i32, c_vp, c_vp,
                                    c_i64, ctypes.POINTER(c_i64), c_vp]),
    ("csl_volume_fraction", c_i32, [c_vp, ctypes.POINTER(CellsDesc), c_vp, c_vp]),
    ("csl_volume_fraction_backward", c_i32, [c_vp, ctypes.POINTER(CellsDesc), c_vp, c_vp, c_vp,
                                             c_vp]),
    ("csl_batch_create", c_i32, [ctypes.POINTER(c_vp), ctypes.POINTER(SliceDesc), c_i32,
                                 ctypes.POINTER(BatchOpts), c_vp, ctypes.POINTER(c_vp)]),
    ("csl_batch_run", c_i32, [c_vp, c_vp]),
    ("csl_batch_contours", c_i32, [c_vp, c_i32, c_i32, ctypes.POINTER(ctypes.POINTER(Contours))]),
    ("csl_batch_sigma", c_i32, [c_vp, c_i32, ctypes.POINTER(c_vp)]),
    ("csl_batch_get_info", c_i32, [c_vp, ctypes.POINTER(BatchInfo)]),
    ("csl_batch_free", None, [c_vp]),
    ("csl_hatch_layers", c_i32, [ctypes.POINTER(Contours), c_f64, c_f64, c_i32, c_i32, c_vp,
                                 ctypes.POINTER(ctypes.POINTER(Hatches))]),
    ("csl_hatches_free", None, [ctypes.POINTER(Hatches)]),
    ("csl_support_metrics", c_i32, [c_vp, ctypes.POINTER(c_f64), c_f64, ctypes.POINTER(c_f64),
                                    ctypes.POINTER(c_f64), ctypes.POINTER(c_f64), c_vp]),
    ("csl_debug_wait_timeout", c_i32, [ctypes.c_uint32, c_vp]),
    ("csl_density_match", c_i32, [c_vp, c_i64, c_vp, c_i64, ctypes.POINTER(Voxels),
                                  ctypes.POINTER(DmParams), c_vp,
                                  ctypes.POINTER(ctypes.POINTER(DmResult))]),
    ("csl_dm_result_free", None, [ctypes.POINTER(DmResult)]),
    ("csl_render_depth", c_i32, [c_vp, ctypes.POINTER(Camera), c_vp, c_vp]),
    ("csl_simplify_contours", c_i32, [ctypes.POINTER(Contours), c_i32, c_i32, c_f64, c_vp,
                                      ctypes.POINTER(ctypes.POINTER(Contours))]),
    ("csl_smooth_contours", c_i32, [ctypes.POINTER(Contours), c_f64, c_f64, c_f64, c_i32, c_i32,
                                    c_f64, c_f64, c_i32, c_vp]),
    ("csl_contours_create", c_i32, [c_i32, c_i64, c_i64, c_vp, c_vp, c_vp, c_vp, c_vp,
                                    ctypes.POINTER(ctypes.POINTER(Contours))]),
    ("csl_support_optimize", c_i32, [c_vp, c_i64, c_vp, c_i64, c_vp, ctypes.POINTER(PoParams),
                                     c_vp, ctypes.POINTER(PoResult), c_vp]),
    ("csl_measure_fp32_peak", c_i32, [ctypes.POINTER(c_f64), ctypes.POINTER(c_f64), c_vp]),
    ("csl_field_layers_static", c_i32, [c_vp, c_i64, c_vp, c_vp, c_i64, c_f64, c_f64, c_i32,
                                        ctypes.POINTER(SliceDesc), c_vp, c_vp]),
]


def lib_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Loads libcslice.so (building it first when it is missing or stale)."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.LIB
    if build_if_missing and _build.is_stale():
        _build.build()
    if not os.path.exists(path):
        raise RuntimeError(f"libcslice.so is not built ({path}); run "
                           "python -m paper_2101_05031_gb300.build")
    lib = ctypes.CDLL(path)
    for name, res, args in SIGNATURES:
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def check(status: int):
    if status != CSL_OK:
        msg = load().csl_last_error()
        raise CslError(status, msg.decode() if msg else "")
