"""Benchmark of the slicing hot path on GB300.

One step = one pass of the whole path over the workload: bin, evaluate the
field on every pixel of every layer, threshold, trace and stitch the contours
(contours stay in device memory). The default workload is the adaptive graded
lattice of about 100M struts (4000 x 4000 pixels of 0.05 mm, 1000 layers).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl cslice|reference]

Prints one JSON line (rank 0). Under torchrun, every rank slices its own
1000 layers (the job's layers shifted by r dz / N: the ranks together slice
the part at N times the layer resolution), so per-GPU work is fixed (weak
scaling) and no collective touches the data path.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import tempfile
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "pixel-evals/s and layers/s at 10M and 100M struts; backward/forward time ratio"
F_PAIR = 36            # FP32 flops of one (pixel, layer, edge) term in the field kernel
# Per field kernel, from an ncu capture of one launch on the 12.96M-strut
# graded lattice (profiles/): the FP32 instructions it executes per cycle as a
# fraction of the FP32 peak (every evaluated lane), and its DRAM bytes (read +
# write) per pixel-layer (scaled by pixel-layers to a launch of the timed
# workload). None where no capture of the current kernel exists.
NCU_FIELD = {
    "block": {"kernel": "k_field", "executed_frac": (2 * 2564.8 + 1382.6 + 2056.6) / (152 * 128 * 2),
              "dram_bytes_per_pixel_layer": (1.212995e9 + 4.259346e9) / (264 * 2000 * 2000),
              "profile": "profiles/k_field_graded-10M.txt"},
    "footprint": {"kernel": "k_field_fp",
                  "executed_frac": (2 * 3131.6 + 1369.7 + 1618.9) / (152 * 128 * 2),
                  "dram_bytes_per_pixel_layer": (0.729793e9 + 4.292423e9) / (264 * 2000 * 2000),
                  "profile": "profiles/k_field_fp_graded-10M.txt"},
}
# The volume fraction's FP32 work beyond the field term: per sample, the
# sigmoid and the mean (forward), the sigmoid and alpha (the adjoint's pass 1);
# per term of the adjoint's pass 2 (coordinates, the clipped chord, the 3-point
# moments M0..M2 and I, and the 7 partials), counting FMA as 2 and add, sub and
# mul as 1, as written in its kernel.
VF_FLOPS_PER_SAMPLE = 4
VF_GRAD_FLOPS_PER_SAMPLE = 8
VF_GRAD_FLOPS_PER_TERM = 124
# Executed FP32 fractions of the volume-fraction kernels from one ncu capture
# each on the 1M-strut Freudenthal lattice: FFMA (2 flops), FADD and FMUL
# thread instructions per cycle over the FP32 peak per cycle.
NCU_VF = {"forward": {"kernel": "k_field",
                      "executed_frac": (2 * 4094.3 + 1978.2 + 3107.9) / (152 * 128 * 2)},
          "backward": {"kernel": "k_vf_grad",
                       "executed_frac": (2 * 2256.0 + 1117.7 + 2062.3) / (152 * 128 * 2)},
          "profile": "profiles/k_vf_grad_freudenthal-1M.txt"}
HBM_GBS = 6772.9       # measured copy bandwidth of the GPU
# algorithmic bytes of the HBM-bound stages
BIN_BYTES_PER_WINDOW_RECORD = 24   # xy box (16) + z range (8) of a record read per slab window
BIN_BYTES_PER_ENTRY = 8            # (key, record) of a bin entry written
MS_BYTES_PER_PIXEL = 0.125         # inside-mask bit of a pixel read
MS_BYTES_PER_CROSSING = 16         # two Sigma values read, the vertex (x, y) written
MS_BYTES_PER_LOOP = 8              # the loop's vertex offset written
N_SM = 152
FP32_LANES = 128
MAX_SM_MHZ = 2070.0


# --------------------------------------------------------------------------- clocks

class ClockSampler:
    """nvidia-smi samples every 200 ms during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index=0):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        rows = []
        try:
            for line in open(self.path):
                f = [x.strip() for x in line.split(",")]
                if len(f) >= 9:
                    rows.append(f)
        except Exception:
            pass
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i] == "Active"})
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(rows)}


# --------------------------------------------------------------------------- workload

def workload(name):
    import synth
    if name == "graded-100M":
        return synth.config(3)
    if name == "graded-10M":
        nodes, edges, radius, r_ref = synth.adaptive_graded(box=100.0, level_min=4, level_max=7)
        return dict(name=f"adaptive graded lattice, {edges.shape[0]} struts, 2000^2 px x 500 "
                         "layers", nodes=nodes, edges=edges, radius=radius, R=1.5 * r_ref, C=1.0,
                    x0=0.0, y0=0.0, nx=2000, ny=2000, pixel=0.05, z0=0.1, dz=0.2, n_layers=500)
    if name == "freudenthal-430k":
        return synth.config(2)
    if name == "cubic-bcc-812":
        return synth.config(1)
    raise SystemExit(f"unknown workload {name}")


def max_over_ranks(ms, dist, device):
    """The slowest rank's time (every rank's layers count only once all are done)."""
    if dist is None:
        return ms
    import torch
    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank_step, steps, world, t_max_ms):
    """Units processed by all ranks per second of the slowest rank."""
    return units_per_rank_step * steps * world / (t_max_ms / 1e3)


def slice_kwargs(cfg, rank, world):
    z0 = cfg["z0"] + cfg["dz"] * rank / world
    return dict(z0=z0, dz=cfg["dz"], n_layers=cfg["n_layers"], x0=cfg["x0"], y0=cfg["y0"],
                nx=cfg["nx"], ny=cfg["ny"], pixel=cfg["pixel"])


# --------------------------------------------------------------------------- oracle sample

def oracle_sample(cfg, window=256, layer=None, min_seconds=12.0):
    """Times the FP64 oracle (single thread) on a window of one layer: the
    oracle gets the edges whose xy box grown by R meets the window and whose
    z range grown by R contains the layer (its own Eq. 8 sweep then runs)."""
    import oracle
    nl = cfg["n_layers"]
    layer = nl // 2 if layer is None else layer
    z = cfg["z0"] + layer * cfg["dz"]
    w = min(window, cfg["nx"], cfg["ny"])
    i0 = (cfg["nx"] - w) // 2
    j0 = (cfg["ny"] - w) // 2
    px = cfg["pixel"]
    wx0, wy0 = cfg["x0"] + i0 * px, cfg["y0"] + j0 * px
    R = cfg["R"]
    nodes, edges = cfg["nodes"], cfg["edges"]
    a = nodes[edges[:, 0]].astype(np.float64)
    b = nodes[edges[:, 1]].astype(np.float64)
    lo, hi = np.minimum(a, b), np.maximum(a, b)
    keep = ((lo[:, 2] - R <= z) & (hi[:, 2] + R >= z) & (hi[:, 0] + R >= wx0)
            & (lo[:, 0] - R <= wx0 + w * px) & (hi[:, 1] + R >= wy0) & (lo[:, 1] - R <= wy0 + w * px))
    sel = np.nonzero(keep)[0]
    used = np.unique(edges[sel])
    remap = np.full(nodes.shape[0], -1, np.int64)
    remap[used] = np.arange(used.size)
    sub_nodes = nodes[used]
    sub_edges = remap[edges[sel]].astype(np.int32)
    sub_r = cfg["radius"][sel]
    # the same window, repeated until the sample has run long enough
    t0 = time.perf_counter()
    reps = 0
    while True:
        oracle.slice_sigma(sub_nodes, sub_edges, sub_r, R=R, C=cfg["C"], z0=z, dz=cfg["dz"],
                           n_layers=1, x0=wx0, y0=wy0, nx=w, ny=w, pixel=px)
        reps += 1
        if time.perf_counter() - t0 >= min_seconds or reps >= 64:
            break
    t = time.perf_counter() - t0
    evals = reps * w * w
    return {"value": evals / t, "unit": "pixel-evals/s", "cores": 1, "kind": "oracle",
            "seconds": t,
            "sample": f"{reps} x a {w}x{w}-pixel window of layer {layer} (z={z:.2f} mm), "
                      f"{sel.size} edges meeting the window given to the oracle"}


# --------------------------------------------------------------------------- extra lines

def _event_ms(fn, steps, warmup, stream):
    import torch
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        fn()
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / steps


def radius_tuning(lat, cfg, iterations=20):
    """Radius adjustment toward a prescribed density (Sec. 5.4): gradient steps
    on 1/2 ||vf - rho||^2 through the autograd function (forward: update and
    volume fraction; backward: the adjoint), rho(x) the graded density at the
    cell centres, radii clamped to [0.1, 0.9 R]. Returns ms per iteration (CUDA
    events) and the loss of every iteration."""
    import torch

    import synth
    from paper_2101_05031_gb300 import VolumeFraction
    cells = cfg["cells"]
    d, o, h = cells["dims"], cells["origin"], cells["h"]
    xs = o[0] + h * (np.arange(d[0]) + 0.5)
    ys = o[1] + h * (np.arange(d[1]) + 0.5)
    target = synth.graded_density(xs[None, None, :], ys[None, :, None])
    target = torch.tensor(np.broadcast_to(target, (d[2], d[1], d[0])).copy(),
                          dtype=torch.float32, device="cuda")
    nodes = torch.tensor(cfg["nodes"], device="cuda")
    r0 = torch.tensor(cfg["radius"], device="cuda")
    R = cfg["R"]
    # one untimed iteration: the step size (0.01 mm at the 90th percentile of
    # |grad|), and the first use of the autograd path and of torch's kernels
    # (lazily loaded modules, seconds on first use)
    rw = r0.clone().requires_grad_(True)
    loss = 0.5 * ((VolumeFraction.apply(rw, nodes, lat, cells) - target) ** 2).sum()
    loss.backward()
    g90 = float(torch.quantile(rw.grad.detach().abs()[::16].float(), 0.9))
    lr = 0.01 / max(g90, 1e-12)
    with torch.no_grad():   # the update's kernels too (their first use loads a module)
        (r0 - lr * rw.grad).clamp(0.1, 0.9 * R)
    r = r0.clone()
    losses = []
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(iterations):
        r.requires_grad_(True)
        vf = VolumeFraction.apply(r, nodes, lat, cells)
        loss = 0.5 * ((vf - target) ** 2).sum()
        loss.backward()
        with torch.no_grad():
            r = (r - lr * r.grad).clamp(0.1, 0.9 * R)
        losses.append(loss.detach())
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / iterations
    lat.update(radius=torch.tensor(cfg["radius"], device="cuda"))   # back to the input radii
    curve = [float(x) for x in losses]
    return {"iterations": iterations, "ms_per_iteration": ms, "loss": curve,
            "loss_drop": curve[0] / max(curve[-1], 1e-30),
            "basis": "VolumeFraction.apply (lattice update + forward) and backward per "
                     "iteration, CUDA events over all iterations after one untimed iteration "
                     "that fixes the step (0.01 mm / 90th percentile of |grad|); radii "
                     "clamped to [0.1, 0.9 R]"}


def run_vf(steps, warmup):
    """Volume fraction and its adjoint on the 1M-strut Freudenthal lattice
    (64^3 cells x 8^3 samples): ms per forward, per backward, and the ratio."""
    import torch

    import paper_2101_05031_gb300 as cs
    import synth
    from paper_2101_05031_gb300 import volume_fraction, volume_fraction_backward
    cfg = synth.config(5)
    lat = cs.Lattice(cfg["nodes"], cfg["edges"], cfg["radius"], R=cfg["R"], C=cfg["C"])
    cells = cfg["cells"]
    d = cells["dims"]
    stream = torch.cuda.current_stream()
    vf = torch.empty((d[2], d[1], d[0]), device="cuda")
    g = torch.randn((d[2], d[1], d[0]), device="cuda",
                    generator=torch.Generator("cuda").manual_seed(0))
    fwd = _event_ms(lambda: volume_fraction(lat, cells, out=vf), steps, warmup, stream)
    bwd = _event_ms(lambda: volume_fraction_backward(lat, cells, g), steps, warmup, stream)
    samples = d[0] * d[1] * d[2] * cells["m"] ** 3
    # FP32 roofline. The m^3 samples of every cell are the pixels of a grid of
    # pitch h/m whose layers lie every h/m from half a pitch above the origin,
    # so the slicing kernel's exact counting pass on that grid counts the
    # nonzero (sample, strut) terms the forward evaluates (36 flops each, plus
    # the sigmoid and the mean per sample). The backward recomputes them (its
    # pass 1) and then evaluates the moments and the 7 partials only where the
    # sigmoid has not saturated, a thin shell around the iso-surface whose
    # term count the library does not report: its algorithmic figure here is
    # pass 1 alone (a lower bound), beside ncu's executed FP32 fraction.
    m = cells["m"]
    pitch = cells["h"] / m
    lat.slice(z0=cells["origin"][2] + 0.5 * pitch, dz=pitch, n_layers=d[2] * m,
              x0=cells["origin"][0], y0=cells["origin"][1], nx=d[0] * m, ny=d[1] * m,
              pixel=pitch, contours=False, count_pairs=True)
    pairs = int(cs.last_stats().contributing_pairs)
    peak = N_SM * FP32_LANES * 2 * MAX_SM_MHZ * 1e6 / 1e12
    f_fwd = pairs * F_PAIR + samples * VF_FLOPS_PER_SAMPLE
    f_bwd1 = pairs * F_PAIR + samples * VF_GRAD_FLOPS_PER_SAMPLE
    roof = {
        "forward": {"bound": "alu", "achieved": f_fwd / (fwd / 1e3) / 1e12, "peak": peak,
                    "unit": "TFLOP/s", "frac": f_fwd / (fwd / 1e3) / 1e12 / peak,
                    "nonzero_terms": pairs, "flops_per_term": F_PAIR,
                    "flops_per_sample": VF_FLOPS_PER_SAMPLE,
                    "duration_basis": "CUDA events around the whole forward call (binning, "
                                      "field kernel, per-cell mean)",
                    "executed_frac_ncu": NCU_VF["forward"]["executed_frac"],
                    "executed_kernel": NCU_VF["forward"]["kernel"]},
        "backward": {"bound": "alu", "achieved_lower_bound": f_bwd1 / (bwd / 1e3) / 1e12,
                     "peak": peak, "unit": "TFLOP/s",
                     "frac_lower_bound": f_bwd1 / (bwd / 1e3) / 1e12 / peak,
                     "flops_per_term_pass2": VF_GRAD_FLOPS_PER_TERM,
                     "lower_bound_basis": "pass 1 only (Sigma recomputed: 36 flops per nonzero "
                                          "term, sigmoid and alpha per sample); pass 2's "
                                          f"{VF_GRAD_FLOPS_PER_TERM} flops per term where the "
                                          "sigmoid has not saturated are not counted",
                     "executed_frac_ncu": NCU_VF["backward"]["executed_frac"],
                     "executed_kernel": NCU_VF["backward"]["kernel"]},
        "peak_basis": "152 SMs x 128 FP32 lanes x 2 x 2070 MHz (max SM clock)",
        "executed_basis": "ncu FFMA + FADD + FMUL thread instructions per cycle of one launch "
                          f"({NCU_VF['profile']})"}
    # the FP64 oracle on a sample of 2 cells in the middle of the grid (one host core)
    import oracle
    n_cells = d[0] * d[1] * d[2]
    mid = (d[2] // 2 * d[1] + d[1] // 2) * d[0] + d[0] // 2
    ids = np.arange(mid, mid + 2, dtype=np.int64)
    t0 = time.perf_counter()
    oracle.volume_fraction(cfg["nodes"], cfg["edges"], cfg["radius"], cells, R=cfg["R"], ids=ids)
    of = time.perf_counter() - t0
    t0 = time.perf_counter()
    oracle.vf_backward(cfg["nodes"], cfg["edges"], cfg["radius"], cells, np.ones(2), R=cfg["R"],
                       ids=ids)
    ob = time.perf_counter() - t0
    tuning = radius_tuning(lat, cfg, iterations=20)
    return {"workload": cfg["name"], "forward_ms": fwd, "backward_ms": bwd,
            "backward_forward_ratio": bwd / fwd, "samples_per_s_forward": samples / (fwd / 1e3),
            "samples_per_s_backward": samples / (bwd / 1e3), "roofline": roof,
            "radius_tuning": tuning,
            "cpu_baseline": {"kind": "oracle", "cores": 1, "sample": "2 cells of the 64^3 grid",
                             "forward_s_per_cell": of / 2, "backward_s_per_cell": ob / 2,
                             "forward_full_grid_s_extrapolated": of / 2 * n_cells,
                             "backward_full_grid_s_extrapolated": ob / 2 * n_cells}}


def run_10m(steps, warmup):
    """Slicing throughput on the 10M-strut graded lattice."""
    import torch

    import paper_2101_05031_gb300 as cs
    cfg = workload("graded-10M")
    lat = cs.Lattice(cfg["nodes"], cfg["edges"], cfg["radius"], R=cfg["R"], C=cfg["C"])
    kw = slice_kwargs(cfg, 0, 1)

    def step():
        lat.slice(**kw, on_device=True).free()

    ms = _event_ms(step, steps, warmup, torch.cuda.current_stream())
    st = cs.last_stats()
    return {"workload": cfg["name"], "struts": int(cfg["edges"].shape[0]),
            "pixel_evals_per_s": cfg["nx"] * cfg["ny"] * cfg["n_layers"] / (ms / 1e3),
            "layers_per_s": cfg["n_layers"] / (ms / 1e3), "ms_per_step": ms,
            "contours_per_step": {"loops": int(st.loops), "vertices": int(st.crossings)},
            "chunks": int(st.chunks)}


def run_batch(steps, warmup):
    """64 seeded Freudenthal lattices of uneven size (1k-500k struts, boxes of
    10-80 mm), 100 layers each at 0.05 mm pixels: the jobs as one autotuned,
    graph-captured batch against slicing them one after another with
    csl_slice_layers (contours left on the device in both)."""
    import torch

    import paper_2101_05031_gb300 as cs
    import synth
    cfg = synth.config(4)
    jobs = []
    for jb in cfg["jobs"]:
        lat = cs.Lattice(jb["nodes"], jb["edges"], jb["radius"], R=jb["R"], C=jb["C"])
        jobs.append((lat, dict(z0=jb["z0"], dz=jb["dz"], n_layers=jb["n_layers"], x0=jb["x0"],
                               y0=jb["y0"], nx=jb["nx"], ny=jb["ny"], pixel=jb["pixel"])))
    t0 = time.perf_counter()
    b = cs.Batch(jobs, autotune=True)
    create_s = time.perf_counter() - t0
    info = b.info()
    stream = torch.cuda.current_stream()
    batch_ms = _event_ms(b.run, steps, warmup, stream)

    def plain():
        for lat, d in jobs:
            lat.slice(**d, on_device=True).free()

    plain_ms = _event_ms(plain, steps, warmup, stream)
    px = int(info.pixel_evals)
    kname = {1: "block", 2: "footprint"}
    cands = [{"field_kernel": kname.get(int(info.cand_kernel[i]), "?"),
              "tile": int(info.cand_tile[i]), "slab": int(info.cand_slab[i]),
              "ctas_per_sm": int(info.cand_ctas[i]), "stage_records": int(info.cand_stage[i]),
              "ms": float(info.cand_ms[i])} for i in range(info.n_candidates)]
    out = {"workload": cfg["name"], "jobs": len(jobs),
           "struts": int(sum(jb["edges"].shape[0] for jb in cfg["jobs"])),
           "pixel_evals_per_step": px,
           "batched": {"ms_per_step": batch_ms, "pixel_evals_per_s": px / (batch_ms / 1e3),
                       "field_kernel": kname.get(int(info.field_kernel), "?"),
                       "tile": int(info.tile), "slab": int(info.slab),
                       "ctas_per_sm": int(info.ctas_per_sm),
                       "stage_records": int(info.stage_records),
                       "graph_nodes": int(info.graph_nodes), "queue_items": int(info.n_items),
                       "create_s": create_s, "plan_ms": info.plan_ms, "tune_ms": info.tune_ms,
                       "candidates": cands},
           "per_job": {"ms_per_step": plain_ms, "pixel_evals_per_s": px / (plain_ms / 1e3)},
           "batched_over_per_job": plain_ms / batch_ms}
    # the FP64 oracle on a 128^2 window of the middle layer of the largest lattice
    big = max(cfg["jobs"], key=lambda jb: jb["edges"].shape[0])
    ob = oracle_sample(big, window=128, min_seconds=3.0)
    out["cpu_baseline"] = dict(ob, full_batch_s_extrapolated=px / ob["value"])
    b.close()
    return out


def run_hatch(steps, warmup):
    """Zigzag infill of the 10M-strut graded lattice's contours (500 layers of
    2000^2 px; scan lines every 0.1 mm): contours left on the device, then
    csl_hatch_layers with the segments copied to the host."""
    import torch

    import paper_2101_05031_gb300 as cs
    cfg = workload("graded-10M")
    lat = cs.Lattice(cfg["nodes"], cfg["edges"], cfg["radius"], R=cfg["R"], C=cfg["C"])
    dev = lat.slice(**slice_kwargs(cfg, 0, 1), on_device=True, edge_ids=True)
    n_lines = int(round(cfg["ny"] * cfg["pixel"] / 0.1))
    y0 = cfg["y0"] + 0.05
    out = {}

    def step():
        off, seg = dev.hatch(y0, 0.1, n_lines)
        out["segments"] = int(seg.shape[0])

    ms = _event_ms(step, steps, warmup, torch.cuda.current_stream())
    # topology-preserving simplification of the same contours (tolerance 0.25 px)
    simp = {}

    def simplify_step():
        simp["c"] = dev.simplify(cfg["nx"], cfg["ny"], 0.25 * cfg["pixel"])
        simp["n"] = simp["c"].n_verts
        simp["c"].free()

    sms = _event_ms(simplify_step, steps, warmup, torch.cuda.current_stream())
    out_simplify = {"ms_per_step": sms, "vertices_in": int(dev.n_verts),
                    "vertices_out": int(simp["n"]), "vertices_per_s": dev.n_verts / (sms / 1e3),
                    "tolerance_px": 0.25}
    # smoothing of the same contours in place (4 Jacobi steps, lambda 1/2,
    # margin 0.05 of an edge); the last use of them here
    it = 4

    def smooth_step():
        dev.smooth(cfg["x0"], cfg["y0"], cfg["pixel"], cfg["nx"], cfg["ny"], lam=0.5,
                   margin=0.05, iterations=it)

    mms = _event_ms(smooth_step, steps, warmup, torch.cuda.current_stream())
    out_smooth = {"ms_per_step": mms, "iterations": it, "vertices": int(dev.n_verts),
                  "vertex_steps_per_s": dev.n_verts * it / (mms / 1e3)}
    return {"simplify": out_simplify, "smooth": out_smooth,
            "workload": cfg["name"] + ", scan lines every 0.1 mm", "layers": cfg["n_layers"],
            "contour_vertices": int(dev.n_verts), "segments": out["segments"],
            "ms_per_step": ms, "segments_per_s": out["segments"] / (ms / 1e3),
            "vertices_per_s": dev.n_verts / (ms / 1e3),
            "d2h_bytes_per_step": out["segments"] * 12 + (cfg["n_layers"] + 1) * 8}


def run_density(steps, warmup):
    """Density matching (Sec. 5.5) of a 93,750-tetrahedron Kuhn mesh of a
    100 mm box against graded targets on 50^3 voxels of 2 mm: wall time of
    csl_density_match (host mesh in, host lattice out), the lattice it builds,
    and how well the result's volume fraction (Eq. 9, the same 8^3 smoothed
    samples per voxel) matches the targets. The oracle's time on the 48-
    tetrahedron case stands beside the GPU's on the same case."""
    import torch

    import paper_2101_05031_gb300 as cs
    import synth
    from paper_2101_05031_gb300 import volume_fraction

    def call(cfg):
        return cs.density_match(cfg["nodes"], cfg["tets"], cfg["grid"], r_min=cfg["r_min"],
                                tet_n=cfg["tet_n"], vox_m=cfg["vox_m"],
                                max_depth=cfg["max_depth"], iters=cfg["iters"])

    def wall(cfg, n_steps, n_warm):
        for _ in range(n_warm):
            call(cfg)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(n_steps):
            res = call(cfg)
        torch.cuda.synchronize()
        return (time.perf_counter() - t0) / n_steps * 1e3, res

    cfg = synth.density_config()
    ms, res = wall(cfg, steps, warmup)
    grid = cfg["grid"]
    r_min = cfg["r_min"]
    d = grid["dims"]
    cells = dict(origin=grid["origin"], h=grid["h"], dims=d, m=8, T=0.01)
    tgt = grid["target"]

    def error(radius):
        lat = cs.Lattice(res["nodes"], res["edges"], radius, R=6.0 * r_min, C=1.0)
        vf = torch.empty((d[2], d[1], d[0]), device="cuda")
        volume_fraction(lat, cells, out=vf)
        err = vf.cpu().numpy() - tgt
        return {"mean_signed": float(np.mean(err)), "mean_abs": float(np.mean(np.abs(err))),
                "median_rel": float(np.median(np.abs(err) / tgt)),
                "within_10pct": float(np.mean(np.abs(err) <= 0.1 * tgt))}

    small = synth.density_config(small=True)
    gpu_small_ms, _ = wall(small, 3, 1)
    from oracle import density as D
    t0 = time.perf_counter()
    D.density_match(small["nodes"], small["tets"], small["grid"], r_min=small["r_min"],
                    tet_n=small["tet_n"], vox_m=small["vox_m"], max_depth=small["max_depth"],
                    iters=small["iters"])
    oracle_small_s = time.perf_counter() - t0
    n_in = int(cfg["tets"].shape[0])
    return {"workload": cfg["name"], "ms_per_step": ms,
            "input_tets_per_s": n_in / (ms / 1e3),
            "leaf_tets": int(res["tets"].shape[0]), "struts": int(res["edges"].shape[0]),
            "subdivided": int(res["n_subdivided"]),
            "depth_counts": np.bincount(res["depth"]).tolist(),
            "density_error": {"final": error(res["radius"]),
                              "after_step3": error(2 * r_min * res["step3_ratio"]),
                              "basis": "volume fraction of the lattice on the voxels (Eq. 9, "
                                       "8^3 samples, T = 0.01 C) minus the target"},
            "host_topology_ms": float(res["host_ms"]), "call_ms": float(res["wall_ms"]),
            "small_case": {"workload": small["name"], "gpu_ms": gpu_small_ms,
                           "cpu_baseline": {"seconds": oracle_small_s, "cores": 1,
                                            "kind": "oracle", "sample": "the whole small case"}}}


def run_support_opt(steps, warmup):
    """Vertex re-positioning for self-support (Eq. 16-17) on a 50^3-cube Kuhn
    mesh of 2 mm cubes (750,000 tetrahedra, 132,651 nodes), printing along z,
    up to 100 rounds: wall time of csl_support_optimize (host mesh in, host
    nodes out) and Gamma / Psi before and after; the oracle's time on the
    6^3-cube mesh beside the GPU's."""
    import torch

    import paper_2101_05031_gb300 as cs
    import synth
    nodes, tets = synth.kuhn_tet_mesh((50, 50, 50), 2.0, 0.15, seed=synth.SEED_BASE + 7)

    def wall(nd, tt, n_steps, n_warm):
        for _ in range(n_warm):
            cs.support_optimize(nd, tt)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(n_steps):
            res = cs.support_optimize(nd, tt)
        torch.cuda.synchronize()
        return (time.perf_counter() - t0) / n_steps * 1e3, res

    ms, res = wall(nodes, tets, steps, warmup)
    small_n, small_t = synth.kuhn_tet_mesh((6, 6, 6), 4.0, 0.15, seed=synth.SEED_BASE + 7)
    small_ms, _ = wall(small_n, small_t, 3, 1)
    from oracle import support_opt as P
    t0 = time.perf_counter()
    P.optimize(small_n, small_t)
    oracle_s = time.perf_counter() - t0
    return {"workload": "Kuhn tetrahedral mesh 50^3 cubes of 2 mm (750,000 tetrahedra), t_P = z",
            "ms_per_step": ms, "rounds": res["rounds"], "moves": res["moves"],
            "colours": res["n_colours"],
            "host_setup_ms": res["host_ms"], "call_ms": res["wall_ms"],
            "gamma": [res["gamma_before"], res["gamma_after"]],
            "psi_percent": [res["psi_before"], res["psi_after"]],
            "small_case": {"workload": "Kuhn mesh 6^3 cubes of 4 mm (1,296 tetrahedra)",
                           "gpu_ms": small_ms,
                           "cpu_baseline": {"seconds": oracle_s, "cores": 1, "kind": "oracle",
                                            "sample": "the whole small case"}}}


def run_render(steps, warmup):
    """Depth image of the implicit solid (csl_render_depth) of the 430k-strut
    Freudenthal lattice at 1920 x 1080, samples every R/8 along the rays; the
    oracle's time for a 32 x 24 image of the cubic+BCC lattice beside the
    GPU's for the same image."""
    import torch

    import paper_2101_05031_gb300 as cs
    import synth
    cfg = synth.config(2)
    lat = cs.Lattice(cfg["nodes"], cfg["edges"], cfg["radius"], R=cfg["R"], C=cfg["C"])
    lo, hi = synth.lattice_bbox(cfg["nodes"])
    c = 0.5 * (lo + hi)
    ext = float(np.max(hi - lo))
    cam = dict(eye=(float(c[0] + 1.1 * ext), float(c[1] - 0.8 * ext), float(c[2] + 0.7 * ext)),
               target=(float(c[0]), float(c[1]), float(c[2])), up=(0.0, 0.0, 1.0), fov_y=0.6,
               width=1920, height=1080)
    step = cfg["R"] / 8
    out = torch.empty((1080, 1920), dtype=torch.float32, device="cuda")
    ms = _event_ms(lambda: lat.render_depth(**cam, step=step, refine=20, out=out), steps, warmup,
                   torch.cuda.current_stream())
    hits = int(torch.isfinite(out).sum())
    small = synth.config(1)
    lat1 = cs.Lattice(small["nodes"], small["edges"], small["radius"], R=small["R"])
    cam1 = dict(eye=(31.0, -17.0, 24.0), target=(10.0, 10.0, 9.0), up=(0.0, 0.0, 1.0), fov_y=0.9,
                width=32, height=24)
    small_ms = _event_ms(lambda: lat1.render_depth(**cam1, step=0.05, refine=20), 3, 1,
                         torch.cuda.current_stream())
    from oracle import render as V
    t0 = time.perf_counter()
    V.render(small["nodes"], small["edges"], small["radius"], R=small["R"], C=1.0, step=0.05,
             refine=20, **cam1)
    oracle_s = time.perf_counter() - t0
    return {"workload": cfg["name"].split(",")[0] + ", 1920 x 1080 depth image, step R/8",
            "ms_per_step": ms, "rays_per_s": 1920 * 1080 / (ms / 1e3), "hits": hits,
            "small_case": {"workload": "cubic+BCC 812 struts, 32 x 24 image, step 0.05 mm",
                           "gpu_ms": small_ms,
                           "cpu_baseline": {"seconds": oracle_s, "cores": 1, "kind": "oracle",
                                            "sample": "the whole small image"}}}


# --------------------------------------------------------------------------- main

def run_reference(args, cfg, rank, world):
    if rank != 0:
        return
    steps = []
    for _ in range(args.warmup):
        oracle_sample(cfg, window=64, min_seconds=0.5)
    for _ in range(args.steps):
        steps.append(oracle_sample(cfg, window=128, min_seconds=3.0))
    v = float(np.mean([s["value"] for s in steps]))
    t_step = float(np.mean([s["seconds"] for s in steps]))
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "pixel-evals/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": t_step * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": cfg["name"], "parallelism": "single host thread"},
            "cpu_baseline": {"value": v, "unit": "pixel-evals/s", "cores": 1, "kind": "oracle",
                             "sample": steps[0]["sample"]},
            "e2e": {"value": v, "unit": "pixel-evals/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="cslice", choices=["cslice", "reference"])
    ap.add_argument("--workload", default="graded-100M")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--e2e-steps", type=int, default=3)
    ap.add_argument("--slab", type=int, default=0, help="layers per slab (0: library default)")
    ap.add_argument("--field-kernel", default="auto", choices=["auto", "block", "footprint"],
                    help="field kernel (auto: the library's choice)")
    ap.add_argument("--tile", type=int, default=0, help="tile side in pixels (0: auto, 16, 32)")
    ap.add_argument("--stage", type=int, default=0,
                    help="records per staged copy of the footprint kernel (0: 256)")
    ap.add_argument("--no-extra", action="store_true",
                    help="skip the 10M-strut and volume-fraction lines")
    ap.add_argument("--host-contours", action="store_true",
                    help="timed steps return the contours in host memory instead of leaving "
                         "them on the device")
    ap.add_argument("--no-count", action="store_true",
                    help="skip the untimed pass that counts nonzero terms (profiling runs)")
    ap.add_argument("--only", choices=["10M", "vf", "batched", "hatch", "density", "support",
                                       "render"],
                    help="run only one of the extra lines and print it (profiling runs)")
    args = ap.parse_args()
    if args.only:
        import torch
        torch.cuda.set_device(0)
        fn = {"10M": run_10m, "vf": run_vf, "batched": run_batch, "hatch": run_hatch,
              "density": run_density, "support": run_support_opt,
              "render": run_render}[args.only]
        print(json.dumps(fn(args.steps, args.warmup)), flush=True)
        return

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))

    if args.impl == "reference":
        cfg = workload(args.workload) if rank == 0 else None
        run_reference(args, cfg, rank, world)
        return

    import torch
    torch.cuda.set_device(local_rank)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))

    import paper_2101_05031_gb300 as cs
    cs.load()
    t_gen = time.perf_counter()
    cfg = workload(args.workload)
    t_gen = time.perf_counter() - t_gen
    kw = slice_kwargs(cfg, rank, world)
    kw["slab"] = args.slab
    kw["field_kernel"] = args.field_kernel
    kw["tile"] = args.tile
    kw["stage_records"] = args.stage
    stream = torch.cuda.current_stream()

    t_up = time.perf_counter()
    lat = cs.Lattice(cfg["nodes"], cfg["edges"], cfg["radius"], R=cfg["R"], C=cfg["C"])
    t_up = time.perf_counter() - t_up

    def step(flags_time=False):
        if args.host_contours:   # the contours copied to host memory (pinned blocks)
            c = lat.slice(**kw, time_kernels=flags_time)
            st = cs.last_stats()
            return st, (len(c.loop_vert_off) - 1, c.xy.shape[0])
        c = lat.slice(**kw, on_device=True, time_kernels=flags_time)
        st = cs.last_stats()
        n = (c.n_loops, c.n_verts)
        c.free()
        return st, n

    for _ in range(args.warmup):
        step()

    # exact count of nonzero and of evaluated terms, once, outside the timed region
    pairs = evaluated = cand = 0
    if not args.no_count:
        lat.slice(**kw, contours=False, count_pairs=True)
        pairs = cs.last_stats().contributing_pairs
        evaluated = cs.last_stats().evaluated_terms
        cand = cs.last_stats().candidate_pairs

    def barrier():
        if dist is not None:
            dist.barrier()

    launches = 0
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local_rank) as clk:
        barrier()
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(args.steps):
            st, (n_loops, n_verts) = step()
            launches += st.kernel_launches
        e1.record(stream)
        torch.cuda.synchronize()
        barrier()
    # one more step, untimed, with every stage timed by events: the chunks then
    # run one after another (no two-chunk overlap), so each kernel runs alone
    st, _ = step(flags_time=True)
    plan = {"field_kernel": {1: "block", 2: "footprint"}.get(st.field_kernel, "?"),
            "tile": st.tile, "slab": st.slab, "stage_records": st.stage_records,
            "fused": bool(st.fused)}
    peak_main = st.device_bytes_peak
    field_ms, bin_ms, contour_ms, output_ms = st.field_ms, st.bin_ms, st.contour_ms, st.output_ms
    field_launches = st.field_launches
    staged_ms = field_ms + bin_ms + contour_ms + output_ms
    ms = e0.elapsed_time(e1)
    t_max = max_over_ranks(ms, dist, "cuda")
    px_per_step = cfg["nx"] * cfg["ny"] * cfg["n_layers"]
    value = whole_job_rate(px_per_step, args.steps, world, t_max)
    layers_per_s = whole_job_rate(cfg["n_layers"], args.steps, world, t_max)
    clocks = clk.summary()

    # roofline of the field kernel: FP32 ALU
    ncu = NCU_FIELD[plan["field_kernel"]]
    t_field = field_ms / max(field_launches, 1) / 1e3            # s per launch
    flops_per_launch = pairs * F_PAIR / max(field_launches, 1)
    achieved = flops_per_launch / t_field / 1e12 if t_field > 0 else 0.0
    peak = N_SM * FP32_LANES * 2 * MAX_SM_MHZ * 1e6 / 1e12
    px_layers_per_launch = cfg["nx"] * cfg["ny"] * cfg["n_layers"] / max(field_launches, 1)
    roof = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
            "frac": achieved / peak,
            "traffic": (ncu["dram_bytes_per_pixel_layer"] * px_layers_per_launch
                        if ncu["dram_bytes_per_pixel_layer"] else None),
            "traffic_basis": "ncu dram bytes of one field launch on the 12.96M-strut graded "
                             "lattice, scaled by pixel-layers per launch",
            "kernel": ncu["kernel"], "flops_per_term": F_PAIR,
            "nonzero_terms_per_step": pairs, "evaluated_terms_per_step": evaluated,
            "candidate_entries_per_step": cand,
            "field_share_of_step": field_ms / staged_ms if staged_ms > 0 else None,
            "duration_basis": "CUDA events around each field launch in one extra step whose "
                              "stages run one after another",
            "peak_basis": "152 SMs x 128 FP32 lanes x 2 x 2070 MHz (max SM clock)"}
    if clocks.get("sm_mhz"):
        roof["frac_at_observed_clock"] = achieved / (peak * clocks["sm_mhz"] / MAX_SM_MHZ)
    # check of the derived peak: an FFMA microbenchmark of the library on this GPU
    ffma_tflops, _ = cs.measure_fp32_peak()
    roof["peak_check_ffma_microbenchmark_tflops"] = ffma_tflops
    roof["executed_frac_ncu"] = ncu["executed_frac"]
    roof["executed_basis"] = ("ncu FFMA + FADD + FMUL thread instructions per cycle of one "
                              "field launch on the 12.96M-strut graded lattice, every evaluated "
                              f"lane included ({ncu['profile']})")
    # the HBM-bound stages, against the measured copy bandwidth: algorithmic
    # bytes (the minimum each stage must move) over its event-timed duration
    px_layers = cfg["nx"] * cfg["ny"] * cfg["n_layers"]
    bin_bytes = st.window_records * BIN_BYTES_PER_WINDOW_RECORD + \
        st.candidate_pairs * BIN_BYTES_PER_ENTRY
    ms_bytes = px_layers * MS_BYTES_PER_PIXEL + st.crossings * MS_BYTES_PER_CROSSING + \
        st.loops * MS_BYTES_PER_LOOP
    secondary = {}
    for name, nbytes, t_ms in (("binner", bin_bytes, bin_ms), ("contours", ms_bytes, contour_ms)):
        gbs = nbytes / (t_ms / 1e3) / 1e9 if t_ms > 0 else 0.0
        secondary[name] = {"bound": "hbm", "achieved": gbs, "peak": HBM_GBS, "unit": "GB/s",
                           "frac": gbs / HBM_GBS, "algorithmic_bytes_per_step": nbytes,
                           "ms_per_step": t_ms}
    secondary["binner"]["basis"] = (f"{BIN_BYTES_PER_WINDOW_RECORD} B per record of a slab's "
                                    f"z window + {BIN_BYTES_PER_ENTRY} B per (slab, tile, "
                                    "edge) entry written")
    secondary["contours"]["basis"] = (f"{MS_BYTES_PER_PIXEL} B per pixel-layer (inside "
                                      f"mask) + {MS_BYTES_PER_CROSSING} B per vertex (two "
                                      f"Sigma values read, x y written) + {MS_BYTES_PER_LOOP} B "
                                      "per loop offset")

    line = {"metric": METRIC, "value": value, "unit": "pixel-evals/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_max / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic", "layers_per_s": layers_per_s,
            "config": {"workload": cfg["name"], "struts": int(cfg["edges"].shape[0]),
                       "pixel_mm": cfg["pixel"], "layers": cfg["n_layers"],
                       "l2": "inputs larger than L2 (32-byte records x struts)",
                       "contours": "host memory" if args.host_contours else "device memory",
                       "parallelism": f"{world} GPU(s), layers offset per rank"},
            "gpu_launches": launches, "clocks": clocks, "roofline": roof,
            "roofline_hbm_stages": secondary,
            "contours_per_step": {"loops": n_loops, "vertices": n_verts},
            "phase_ms_per_step": {"bin": bin_ms, "field": field_ms, "contours": contour_ms,
                                  "gather": output_ms, "sum": staged_ms,
                                  "basis": "one extra step with the stages run one after "
                                           "another"},
            "setup_s": {"generate": t_gen, "upload_and_sort": t_up}}

    line["slice_workspace_peak_bytes"] = int(peak_main)
    line["plan"] = plan
    if not args.no_e2e:
        # end to end through the public API: pinned host inputs, upload + prepare,
        # slice, contours copied back to host memory
        pn = torch.from_numpy(cfg["nodes"]).pin_memory()
        pe = torch.from_numpy(cfg["edges"]).pin_memory()
        pr = torch.from_numpy(cfg["radius"]).pin_memory()
        h2d = pn.numel() * 4 + pe.numel() * 4 + pr.numel() * 4

        e2e_peak = [0]

        phase_wall = []

        def e2e_step():
            t0 = time.perf_counter()
            L2 = cs.Lattice(pn, pe, pr, R=cfg["R"], C=cfg["C"])
            torch.cuda.synchronize()   # (the upload returns synchronised; phase attribution)
            t1 = time.perf_counter()
            cont = L2.slice(**kw)
            t2 = time.perf_counter()
            e2e_peak[0] = cs.last_stats().device_bytes_peak
            nbytes = cont.layer_loop_off.nbytes + cont.loop_vert_off.nbytes + cont.xy.nbytes
            L2.close()
            del cont
            phase_wall.append(((t1 - t0) * 1e3, (t2 - t1) * 1e3, (time.perf_counter() - t2) * 1e3))
            return nbytes

        e2e_step()   # untimed: the library's page-locked result blocks are allocated here
        barrier()
        torch.cuda.synchronize()
        a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a0.record(stream)
        d2h = 0
        wall = []
        for _ in range(args.e2e_steps):
            t_step = time.perf_counter()
            d2h = e2e_step()
            wall.append((time.perf_counter() - t_step) * 1e3)
        a1.record(stream)
        torch.cuda.synchronize()
        barrier()
        e2e_ms = max_over_ranks(a0.elapsed_time(a1) / args.e2e_steps, dist, "cuda")
        line["e2e"] = {"value": whole_job_rate(px_per_step, 1, world, e2e_ms),
                       "unit": "pixel-evals/s",
                       "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
                       "ms_per_step": e2e_ms, "wall_ms_each_step": wall,
                       "wall_ms_upload_slice_release": [
                           [round(x, 1) for x in ph] for ph in phase_wall[1:]],
                       "slice_workspace_peak_bytes": int(e2e_peak[0])}

    if world == 1 and not args.no_extra and plan["field_kernel"] == "footprint":
        # the same slice with the fused field and contour pass (no Sigma plane):
        # time per step and workspace, beside the default (Sigma plane); after the
        # end-to-end line, whose lattice uploads it would otherwise precede
        kw_u = dict(kw, fused=True)
        lat.slice(**kw_u, on_device=True).free()
        peak_u = cs.last_stats().device_bytes_peak
        u_ms = _event_ms(lambda: lat.slice(**kw_u, on_device=True).free(), args.steps, 1,
                         stream)
        line["fused_vs_unfused"] = {
            "fused_ms_per_step": u_ms, "unfused_ms_per_step": t_max / args.steps,
            "fused_workspace_peak_bytes": int(peak_u),
            "unfused_workspace_peak_bytes": int(peak_main),
            "basis": "the same steps through csl_slice_layers with CSL_SLICE_FUSED (each "
                     "tile's crossing vertices from shared memory, no Sigma plane) and without "
                     "(the default: Sigma plane, marching squares reads it); contours kept on "
                     "the device; workspace = largest device memory the call held at once"}

    if world == 1 and not args.no_extra:
        # self-support metrics (Eq. 11-14) of the same lattice, printing along z
        res = {}

        def support_step():
            res["v"] = lat.support_metrics((0.0, 0.0, 1.0), math.pi / 4)

        sms = _event_ms(support_step, args.steps, args.warmup, stream)
        line["support_metrics"] = {"workload": cfg["name"], "gamma": res["v"][0],
                                   "psi_percent": res["v"][1], "ms": sms,
                                   "struts_per_s": cfg["edges"].shape[0] / (sms / 1e3)}
        # the binary images alone (what a DLP printer takes, Sec. 4): no contours and no
        # Sigma plane; then the same with the bit-packed images copied to pinned host memory
        wpr = (cfg["nx"] + 31) // 32
        mask = torch.empty((cfg["n_layers"], cfg["ny"], wpr), dtype=torch.int32, device="cuda")
        host_mask = torch.empty(mask.shape, dtype=torch.int32, pin_memory=True)
        dms = _event_ms(lambda: lat.slice(**kw, contours=False, mask_out=mask), args.steps,
                        args.warmup, stream)

        def dlp_to_host():
            lat.slice(**kw, contours=False, mask_out=mask)
            host_mask.copy_(mask)

        hms = _event_ms(dlp_to_host, args.steps, args.warmup, stream)
        px = cfg["nx"] * cfg["ny"] * cfg["n_layers"]
        line["binary_images"] = {"workload": cfg["name"], "ms_per_step": dms,
                                 "pixel_evals_per_s": px / (dms / 1e3),
                                 "s_per_slice": dms / 1e3 / cfg["n_layers"],
                                 "to_host_ms_per_step": hms,
                                 "d2h_bytes_per_step": int(mask.numel() * 4)}
        del mask, host_mask
        # the same slicing from a host-resident lattice: records in page-locked host
        # memory, each chunk's z window copied to the device (the out-of-core sweep)
        t_up = time.perf_counter()
        lat_h = cs.Lattice(cfg["nodes"], cfg["edges"], cfg["radius"], R=cfg["R"], C=cfg["C"],
                           host_resident=True)
        up_s = time.perf_counter() - t_up
        hr = {}

        def host_resident_step():
            lat_h.slice(**kw, on_device=True).free()
            hr["peak"] = cs.last_stats().device_bytes_peak

        hr_ms = _event_ms(host_resident_step, args.steps, args.warmup, stream)
        ne, nn = int(cfg["edges"].shape[0]), int(cfg["nodes"].shape[0])
        line["host_resident"] = {
            "workload": cfg["name"], "ms_per_step": hr_ms,
            "pixel_evals_per_s": px / (hr_ms / 1e3), "upload_and_prepare_s": up_s,
            "lattice_device_bytes": nn * 12,
            "lattice_device_bytes_resident": nn * 12 + ne * (8 + 4 + 32 + 16 + 4 + 4 + 4),
            "slice_workspace_peak_bytes": int(hr.get("peak", 0)),
            "basis": "lattice bytes by layout (nodes only when host-resident; nodes, edges, "
                     "radii and the prepared arrays when resident); the workspace peak from "
                     "csl_last_stats"}
        del lat_h
        # the same slice, contours to host memory, within a device-memory
        # budget of 8 GB besides the lattice (chunks sized by the library)
        budget = 8 << 30
        lat.slice(**kw, workspace_budget=budget)
        bst = cs.last_stats()
        b_ms = _event_ms(lambda: lat.slice(**kw, workspace_budget=budget), 1, 0, stream)
        line["memory_budget"] = {
            "workload": cfg["name"], "budget_bytes": budget, "ms_per_step": b_ms,
            "pixel_evals_per_s": px / (b_ms / 1e3), "chunks": int(bst.chunks),
            "slice_workspace_peak_bytes": int(bst.device_bytes_peak),
            "unbounded_workspace_peak_bytes": int(line.get("e2e", {}).get(
                "slice_workspace_peak_bytes", 0)),
            "basis": "csl_slice_layers with workspace_budget, contours copied to host memory "
                     "chunk by chunk (pageable), one step timed with CUDA events; the "
                     "unbounded figure is the end-to-end line's"}
        del lat
        torch.cuda.empty_cache()
        line["at_10M"] = run_10m(args.steps, args.warmup)
        line["volume_fraction"] = run_vf(args.steps, args.warmup)
        line["batched_64"] = run_batch(args.steps, args.warmup)
        line["zigzag_infill_10M"] = run_hatch(args.steps, args.warmup)
        line["density_matching"] = run_density(args.steps, args.warmup)
        line["support_optimisation"] = run_support_opt(args.steps, args.warmup)
        line["depth_image"] = run_render(args.steps, args.warmup)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = oracle_sample(cfg)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
