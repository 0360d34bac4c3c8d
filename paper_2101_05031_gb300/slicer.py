"""Python face of libcslice: lattices, slicing and contours.

Only argument marshalling happens here; every step of the method runs in the
CUDA library. Inputs may be numpy arrays (host) or torch tensors (host or
CUDA); outputs are numpy arrays (host contours) or stay in device memory.
"""
from __future__ import annotations

import ctypes
from dataclasses import dataclass

import numpy as np

from . import _lib

try:  # torch is plumbing only: device buffers and streams
    import torch
except Exception:  # pragma: no cover - the CPU test image has torch
    torch = None


def _stream_ptr(stream):
    if stream is None:
        if torch is not None and torch.cuda.is_available():
            return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
        return ctypes.c_void_p(0)
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(stream.cuda_stream)


def _as_buffer(x, dtype, width):
    """Returns (pointer, n_rows, on_device, keepalive)."""
    if torch is not None and isinstance(x, torch.Tensor):
        tdt = {np.float32: torch.float32, np.int32: torch.int32}[dtype]
        t = x.detach().to(tdt).contiguous()
        n = t.numel() // width
        return ctypes.c_void_p(t.data_ptr()), n, t.is_cuda, t
    a = np.ascontiguousarray(x, dtype=dtype)
    n = a.size // width
    return a.ctypes.data_as(ctypes.c_void_p), n, False, a


@dataclass
class ContourSet:
    """Closed loops of every layer (host arrays).

    layer_loop_off[n_layers + 1], loop_vert_off[n_loops + 1], xy[n_verts, 2]
    (mm), edge_id[n_verts] (or None)."""
    layer_loop_off: np.ndarray
    loop_vert_off: np.ndarray
    xy: np.ndarray
    edge_id: np.ndarray | None

    @property
    def n_layers(self):
        return len(self.layer_loop_off) - 1

    def layer(self, k):
        """Loops of layer k as a list of (edge_id or None, xy) arrays."""
        out = []
        for li in range(self.layer_loop_off[k], self.layer_loop_off[k + 1]):
            a, b = self.loop_vert_off[li], self.loop_vert_off[li + 1]
            out.append((None if self.edge_id is None else self.edge_id[a:b], self.xy[a:b]))
        return out


class DeviceContours:
    """Contours left in device memory (CSL_SLICE_CONTOURS_ON_DEVICE)."""

    def __init__(self, ptr):
        self._ptr = ptr
        c = ptr.contents
        self.n_layers, self.n_loops, self.n_verts = c.n_layers, c.n_loops, c.n_verts
        self.has_edge_ids = bool(c.edge_id)

    def to_host(self) -> ContourSet:
        lo = np.empty(self.n_layers + 1, np.int64)
        vo = np.empty(self.n_loops + 1, np.int64)
        xy = np.empty((self.n_verts, 2), np.float32)
        eid = np.empty(self.n_verts, np.int32) if self.has_edge_ids else None
        _lib.check(_lib.load().csl_contours_copy(
            self._ptr, lo.ctypes.data_as(ctypes.c_void_p), vo.ctypes.data_as(ctypes.c_void_p),
            xy.ctypes.data_as(ctypes.c_void_p),
            eid.ctypes.data_as(ctypes.c_void_p) if eid is not None else None, 0, _stream_ptr(None)))
        return ContourSet(lo, vo, xy, eid)

    def hatch(self, y0, spacing, n_lines, stream=None):
        """Zigzag infill (csl_hatch_layers): (layer_seg_off[n_layers + 1],
        seg[n_segments, 3] = (x_from, x_to, y) in toolpath order), host arrays."""
        lib = _lib.load()
        h = ctypes.POINTER(_lib.Hatches)()
        _lib.check(lib.csl_hatch_layers(self._ptr, float(y0), float(spacing), int(n_lines), 0,
                                        _stream_ptr(stream), ctypes.byref(h)))
        try:
            c = h.contents
            off = np.ctypeslib.as_array((ctypes.c_int64 * (c.n_layers + 1)).from_address(
                c.layer_seg_off)).copy()
            n = c.n_segments
            seg = (np.ctypeslib.as_array((ctypes.c_float * (3 * n)).from_address(c.seg)).copy()
                   .reshape(n, 3) if n else np.zeros((0, 3), np.float32))
        finally:
            lib.csl_hatches_free(h)
        return off, seg

    @classmethod
    def from_host(cls, layer_loop_off, loop_vert_off, xy, edge_id=None, stream=None):
        """csl_contours_create: device contours from host arrays in the layout
        of csl_contours (offsets int64, xy float32 [n, 2], edge ids int32)."""
        lo = np.ascontiguousarray(layer_loop_off, dtype=np.int64)
        vo = np.ascontiguousarray(loop_vert_off, dtype=np.int64)
        xy = np.ascontiguousarray(xy, dtype=np.float32).reshape(-1, 2)
        eid = None if edge_id is None else np.ascontiguousarray(edge_id, dtype=np.int32)
        if lo.ndim != 1 or vo.ndim != 1 or lo.size < 1 or vo.size < 1:
            raise ValueError("offsets must be 1-D with at least one entry")
        if eid is not None and eid.shape != (xy.shape[0],):
            raise ValueError("edge_id must have one entry per vertex")
        out = ctypes.POINTER(_lib.Contours)()
        _lib.check(_lib.load().csl_contours_create(
            lo.size - 1, vo.size - 1, xy.shape[0], lo.ctypes.data_as(ctypes.c_void_p),
            vo.ctypes.data_as(ctypes.c_void_p), xy.ctypes.data_as(ctypes.c_void_p),
            eid.ctypes.data_as(ctypes.c_void_p) if eid is not None else None,
            _stream_ptr(stream), ctypes.byref(out)))
        return cls(out)

    def smooth(self, x0, y0, pixel, nx, ny, lam=0.5, margin=0.05, iterations=4, stream=None):
        """csl_smooth_contours, in place: every vertex slides along its own grid
        edge toward its loop neighbours (needs edge ids). Returns self."""
        _lib.check(_lib.load().csl_smooth_contours(self._ptr, float(x0), float(y0), float(pixel),
                                                   int(nx), int(ny), float(lam), float(margin),
                                                   int(iterations), _stream_ptr(stream)))
        return self

    def simplify(self, nx, ny, tol, stream=None):
        """csl_simplify_contours: new DeviceContours with vertices dropped where
        that cannot create an intersection (needs edge ids; tol in mm)."""
        out = ctypes.POINTER(_lib.Contours)()
        _lib.check(_lib.load().csl_simplify_contours(self._ptr, int(nx), int(ny), float(tol),
                                                     _stream_ptr(stream), ctypes.byref(out)))
        return DeviceContours(out)

    def free(self):
        if self._ptr is not None:
            _lib.load().csl_contours_free(self._ptr)
            self._ptr = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


class _ContoursOwner:
    """Frees a library-owned csl_contours when the last array viewing it dies."""

    def __init__(self, ptr):
        self.ptr = ptr

    def __del__(self):
        try:
            _lib.load().csl_contours_free(self.ptr)
        except Exception:
            pass


def _host_contours(ptr) -> ContourSet:
    """Wraps the library's host arrays without copying them."""
    c = ptr.contents
    owner = _ContoursOwner(ptr)
    nl, nloops, nv = c.n_layers, c.n_loops, c.n_verts

    def view(addr, n, ct, dtype):
        if n == 0:
            return np.zeros(0, dtype=dtype)
        buf = (ct * n).from_address(addr)
        buf._owner = owner
        return np.frombuffer(buf, dtype=dtype)

    lo = view(c.layer_loop_off, nl + 1, ctypes.c_int64, np.int64)
    vo = view(c.loop_vert_off, nloops + 1, ctypes.c_int64, np.int64)
    xy = view(c.xy, 2 * nv, ctypes.c_float, np.float32).reshape(nv, 2)
    eid = view(c.edge_id, nv, ctypes.c_int32, np.int32) if c.edge_id else None
    return ContourSet(lo, vo, xy, eid)


class Lattice:
    """A lattice uploaded to the GPU (csl_lattice_upload).

    nodes float[Nn, 3] (mm), edges int32[Ne, 2], radius float[Ne] (PHYSICAL:
    strut radius; RAW: the paper's r_i weight). R None -> 1.5 x max radius."""

    def __init__(self, nodes, edges, radius, R=None, C=1.0, mode="physical", stream=None,
                 host_resident=False, batch_edges=0):
        """host_resident=True: csl_lattice_upload_streamed (host arrays; the
        prepared records stay in page-locked host memory, at most batch_edges
        edges on the device while preparing, and slicing streams each chunk's
        window; the lattice then serves slicing only)."""
        lib = _lib.load()
        pn, nn, dn, kn = _as_buffer(nodes, np.float32, 3)
        pe, ne, de, ke = _as_buffer(edges, np.int32, 2)
        pr, nr, dr, kr = _as_buffer(radius, np.float32, 1)
        if nr != ne:
            raise ValueError("radius needs one value per edge")
        if not (dn == de == dr):
            raise ValueError("nodes, edges and radius must all be host or all device")
        params = _lib.Params(float(R) if R else 0.0, float(C),
                             _lib.MODE_RAW if mode == "raw" else _lib.MODE_PHYSICAL, int(dn))
        h = ctypes.c_void_p()
        if host_resident:
            _lib.check(lib.csl_lattice_upload_streamed(pn, nn, pe, pr, ne, ctypes.byref(params),
                                                       int(batch_edges), _stream_ptr(stream),
                                                       ctypes.byref(h)))
        else:
            _lib.check(lib.csl_lattice_upload(pn, nn, pe, pr, ne, ctypes.byref(params),
                                              _stream_ptr(stream), ctypes.byref(h)))
        self._h = h
        del kn, ke, kr
        info = self.info()
        self.R, self.C = info.R, info.C
        self.n_nodes, self.n_edges = info.n_nodes, info.n_edges

    @property
    def handle(self):
        return self._h

    def info(self) -> _lib.LatticeInfo:
        out = _lib.LatticeInfo()
        _lib.check(_lib.load().csl_lattice_get_info(self._h, ctypes.byref(out)))
        return out

    def update(self, nodes=None, radius=None, stream=None):
        """Replace node positions / radii with CUDA tensors (same edges)."""
        keep = []
        pn = pr = None
        if nodes is not None:
            t = nodes.detach().to(torch.float32).contiguous()
            keep.append(t)
            pn = ctypes.c_void_p(t.data_ptr())
        if radius is not None:
            t = radius.detach().to(torch.float32).contiguous()
            keep.append(t)
            pr = ctypes.c_void_p(t.data_ptr())
        _lib.check(_lib.load().csl_lattice_update(self._h, pn, pr, _stream_ptr(stream)))

    def _desc(self, z0, dz, n_layers, x0, y0, nx, ny, pixel, flags, sigma_out, slab, chunk_layers,
              mask_out=None, tile=0, field_kernel="auto", stage_records=0):
        d = _lib.SliceDesc()
        d.mask_out = ctypes.c_void_p(mask_out.data_ptr()) if mask_out is not None else None
        d.z0, d.dz, d.n_layers = float(z0), float(dz), int(n_layers)
        d.nx, d.ny, d.flags = int(nx), int(ny), int(flags)
        d.x0, d.y0, d.pixel = float(x0), float(y0), float(pixel)
        d.sigma_out = ctypes.c_void_p(sigma_out.data_ptr()) if sigma_out is not None else None
        d.tile, d.slab, d.chunk_layers = int(tile), int(slab), int(chunk_layers)
        d.field_kernel = _lib.FIELD_KERNELS[field_kernel]
        d.stage_records = int(stage_records)
        return d

    def slice(self, *, z0, dz, n_layers, x0, y0, nx, ny, pixel, sigma_out=None, mask_out=None,
              contours=True, on_device=False, edge_ids=False, slab=0, chunk_layers=0,
              time_kernels=False, count_pairs=False, stream=None, tile=0, field_kernel="auto",
              stage_records=0, fused=False, workspace_budget=0):
        """csl_slice_layers. sigma_out: optional CUDA float32 tensor
        [n_layers, ny, nx] that receives Sigma; mask_out: optional CUDA int32
        tensor [n_layers, ny, ceil(nx / 32)] that receives the bit-packed inside
        mask (bit i % 32 of word i / 32: pixel i inside). field_kernel: "auto",
        "block" or "footprint"; tile: 0 (auto), 16 or 32; stage_records: records
        per staged copy of the footprint kernel (0: 256); fused: with the
        footprint kernel, the fused field and contour pass (no Sigma plane; the
        same contours as the default, which writes a Sigma plane and runs
        marching squares on it); workspace_budget: bytes of device memory the
        call may hold besides the lattice (0: no limit; host contours). Returns a ContourSet
        (host), a DeviceContours (on_device=True) or None (contours=False)."""
        if sigma_out is not None:
            if not (sigma_out.is_cuda and sigma_out.dtype == torch.float32
                    and sigma_out.is_contiguous()
                    and sigma_out.numel() >= int(n_layers) * int(ny) * int(nx)):
                raise ValueError("sigma_out must be a contiguous CUDA float32 tensor "
                                 "of n_layers * ny * nx elements")
        if mask_out is not None:
            wpr = (int(nx) + 31) // 32
            if not (mask_out.is_cuda and mask_out.element_size() == 4 and mask_out.is_contiguous()
                    and mask_out.numel() >= int(n_layers) * int(ny) * wpr):
                raise ValueError("mask_out must be a contiguous CUDA tensor of 32-bit words, "
                                 "n_layers * ny * ceil(nx / 32) of them")
        flags = 0
        if not contours:
            flags |= _lib.SLICE_NO_CONTOURS
        if on_device:
            flags |= _lib.SLICE_CONTOURS_ON_DEVICE
        if edge_ids:
            flags |= _lib.SLICE_EDGE_IDS
        if time_kernels:
            flags |= _lib.SLICE_TIME_KERNELS
        if count_pairs:
            flags |= _lib.SLICE_COUNT_PAIRS
        if fused:
            flags |= _lib.SLICE_FUSED
        d = self._desc(z0, dz, n_layers, x0, y0, nx, ny, pixel, flags, sigma_out, slab,
                       chunk_layers, mask_out, tile, field_kernel, stage_records)
        d.workspace_budget = int(workspace_budget)
        out = ctypes.POINTER(_lib.Contours)()
        _lib.check(_lib.load().csl_slice_layers(self._h, ctypes.byref(d), _stream_ptr(stream),
                                                ctypes.byref(out)))
        if not contours:
            return None
        if on_device:
            return DeviceContours(out)
        return _host_contours(out)

    def slab_bins(self, *, z0, dz, first_layer, n_slab_layers, x0, y0, nx, ny, pixel,
                  tile=16, halo=False, stream=None):
        """Binner output for one slab of tiles of `tile` pixels (16 or 32), with
        the fused pass's one-pixel halo or without: (tile_off[n_tiles+1], edge
        ids sorted per tile)."""
        kern = "footprint" if (tile == 32 or halo) else "auto"
        d = self._desc(z0, dz, first_layer + n_slab_layers, x0, y0, nx, ny, pixel,
                       _lib.SLICE_FUSED if halo else 0, None, 0, 0, tile=tile,
                       field_kernel=kern)
        n_tiles = ((int(nx) + tile - 1) // tile) * ((int(ny) + tile - 1) // tile)
        off = np.zeros(n_tiles + 1, np.int64)
        n = ctypes.c_int64()
        lib = _lib.load()
        st = lib.csl_debug_slab_bins(self._h, ctypes.byref(d), int(first_layer),
                                     int(n_slab_layers), off.ctypes.data_as(ctypes.c_void_p),
                                     None, 0, ctypes.byref(n), _stream_ptr(stream))
        if st not in (_lib.CSL_OK, 5):
            _lib.check(st)
        ids = np.zeros(max(1, n.value), np.int32)
        _lib.check(lib.csl_debug_slab_bins(self._h, ctypes.byref(d), int(first_layer),
                                           int(n_slab_layers), off.ctypes.data_as(ctypes.c_void_p),
                                           ids.ctypes.data_as(ctypes.c_void_p), ids.size,
                                           ctypes.byref(n), _stream_ptr(stream)))
        return off, ids[:n.value]

    def support_metrics(self, t_p=(0.0, 0.0, 1.0), alpha=np.pi / 4, coeffs=None, stream=None):
        """(Gamma, Psi) of Eq. 13-14 for printing direction t_p and angle alpha
        (csl_support_metrics); coeffs: a_0..a_5 of g(theta), None for the paper's."""
        t = (ctypes.c_double * 3)(*[float(v) for v in t_p])
        a = (ctypes.c_double * 6)(*[float(v) for v in coeffs]) if coeffs is not None else None
        g, p = ctypes.c_double(), ctypes.c_double()
        _lib.check(_lib.load().csl_support_metrics(self._h, t, float(alpha), a, ctypes.byref(g),
                                                   ctypes.byref(p), _stream_ptr(stream)))
        return g.value, p.value

    def render_depth(self, *, eye, target, up=(0.0, 0.0, 1.0), fov_y=0.7, width, height,
                     step, refine=24, out=None, stream=None):
        """csl_render_depth: distances along the pixels' rays to the solid, a
        CUDA float32 tensor [height, width] (+inf where a ray misses)."""
        if out is None:
            out = torch.empty((int(height), int(width)), dtype=torch.float32, device="cuda")
        if not (out.is_cuda and out.dtype == torch.float32 and out.is_contiguous()
                and out.numel() >= int(width) * int(height)):
            raise ValueError("out must be a contiguous CUDA float32 tensor of width * height")
        cam = _lib.Camera((ctypes.c_double * 3)(*[float(v) for v in eye]),
                          (ctypes.c_double * 3)(*[float(v) for v in target]),
                          (ctypes.c_double * 3)(*[float(v) for v in up]), float(fov_y),
                          int(width), int(height), float(step), int(refine), 0)
        _lib.check(_lib.load().csl_render_depth(self._h, ctypes.byref(cam),
                                                ctypes.c_void_p(out.data_ptr()),
                                                _stream_ptr(stream)))
        return out

    def close(self):
        if getattr(self, "_h", None):
            _lib.load().csl_lattice_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def measure_fp32_peak(stream=None):
    """(TFLOP/s of an FFMA microbenchmark at full occupancy, nominal max SM clock in GHz)."""
    t = ctypes.c_double()
    g = ctypes.c_double()
    _lib.check(_lib.load().csl_measure_fp32_peak(ctypes.byref(t), ctypes.byref(g),
                                                 _stream_ptr(stream)))
    return t.value, g.value


def last_stats() -> _lib.Stats:
    s = _lib.Stats()
    _lib.check(_lib.load().csl_last_stats(ctypes.byref(s)))
    return s
