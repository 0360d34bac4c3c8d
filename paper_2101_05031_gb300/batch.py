"""Batched slicing (C ABI: csl_batch_*): many (lattice, slicing request) jobs
planned once and replayed as one CUDA graph whose field stage is a single
persistent launch. Only argument marshalling happens here."""
from __future__ import annotations

import ctypes

from . import _lib
from .slicer import ContourSet, Lattice, _host_contours, _stream_ptr

try:
    import torch
except Exception:  # pragma: no cover
    torch = None


class _DeviceArray:
    """__cuda_array_interface__ over a library-owned device array."""

    def __init__(self, ptr, shape, owner):
        self.__cuda_array_interface__ = {"shape": tuple(shape), "typestr": "<f4",
                                         "data": (ptr, False), "version": 2, "strides": None}
        self._owner = owner


class Batch:
    """jobs: list of (Lattice, dict(z0, dz, n_layers, x0, y0, nx, ny, pixel
    [, edge_ids])). autotune: time the field kernel and tile, slab depth x CTAs
    per SM and the staging chunk, and keep the best (cached per process for
    the same job sizes); otherwise field_kernel ("auto" = "block", or
    "footprint"), tile (0, 16, 32) and stage_records (0 = 256) as given."""

    def __init__(self, jobs, *, autotune=False, slab=0, ctas_per_sm=0, branches=0,
                 field_kernel="auto", tile=0, stage_records=0, stream=None):
        n = len(jobs)
        self._lats = [lat for lat, _ in jobs]   # the lattices must outlive the batch
        self._shapes = []
        descs = (_lib.SliceDesc * n)()
        handles = (ctypes.c_void_p * n)()
        for j, (lat, d) in enumerate(jobs):
            if not isinstance(lat, Lattice):
                raise TypeError("jobs must be (Lattice, dict) pairs")
            handles[j] = lat.handle
            x = descs[j]
            x.z0, x.dz, x.n_layers = float(d["z0"]), float(d["dz"]), int(d["n_layers"])
            x.nx, x.ny = int(d["nx"]), int(d["ny"])
            x.x0, x.y0, x.pixel = float(d["x0"]), float(d["y0"]), float(d["pixel"])
            x.flags = _lib.SLICE_EDGE_IDS if d.get("edge_ids") else 0
            self._shapes.append((x.n_layers, x.ny, x.nx))
        opts = _lib.BatchOpts(1 if autotune else 0, int(slab), int(ctas_per_sm), int(branches),
                              _lib.FIELD_KERNELS[field_kernel], int(tile), int(stage_records), 0)
        h = ctypes.c_void_p()
        _lib.check(_lib.load().csl_batch_create(handles, descs, n, ctypes.byref(opts),
                                                _stream_ptr(stream), ctypes.byref(h)))
        self._h = h

    def run(self, stream=None):
        _lib.check(_lib.load().csl_batch_run(self._h, _stream_ptr(stream)))

    def contours(self, j) -> ContourSet:
        out = ctypes.POINTER(_lib.Contours)()
        _lib.check(_lib.load().csl_batch_contours(self._h, int(j), 0, ctypes.byref(out)))
        return _host_contours(out)

    def sigma(self, j):
        """Job j's Sigma as a CUDA tensor view [n_layers, ny, nx] (overwritten by run)."""
        p = ctypes.c_void_p()
        _lib.check(_lib.load().csl_batch_sigma(self._h, int(j), ctypes.byref(p)))
        return torch.as_tensor(_DeviceArray(p.value, self._shapes[j], self), device="cuda")

    def info(self) -> _lib.BatchInfo:
        out = _lib.BatchInfo()
        _lib.check(_lib.load().csl_batch_get_info(self._h, ctypes.byref(out)))
        return out

    def close(self):
        if getattr(self, "_h", None):
            _lib.load().csl_batch_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
