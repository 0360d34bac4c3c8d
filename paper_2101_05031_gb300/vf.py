"""Smoothed volume fraction per density cell and its adjoint (C ABI:
csl_volume_fraction, csl_volume_fraction_backward), with a
torch.autograd.Function so that strut radii and node positions can be tuned
toward a target density by gradient steps (the radius tuning of Sec. 5.4).
Only argument marshalling happens here."""
from __future__ import annotations

import ctypes

import torch

from . import _lib
from .slicer import Lattice, _stream_ptr


def cells_desc(cells) -> _lib.CellsDesc:
    """cells: dict(origin=(x, y, z), h=..., dims=(cx, cy, cz), m=..., T=...)."""
    d = _lib.CellsDesc()
    for k in range(3):
        d.origin[k] = float(cells["origin"][k])
        d.dims[k] = int(cells["dims"][k])
    d.h = float(cells["h"])
    d.m = int(cells["m"])
    d.temperature = float(cells["T"])
    return d


def _shape(cells):
    cx, cy, cz = (int(v) for v in cells["dims"])
    return (cz, cy, cx)


def volume_fraction(lat: Lattice, cells, out: torch.Tensor | None = None, stream=None):
    """vf[cz, cy, cx] (CUDA float32) of the uploaded lattice."""
    if out is None:
        out = torch.empty(_shape(cells), dtype=torch.float32, device="cuda")
    d = cells_desc(cells)
    _lib.check(_lib.load().csl_volume_fraction(lat.handle, ctypes.byref(d),
                                               ctypes.c_void_p(out.data_ptr()),
                                               _stream_ptr(stream)))
    return out


def volume_fraction_backward(lat: Lattice, cells, grad_vf: torch.Tensor, stream=None):
    """(grad_radius[n_edges], grad_nodes[n_nodes, 3]) of sum(grad_vf * vf)."""
    g = grad_vf.detach().to(torch.float32).contiguous()
    gr = torch.empty(lat.n_edges, dtype=torch.float32, device="cuda")
    gn = torch.empty((lat.n_nodes, 3), dtype=torch.float32, device="cuda")
    d = cells_desc(cells)
    _lib.check(_lib.load().csl_volume_fraction_backward(
        lat.handle, ctypes.byref(d), ctypes.c_void_p(g.data_ptr()),
        ctypes.c_void_p(gr.data_ptr()), ctypes.c_void_p(gn.data_ptr()), _stream_ptr(stream)))
    return gr, gn


class VolumeFraction(torch.autograd.Function):
    """vf = VolumeFraction.apply(radius, nodes, lattice, cells).

    radius (n_edges) and nodes (n_nodes, 3) are CUDA tensors; the lattice's
    device copy is updated from them (csl_lattice_update) before the forward
    pass. Backward recomputes the field (nothing is stored in between)."""

    @staticmethod
    def forward(ctx, radius, nodes, lattice: Lattice, cells):
        lattice.update(nodes=nodes, radius=radius)
        ctx.lattice = lattice
        ctx.cells = cells
        return volume_fraction(lattice, cells)

    @staticmethod
    def backward(ctx, grad_vf):
        gr, gn = volume_fraction_backward(ctx.lattice, ctx.cells, grad_vf)
        return gr, gn, None, None
