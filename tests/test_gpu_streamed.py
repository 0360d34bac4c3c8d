"""Host-resident lattices (csl_lattice_upload_streamed): prepared in small
device batches merged on the host, sliced from per-chunk windows copied to the
device. The field and the contours equal those of the device-resident lattice
bit for bit."""
import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _slice(lat, cfg, n_layers, **kw):
    sig = torch.empty((n_layers, cfg["ny"], cfg["nx"]), dtype=torch.float32, device="cuda")
    cont = lat.slice(z0=cfg["z0"], dz=cfg["dz"], n_layers=n_layers, x0=cfg["x0"], y0=cfg["y0"],
                     nx=cfg["nx"], ny=cfg["ny"], pixel=cfg["pixel"], sigma_out=sig,
                     edge_ids=True, **kw)
    torch.cuda.synchronize()
    return sig, cont


def _same(a, b):
    assert torch.equal(a[0], b[0])
    for f in ("layer_loop_off", "loop_vert_off", "xy", "edge_id"):
        assert np.array_equal(getattr(a[1], f), getattr(b[1], f)), f


@pytest.mark.parametrize("batch,slab,chunk", [(100, 8, 0), (97, 2, 2), (5000, 4, 8)])
def test_cubic_bcc_streamed_equals_resident(batch, slab, chunk):
    import paper_2101_05031_gb300 as cs
    cfg = synth.config(1)
    res = cs.Lattice(cfg["nodes"], cfg["edges"], cfg["radius"], R=cfg["R"])
    st = cs.Lattice(cfg["nodes"], cfg["edges"], cfg["radius"], R=cfg["R"], host_resident=True,
                    batch_edges=batch)
    a, b = res.info(), st.info()
    assert (a.R, a.max_dz, a.max_radius) == (b.R, b.max_dz, b.max_radius)
    _same(_slice(res, cfg, 20, slab=slab, chunk_layers=chunk),
          _slice(st, cfg, 20, slab=slab, chunk_layers=chunk))


def test_freudenthal_streamed_equals_resident():
    import paper_2101_05031_gb300 as cs
    cfg = synth.config(2, small=True)
    res = cs.Lattice(cfg["nodes"], cfg["edges"], cfg["radius"], R=cfg["R"])
    st = cs.Lattice(cfg["nodes"], cfg["edges"], cfg["radius"], R=cfg["R"], host_resident=True,
                    batch_edges=1000)
    _same(_slice(res, cfg, cfg["n_layers"], chunk_layers=2, slab=2),
          _slice(st, cfg, cfg["n_layers"], chunk_layers=2, slab=2))


def test_graded_10M_streamed_windows():
    """The 10M-strut graded lattice at its full 2000^2 grid, prepared in four
    batches: a block of layers in the middle of the part."""
    import paper_2101_05031_gb300 as cs
    nodes, edges, radius, r_ref = synth.adaptive_graded(box=100.0, level_min=4, level_max=7)
    cfg = dict(x0=0.0, y0=0.0, nx=2000, ny=2000, pixel=0.05, z0=50.1, dz=0.2)
    res = cs.Lattice(nodes, edges, radius, R=1.5 * r_ref)
    st = cs.Lattice(nodes, edges, radius, R=1.5 * r_ref, host_resident=True,
                    batch_edges=(edges.shape[0] + 3) // 4)
    _same(_slice(res, cfg, 24, chunk_layers=8), _slice(st, cfg, 24, chunk_layers=8))


def test_streamed_lattice_serves_slicing_only():
    import paper_2101_05031_gb300 as cs
    cfg = synth.config(5, small=True)
    st = cs.Lattice(cfg["nodes"], cfg["edges"], cfg["radius"], R=cfg["R"], host_resident=True)
    with pytest.raises(cs.CslError) as e:
        cs.volume_fraction(st, cfg["cells"])
    assert e.value.code == 6
    with pytest.raises(cs.CslError) as e:
        st.support_metrics()
    assert e.value.code == 6


@pytest.mark.parametrize("on_device", [False, True])
def test_streamed_chunk_buffers_reused_equal_resident(on_device):
    """Two chunks in flight with the library's own Sigma and mask buffers:
    chunk k + 2 reuses chunk k's buffers once its contours (on their own
    stream) are done. Ten 2-layer chunks, contours (host or device output)
    bit-identical to the device-resident lattice's."""
    import paper_2101_05031_gb300 as cs
    cfg = synth.config(1)
    res = cs.Lattice(cfg["nodes"], cfg["edges"], cfg["radius"], R=cfg["R"])
    st = cs.Lattice(cfg["nodes"], cfg["edges"], cfg["radius"], R=cfg["R"], host_resident=True,
                    batch_edges=300)
    kw = dict(z0=cfg["z0"], dz=cfg["dz"], n_layers=20, x0=cfg["x0"], y0=cfg["y0"],
              nx=cfg["nx"], ny=cfg["ny"], pixel=cfg["pixel"], edge_ids=True, slab=2,
              chunk_layers=2, on_device=on_device)
    a = res.slice(**kw)
    b = st.slice(**kw)
    if on_device:
        a, b = a.to_host(), b.to_host()
    for f in ("layer_loop_off", "loop_vert_off", "xy", "edge_id"):
        assert np.array_equal(getattr(a, f), getattr(b, f)), f
    assert a.xy.shape[0] > 0
