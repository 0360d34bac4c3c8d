"""GPU slicing path vs the FP64 oracle (field, classification, contours, bins)."""
import math

import numpy as np
import pytest

import oracle
import synth
from oracle import binning
from tests import helpers

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _cslice():
    import paper_2101_05031_gb300 as cs
    return cs


def gpu_slice(lat, cfg, *, z0=None, n_layers=None, slab=0, chunk_layers=0, edge_ids=True,
              nx=None, ny=None, x0=None, y0=None):
    nx = nx or cfg["nx"]
    ny = ny or cfg["ny"]
    x0 = cfg["x0"] if x0 is None else x0
    y0 = cfg["y0"] if y0 is None else y0
    z0 = cfg["z0"] if z0 is None else z0
    nl = cfg["n_layers"] if n_layers is None else n_layers
    sig = torch.empty((nl, ny, nx), dtype=torch.float32, device="cuda")
    cont = lat.slice(z0=z0, dz=cfg["dz"], n_layers=nl, x0=x0, y0=y0, nx=nx, ny=ny,
                     pixel=cfg["pixel"], sigma_out=sig, edge_ids=edge_ids, slab=slab,
                     chunk_layers=chunk_layers)
    torch.cuda.synchronize()
    return sig.cpu().numpy(), cont


def oracle_slice(cfg, *, z0=None, n_layers=None, nx=None, ny=None, x0=None, y0=None):
    return oracle.slice_sigma(cfg["nodes"], cfg["edges"], cfg["radius"], R=cfg["R"], C=cfg["C"],
                              z0=cfg["z0"] if z0 is None else z0, dz=cfg["dz"],
                              n_layers=cfg["n_layers"] if n_layers is None else n_layers,
                              x0=cfg["x0"] if x0 is None else x0,
                              y0=cfg["y0"] if y0 is None else y0,
                              nx=nx or cfg["nx"], ny=ny or cfg["ny"], pixel=cfg["pixel"])


def check_contours(cont, sig_ref, cfg, x0=None, y0=None):
    tot_m = tot_x = 0
    for k in range(sig_ref.shape[0]):
        m, x = helpers.compare_layer_contours(cont.layer(k), sig_ref[k],
                                              x0=cfg["x0"] if x0 is None else x0,
                                              y0=cfg["y0"] if y0 is None else y0,
                                              pixel=cfg["pixel"], C=cfg["C"])
        tot_m += m
        tot_x += x
    assert tot_m > 0
    assert tot_x <= 0.02 * (tot_m + tot_x) + 2
    return tot_m, tot_x


@pytest.fixture(scope="module")
def c1():
    cfg = synth.config(1)
    cs = _cslice()
    lat = cs.Lattice(cfg["nodes"], cfg["edges"], cfg["radius"], R=cfg["R"])
    return cfg, lat


def test_non_finite_dz_is_refused_for_one_layer(c1):
    """Layer k lies at z0 + k dz, so even a single layer needs a finite dz."""
    cfg, lat = c1
    import paper_2101_05031_gb300 as cs
    for dz in (float("inf"), float("nan")):
        with pytest.raises(cs.CslError, match="INVALID_ARG"):
            lat.slice(z0=1.0, dz=dz, n_layers=1, x0=0.0, y0=0.0, nx=16, ny=16, pixel=0.1,
                      contours=False, sigma_out=torch.empty((1, 16, 16), device="cuda"))


def test_c1_full_parity(c1):
    """Configuration 1 in full (812 struts, 200x200 px, 50 layers)."""
    cfg, lat = c1
    sig, cont = gpu_slice(lat, cfg)
    ref = oracle_slice(cfg)
    helpers.assert_field(sig, ref, cfg["C"])
    check_contours(cont, ref, cfg)


@pytest.mark.parametrize("slab", [1, 2, 4, 8])
def test_c1_slab_depths_agree(c1, slab):
    cfg, lat = c1
    sig, cont = gpu_slice(lat, cfg, n_layers=13, slab=slab, chunk_layers=slab * 2)
    ref = oracle_slice(cfg, n_layers=13)
    helpers.assert_field(sig, ref, cfg["C"])
    check_contours(cont, ref, cfg)


def test_c2_small_parity():
    cfg = synth.config(2, small=True)
    cs = _cslice()
    lat = cs.Lattice(cfg["nodes"], cfg["edges"], cfg["radius"], R=cfg["R"])
    sig, cont = gpu_slice(lat, cfg)
    ref = oracle_slice(cfg)
    helpers.assert_field(sig, ref, cfg["C"])
    check_contours(cont, ref, cfg)


def test_c3_small_parity():
    cfg = synth.config(3, small=True)
    cs = _cslice()
    lat = cs.Lattice(cfg["nodes"], cfg["edges"], cfg["radius"], R=cfg["R"])
    sig, cont = gpu_slice(lat, cfg)
    ref = oracle_slice(cfg)
    helpers.assert_field(sig, ref, cfg["C"])
    check_contours(cont, ref, cfg)


def test_ragged_grid_and_offsets(c1):
    """Grid sizes that are not multiples of the 16-pixel tile, an odd origin."""
    cfg, lat = c1
    kw = dict(nx=37, ny=23, x0=3.217, y0=8.05, z0=1.13, n_layers=5)
    sig, cont = gpu_slice(lat, cfg, **kw)
    ref = oracle_slice(cfg, **kw)
    helpers.assert_field(sig, ref, cfg["C"])
    check_contours(cont, ref, cfg, x0=kw["x0"], y0=kw["y0"])


def test_single_pixel_and_far_grid(c1):
    cfg, lat = c1
    sig, cont = gpu_slice(lat, cfg, nx=1, ny=1, x0=2.45, y0=2.45, z0=2.5, n_layers=3)
    ref = oracle_slice(cfg, nx=1, ny=1, x0=2.45, y0=2.45, z0=2.5, n_layers=3)
    helpers.assert_field(sig, ref, cfg["C"])
    assert cont.n_layers == 3
    sig, cont = gpu_slice(lat, cfg, nx=40, ny=30, x0=100.0, y0=100.0, n_layers=2)
    assert np.all(sig == 0) and len(cont.loop_vert_off) == 1


def test_empty_lattice_and_zero_layers():
    cs = _cslice()
    lat = cs.Lattice(np.zeros((0, 3), np.float32), np.zeros((0, 2), np.int32),
                     np.zeros(0, np.float32), R=1.0)
    sig = torch.full((2, 20, 20), 7.0, device="cuda")
    cont = lat.slice(z0=0, dz=1, n_layers=2, x0=0, y0=0, nx=20, ny=20, pixel=0.1, sigma_out=sig)
    assert float(sig.abs().max()) == 0.0
    assert cont.layer_loop_off.tolist() == [0, 0, 0] and cont.xy.shape == (0, 2)
    c1cfg = synth.config(1)
    lat = cs.Lattice(c1cfg["nodes"], c1cfg["edges"], c1cfg["radius"])
    cont = lat.slice(z0=0, dz=1, n_layers=0, x0=0, y0=0, nx=20, ny=20, pixel=0.1)
    assert cont.layer_loop_off.tolist() == [0]


def test_zero_length_and_horizontal_struts():
    """Degenerate edges: a zero-length edge contributes nothing; edges lying
    in a slicing plane are handled by the horizontal branch."""
    cs = _cslice()
    nodes = np.array([[0, 0, 1.0], [2, 0, 1.0], [2, 0, 1.0], [0, 2, 1.0], [1, 1, 0.2]],
                     np.float32)
    edges = np.array([[0, 1], [1, 2], [0, 3], [3, 4], [2, 2]], np.int32)
    radius = np.full(5, 0.3, np.float32)
    cfg = dict(nodes=nodes, edges=edges, radius=radius, R=0.45, C=1.0, x0=-0.6, y0=-0.6,
               nx=70, ny=70, pixel=0.05, z0=0.8, dz=0.1, n_layers=5)
    lat = cs.Lattice(nodes, edges, radius, R=0.45)
    sig, cont = gpu_slice(lat, cfg)
    ref = oracle_slice(cfg)
    helpers.assert_field(sig, ref, 1.0)
    check_contours(cont, ref, cfg)


def test_raw_mode_parity():
    """The paper's literal r_i weights (RAW mode) and a non-unit iso-value."""
    cs = _cslice()
    cfg = synth.config(1)
    w = np.full(cfg["edges"].shape[0], 2.4, np.float32)
    lat = cs.Lattice(cfg["nodes"], cfg["edges"], w, R=0.75, C=1.7, mode="raw")
    sig = torch.empty((4, 200, 200), device="cuda")
    lat.slice(z0=0.9, dz=0.7, n_layers=4, x0=0, y0=0, nx=200, ny=200, pixel=0.1,
              sigma_out=sig, contours=False)
    ref = oracle.slice_sigma(cfg["nodes"], cfg["edges"], w, R=0.75, C=1.7, mode=oracle.RAW,
                             z0=0.9, dz=0.7, n_layers=4, x0=0, y0=0, nx=200, ny=200, pixel=0.1)
    helpers.assert_field(sig.cpu().numpy(), ref, 1.7)


def test_invalid_inputs_rejected():
    cs = _cslice()
    nodes = np.array([[0, 0, 0], [1, 0, 0]], np.float32)
    with pytest.raises(cs.CslError, match="INVALID_ARG"):
        cs.Lattice(nodes, np.array([[0, 2]], np.int32), np.array([0.1], np.float32))
    with pytest.raises(cs.CslError, match="INVALID_ARG"):
        cs.Lattice(np.array([[0, 0, np.nan], [1, 0, 0]], np.float32), np.array([[0, 1]]),
                   np.array([0.1], np.float32))
    with pytest.raises(cs.CslError, match="INVALID_ARG"):
        cs.Lattice(nodes, np.array([[0, 1]]), np.array([0.5], np.float32), R=0.5)
    with pytest.raises(cs.CslError, match="INVALID_ARG"):
        cs.Lattice(nodes, np.array([[0, 1]]), np.array([-0.1], np.float32))
    lat = cs.Lattice(nodes, np.array([[0, 1]]), np.array([0.1], np.float32))
    for bad in (dict(dz=0.0), dict(pixel=-1.0), dict(nx=0), dict(n_layers=-1)):
        kw = dict(z0=0, dz=0.1, n_layers=3, x0=0, y0=0, nx=10, ny=10, pixel=0.1)
        kw.update(bad)
        with pytest.raises(cs.CslError, match="INVALID_ARG"):
            lat.slice(**kw)
    with pytest.raises(cs.CslError, match="INVALID_ARG"):
        lat.slice(z0=0, dz=0.1, n_layers=3, x0=0, y0=0, nx=10, ny=10, pixel=0.1, slab=3)


def _check_bins(lat, cfg, first_layer, n_slab_layers, tiles_to_check=12, seed=0):
    off, ids = lat.slab_bins(z0=cfg["z0"], dz=cfg["dz"], first_layer=first_layer,
                             n_slab_layers=n_slab_layers, x0=cfg["x0"], y0=cfg["y0"],
                             nx=cfg["nx"], ny=cfg["ny"], pixel=cfg["pixel"])
    roff, rids = binning.bin_lists_fp32(cfg["nodes"], cfg["edges"], lat.R, z0=cfg["z0"],
                                        dz=cfg["dz"], first_layer=first_layer,
                                        n_slab_layers=n_slab_layers, x0=cfg["x0"], y0=cfg["y0"],
                                        nx=cfg["nx"], ny=cfg["ny"], pixel=cfg["pixel"])
    assert np.array_equal(off, roff)
    assert np.array_equal(ids, rids)
    # every FP64 contributor of a tile is in its list
    ntx = -(-cfg["nx"] // 16)
    r = np.random.default_rng(seed)
    n_tiles = len(off) - 1
    for t in r.choice(n_tiles, min(tiles_to_check, n_tiles), replace=False):
        tx, ty = t % ntx, t // ntx
        ii = np.arange(tx * 16, min(tx * 16 + 16, cfg["nx"]))
        jj = np.arange(ty * 16, min(ty * 16 + 16, cfg["ny"]))
        ks = np.arange(first_layer, first_layer + n_slab_layers)
        K, J, I = np.meshgrid(ks, jj, ii, indexing="ij")
        pts = np.stack([cfg["x0"] + (I + 0.5) * cfg["pixel"], cfg["y0"] + (J + 0.5) * cfg["pixel"],
                        cfg["z0"] + K * cfg["dz"]], -1).reshape(-1, 3)
        contrib = binning.contributors_fp64(cfg["nodes"], cfg["edges"], lat.R, pts)
        assert contrib <= set(ids[off[t]:off[t + 1]].tolist())


def test_bins_bit_exact_c1(c1):
    cfg, lat = c1
    for first, n in ((0, 8), (17, 4), (49, 1)):
        _check_bins(lat, cfg, first, n)


def test_bins_bit_exact_c3_small():
    cfg = synth.config(3, small=True)
    cs = _cslice()
    lat = cs.Lattice(cfg["nodes"], cfg["edges"], cfg["radius"], R=cfg["R"])
    _check_bins(lat, cfg, 0, 4, tiles_to_check=6)


def test_deterministic_repeat(c1):
    cfg, lat = c1
    s1, c_1 = gpu_slice(lat, cfg, n_layers=10)
    s2, c_2 = gpu_slice(lat, cfg, n_layers=10)
    assert np.array_equal(s1, s2)
    assert np.array_equal(c_1.xy, c_2.xy) and np.array_equal(c_1.edge_id, c_2.edge_id)


def test_device_contours_match_host(c1):
    cfg, lat = c1
    host = lat.slice(z0=cfg["z0"], dz=cfg["dz"], n_layers=12, x0=0, y0=0, nx=200, ny=200,
                     pixel=0.1, edge_ids=True, chunk_layers=4, slab=4)
    dev = lat.slice(z0=cfg["z0"], dz=cfg["dz"], n_layers=12, x0=0, y0=0, nx=200, ny=200,
                    pixel=0.1, edge_ids=True, chunk_layers=4, slab=4, on_device=True)
    h2 = dev.to_host()
    for a, b in zip((host.layer_loop_off, host.loop_vert_off, host.xy, host.edge_id),
                    (h2.layer_loop_off, h2.loop_vert_off, h2.xy, h2.edge_id)):
        assert np.array_equal(a, b)


def test_device_contours_assembled_in_place(c1):
    """Device contours are written chunk by chunk into arrays that grow in
    place: the same as the host result with chunks that have crossings and
    chunks that have none (layers below the lattice), with and without edge
    ids; and their memory comes back when they are freed."""
    cfg, lat = c1
    z0 = cfg["z0"] - 6 * cfg["dz"]          # the first 6 layers lie below the lattice
    kw = dict(z0=z0, dz=cfg["dz"], n_layers=14, x0=0, y0=0, nx=200, ny=200, pixel=0.1,
              chunk_layers=2, slab=2)
    for eid in (True, False):
        host = lat.slice(edge_ids=eid, **kw)
        dev = lat.slice(edge_ids=eid, on_device=True, **kw)
        got = dev.to_host()
        dev.free()
        assert host.layer_loop_off[4] == 0 and host.layer_loop_off[-1] > 0
        assert np.array_equal(got.layer_loop_off, host.layer_loop_off)
        assert np.array_equal(got.loop_vert_off, host.loop_vert_off)
        assert np.array_equal(got.xy, host.xy)
        assert (got.edge_id is None) == (not eid)
        if eid:
            assert np.array_equal(got.edge_id, host.edge_id)
    lat.slice(edge_ids=True, on_device=True, **kw).free()
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for _ in range(5):
        lat.slice(edge_ids=True, on_device=True, **kw).free()
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] >= free0 - (64 << 20)


def test_host_results_streamed_into_cached_blocks(c1):
    """Host results reuse page-locked blocks: a later call copies each chunk's
    vertices into the largest cached block while it computes the next chunks
    (or, when that block is too small, copies everything at the end). Every
    path gives the device result exactly."""
    cfg, lat = c1
    kw = dict(z0=cfg["z0"], dz=cfg["dz"], x0=0, y0=0, nx=200, ny=200, pixel=0.1,
              edge_ids=True, chunk_layers=4, slab=4)
    ref = lat.slice(n_layers=12, on_device=True, **kw).to_host()

    def same(h):
        for a, b in zip((h.layer_loop_off, h.loop_vert_off, h.xy, h.edge_id),
                        (ref.layer_loop_off, ref.loop_vert_off, ref.xy, ref.edge_id)):
            assert np.array_equal(a, b)

    small = lat.slice(n_layers=2, **kw)   # leaves a small block in the cache
    del small
    same(lat.slice(n_layers=12, **kw))   # block too small: copied at the end
    for _ in range(2):                    # now a block of the right size is cached
        same(lat.slice(n_layers=12, **kw))
    kw_noeid = dict(kw, edge_ids=False)
    h = lat.slice(n_layers=12, **kw_noeid)
    assert h.edge_id is None and np.array_equal(h.xy, ref.xy)


@pytest.mark.parametrize("nx,contours,chunk", [(200, False, 0), (70, True, 2)])
def test_mask_out_is_the_thresholded_field(c1, nx, contours, chunk):
    """The bit-packed binary image (Sec. 4, the DLP mask) is exactly Sigma >= C
    of the returned field, bits past nx are 0, and it matches the oracle's
    classification away from the iso-value."""
    cfg, lat = c1
    n, ny = 6, 90
    wpr = (nx + 31) // 32
    sig = torch.empty((n, ny, nx), dtype=torch.float32, device="cuda")
    mk = torch.full((n, ny, wpr), -1, dtype=torch.int32, device="cuda")
    lat.slice(z0=cfg["z0"], dz=cfg["dz"], n_layers=n, x0=cfg["x0"] + 3.0, y0=cfg["y0"] + 1.0,
              nx=nx, ny=ny, pixel=cfg["pixel"], sigma_out=sig, mask_out=mk, contours=contours,
              slab=2, chunk_layers=chunk)
    torch.cuda.synchronize()
    words = mk.cpu().numpy().view(np.uint32)
    bits = np.unpackbits(words.view(np.uint8), bitorder="little").reshape(n, ny, wpr * 32)
    s = sig.cpu().numpy()
    assert np.array_equal(bits[:, :, :nx].astype(bool), s >= cfg["C"])
    assert not bits[:, :, nx:].any()
    ref = oracle_slice(cfg, n_layers=n, nx=nx, ny=ny, x0=cfg["x0"] + 3.0, y0=cfg["y0"] + 1.0)
    far = np.abs(ref - cfg["C"]) >= 1e-5 * cfg["C"]
    assert np.array_equal(bits[:, :, :nx].astype(bool)[far], (ref >= cfg["C"])[far])


def test_mask_only_slice_gives_the_same_image(c1):
    """Without contours and without sigma_out no Sigma plane is written; the
    binary image is the one of the slice that also returns Sigma."""
    cfg, lat = c1
    n, nx, ny = 10, 200, 120
    wpr = (nx + 31) // 32
    kw = dict(z0=cfg["z0"], dz=cfg["dz"], n_layers=n, x0=cfg["x0"], y0=cfg["y0"], nx=nx, ny=ny,
              pixel=cfg["pixel"], contours=False)
    sig = torch.empty((n, ny, nx), dtype=torch.float32, device="cuda")
    mk1 = torch.full((n, ny, wpr), -1, dtype=torch.int32, device="cuda")
    mk2 = torch.full((n, ny, wpr), -1, dtype=torch.int32, device="cuda")
    lat.slice(**kw, sigma_out=sig, mask_out=mk1)
    lat.slice(**kw, mask_out=mk2)
    torch.cuda.synchronize()
    assert torch.equal(mk1, mk2) and int(mk1.count_nonzero()) > 0


def test_isolated_strut_circle_on_gpu():
    """The cross-section of an isolated long strut is the circle of its radius."""
    cs = _cslice()
    rho = 0.5
    lat = cs.Lattice(np.array([[0, 0, -10], [0, 0, 10]], np.float32), np.array([[0, 1]]),
                     np.array([rho], np.float32), R=0.75)
    cont = lat.slice(z0=0.0, dz=1.0, n_layers=1, x0=-1, y0=-1, nx=100, ny=100, pixel=0.02)
    loops = cont.layer(0)
    assert len(loops) == 1
    xy = loops[0][1].astype(np.float64)
    assert np.max(np.abs(np.hypot(xy[:, 0], xy[:, 1]) - rho)) < 0.01 * 0.02
    area = 0.5 * np.sum(xy[:, 0] * np.roll(xy[:, 1], -1) - np.roll(xy[:, 0], -1) * xy[:, 1])
    assert area == pytest.approx(math.pi * rho * rho, rel=2e-3)


def test_bounded_wait_reports_timeout_and_device_stays_usable(c1):
    """The field kernel's mbarrier wait, on a barrier that nothing arms, gives
    up after its poll limit and reports CSL_ERR_TIMEOUT; the context is intact
    and the next slice is unchanged."""
    from paper_2101_05031_gb300 import _lib
    cfg, lat = c1
    before, _ = gpu_slice(lat, cfg, n_layers=3)
    lib = _lib.load()
    for polls in (1, 1000):
        assert lib.csl_debug_wait_timeout(polls, None) == 4
        assert b"gave up" in lib.csl_last_error()
    after, _ = gpu_slice(lat, cfg, n_layers=3)
    assert np.array_equal(before, after)


def test_workspace_budget_bounds_memory_and_keeps_results():
    """A device-memory budget: one chunk in flight, a first chunk of two slabs
    measures the workspace per layer, the others are sized to fit. Contours
    identical to the unbounded call; the workspace peak within the budget; a
    budget that one slab cannot meet is refused."""
    import paper_2101_05031_gb300 as cs
    cfg = synth.config(2, small=True)
    lat = cs.Lattice(cfg["nodes"], cfg["edges"], cfg["radius"], R=cfg["R"])
    kw = dict(z0=cfg["z0"], dz=0.05, n_layers=40, x0=cfg["x0"], y0=cfg["y0"], nx=cfg["nx"],
              ny=cfg["ny"], pixel=cfg["pixel"], edge_ids=True, slab=2)
    ref = lat.slice(**kw)
    full = cs.last_stats()
    assert full.chunks == 1
    budget = full.device_bytes_peak // 3
    got = lat.slice(**kw, workspace_budget=budget)
    st = cs.last_stats()
    assert st.chunks >= 3
    assert 0 < st.device_bytes_peak <= budget
    for a, b in ((ref.layer_loop_off, got.layer_loop_off), (ref.loop_vert_off, got.loop_vert_off),
                 (ref.edge_id, got.edge_id)):
        assert np.array_equal(a, b)
    assert np.array_equal(ref.xy.view(np.uint32), got.xy.view(np.uint32))
    with pytest.raises(cs.CslError, match="CAPACITY"):
        lat.slice(**kw, workspace_budget=4096)
    with pytest.raises(cs.CslError, match="INVALID_ARG"):
        lat.slice(**kw, workspace_budget=budget, on_device=True)
