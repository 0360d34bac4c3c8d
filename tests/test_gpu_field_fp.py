"""The footprint field kernel (each layer's warp walks every edge's footprint)
against the FP64 oracle, against the block kernel, and on its edge cases:
ragged grids, tiles of 16 and 32 pixels, every slab depth, small staging
chunks, struts along the axes and in the layer planes, zero-length struts."""
import numpy as np
import pytest

import oracle
import synth
from oracle import binning
from tests import helpers

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _cs():
    import paper_2101_05031_gb300 as cs
    return cs


def _slice(lat, cfg, **kw):
    g = dict(z0=cfg["z0"], dz=cfg["dz"], n_layers=cfg["n_layers"], x0=cfg["x0"], y0=cfg["y0"],
             nx=cfg["nx"], ny=cfg["ny"], pixel=cfg["pixel"])
    for k in list(kw):
        if k in g:
            g[k] = kw.pop(k)
    sig = torch.empty((g["n_layers"], g["ny"], g["nx"]), dtype=torch.float32, device="cuda")
    cont = lat.slice(**g, sigma_out=sig, edge_ids=True, **kw)
    torch.cuda.synchronize()
    return sig.cpu().numpy(), cont, g


def _oracle(cfg, g):
    return oracle.slice_sigma(cfg["nodes"], cfg["edges"], cfg["radius"], R=cfg["R"], C=cfg["C"],
                              z0=g["z0"], dz=g["dz"], n_layers=g["n_layers"], x0=g["x0"],
                              y0=g["y0"], nx=g["nx"], ny=g["ny"], pixel=g["pixel"])


def _contours_vs_oracle(cont, ref, cfg, g):
    tot = 0
    for k in range(ref.shape[0]):
        m, _ = helpers.compare_layer_contours(cont.layer(k), ref[k], x0=g["x0"], y0=g["y0"],
                                              pixel=g["pixel"], C=cfg["C"])
        tot += m
    return tot


@pytest.fixture(scope="module")
def c1():
    cfg = synth.config(1)
    return cfg, _cs().Lattice(cfg["nodes"], cfg["edges"], cfg["radius"], R=cfg["R"])


@pytest.fixture(scope="module")
def c3s():
    cfg = synth.config(3, small=True)
    return cfg, _cs().Lattice(cfg["nodes"], cfg["edges"], cfg["radius"], R=cfg["R"])


@pytest.mark.parametrize("tile", [16, 32])
def test_c1_full_parity(c1, tile):
    cfg, lat = c1
    sig, cont, g = _slice(lat, cfg, field_kernel="footprint", tile=tile)
    ref = _oracle(cfg, g)
    helpers.assert_field(sig, ref, cfg["C"])
    assert _contours_vs_oracle(cont, ref, cfg, g) > 0


@pytest.mark.parametrize("tile,slab", [(16, 1), (16, 8), (32, 2), (32, 4), (32, 8)])
def test_graded_small_parity(c3s, tile, slab):
    """The small graded lattice (supports of ~7 px, the kernel's design case)."""
    cfg, lat = c3s
    sig, cont, g = _slice(lat, cfg, field_kernel="footprint", tile=tile, slab=slab)
    ref = _oracle(cfg, g)
    helpers.assert_field(sig, ref, cfg["C"])
    assert _contours_vs_oracle(cont, ref, cfg, g) > 0


def test_freudenthal_small_parity():
    """Supports of ~13 px (0.525 mm at 0.04 mm), wider than a 8 x 4 block."""
    cfg = synth.config(2, small=True)
    lat = _cs().Lattice(cfg["nodes"], cfg["edges"], cfg["radius"], R=cfg["R"])
    sig, cont, g = _slice(lat, cfg, field_kernel="footprint", tile=32, n_layers=4, nx=250,
                          ny=170)
    ref = _oracle(cfg, g)
    helpers.assert_field(sig, ref, cfg["C"])
    assert _contours_vs_oracle(cont, ref, cfg, g) > 0


@pytest.mark.parametrize("slab", [1, 2, 4, 8])
def test_agrees_with_the_block_kernel(c1, c3s, slab):
    """The same terms summed in the same list order, the pixel coordinates
    rounded differently: the two kernels agree to a few FP32 ulps (each is within
    1e-5 of the oracle; half of that bounds their difference)."""
    for cfg, lat in (c1, c3s):
        nl = 11 if cfg is c1[0] else 4
        for tile in (16, 32):
            a, _, _ = _slice(lat, cfg, field_kernel="footprint", tile=tile, slab=slab, n_layers=nl)
            b, _, _ = _slice(lat, cfg, field_kernel="block", tile=16, slab=slab, n_layers=nl)
            assert helpers.field_error(a, b, cfg["C"]) <= 5e-6


def test_ragged_grid_odd_origin_and_small_staging(c1):
    """A grid that is no multiple of the tile, an origin off the pixel lattice,
    and 32 records per staged copy (tiles with several copies)."""
    cfg, lat = c1
    for tile, stage in ((32, 32), (16, 64), (32, 1024)):
        sig, cont, g = _slice(lat, cfg, field_kernel="footprint", tile=tile,
                              stage_records=stage, n_layers=5, z0=3.3, nx=157, ny=93,
                              x0=1.234, y0=-0.77)
        ref = _oracle(cfg, g)
        helpers.assert_field(sig, ref, cfg["C"])
        _contours_vs_oracle(cont, ref, cfg, g)


def test_deterministic_repeat(c3s):
    cfg, lat = c3s
    a, ca, _ = _slice(lat, cfg, field_kernel="footprint")
    b, cb, _ = _slice(lat, cfg, field_kernel="footprint")
    assert np.array_equal(a.view(np.uint32), b.view(np.uint32))
    assert np.array_equal(ca.edge_id, cb.edge_id)


def _axis_struts():
    """Struts along x, y, z, the diagonals of the planes, slanted, lying in a
    layer plane, and two of zero length."""
    nodes = np.array([
        [1.0, 1.0, 1.0], [3.0, 1.0, 1.0],       # along x, in the plane z = 1.0
        [1.0, 2.0, 0.9], [1.0, 4.0, 0.9],       # along y, 0.1 below the plane
        [2.0, 2.5, 0.0], [2.0, 2.5, 2.0],       # along z
        [3.0, 3.0, 1.05], [4.2, 4.2, 1.05],     # diagonal, horizontal
        [0.5, 3.5, 0.2], [1.5, 4.8, 1.9],       # slanted
        [3.5, 0.5, 0.4], [4.5, 1.3, 1.6],       # slanted the other way
        [2.8, 4.4, 1.0], [2.8, 4.4, 1.0],       # zero length, in the plane
        [4.4, 2.2, 1.2], [4.4, 2.2, 1.2],       # zero length, off the plane
    ], np.float32)
    edges = np.arange(16, dtype=np.int32).reshape(8, 2)
    radius = np.full(8, 0.12, np.float32)
    return nodes, edges, radius


@pytest.mark.parametrize("tile", [16, 32])
def test_struts_along_the_axes_and_in_the_planes(tile):
    nodes, edges, radius = _axis_struts()
    cfg = dict(nodes=nodes, edges=edges, radius=radius, R=0.2, C=1.0, z0=0.6, dz=0.2,
               n_layers=6, x0=0.0, y0=0.0, nx=110, ny=105, pixel=0.05)
    lat = _cs().Lattice(nodes, edges, radius, R=0.2)
    sig, cont, g = _slice(lat, cfg, field_kernel="footprint", tile=tile)
    ref = _oracle(cfg, g)
    helpers.assert_field(sig, ref, 1.0)
    assert np.max(ref) > 1.0
    _contours_vs_oracle(cont, ref, cfg, g)


def test_bins_bit_exact_on_32px_tiles(c1, c3s):
    """The binner on 32-pixel tiles against its independent FP32 restatement,
    and every FP64 contributor of a sampled tile in its list."""
    for cfg, lat in (c1, c3s):
        for first, n in ((0, 8), (1, 4)):
            off, ids = lat.slab_bins(z0=cfg["z0"], dz=cfg["dz"], first_layer=first,
                                     n_slab_layers=n, x0=cfg["x0"], y0=cfg["y0"], nx=cfg["nx"],
                                     ny=cfg["ny"], pixel=cfg["pixel"], tile=32)
            roff, rids = binning.bin_lists_fp32(cfg["nodes"], cfg["edges"], lat.R, z0=cfg["z0"],
                                                dz=cfg["dz"], first_layer=first,
                                                n_slab_layers=n, x0=cfg["x0"], y0=cfg["y0"],
                                                nx=cfg["nx"], ny=cfg["ny"], pixel=cfg["pixel"],
                                                tile=32)
            assert np.array_equal(off, roff) and np.array_equal(ids, rids)
            ntx = -(-cfg["nx"] // 32)
            for t in np.random.default_rng(first).choice(len(off) - 1, 4, replace=False):
                tx, ty = t % ntx, t // ntx
                ii = np.arange(tx * 32, min(tx * 32 + 32, cfg["nx"]))
                jj = np.arange(ty * 32, min(ty * 32 + 32, cfg["ny"]))
                K, J, I = np.meshgrid(np.arange(first, first + n), jj, ii, indexing="ij")
                pts = np.stack([cfg["x0"] + (I + 0.5) * cfg["pixel"],
                                cfg["y0"] + (J + 0.5) * cfg["pixel"],
                                cfg["z0"] + K * cfg["dz"]], -1).reshape(-1, 3)
                assert binning.contributors_fp64(cfg["nodes"], cfg["edges"], lat.R, pts) <= \
                    set(ids[off[t]:off[t + 1]].tolist())


def test_mask_output_matches_the_field(c3s):
    cfg, lat = c3s
    g = dict(z0=cfg["z0"], dz=cfg["dz"], n_layers=cfg["n_layers"], x0=cfg["x0"], y0=cfg["y0"],
             nx=cfg["nx"], ny=cfg["ny"], pixel=cfg["pixel"])
    wpr = (g["nx"] + 31) // 32
    sig = torch.empty((g["n_layers"], g["ny"], g["nx"]), dtype=torch.float32, device="cuda")
    mask = torch.zeros((g["n_layers"], g["ny"], wpr), dtype=torch.int32, device="cuda")
    lat.slice(**g, sigma_out=sig, mask_out=mask, contours=False, field_kernel="footprint")
    torch.cuda.synchronize()
    s = sig.cpu().numpy()
    m = mask.cpu().numpy().view(np.uint32)
    bits = (m[..., None] >> np.arange(32, dtype=np.uint32)) & 1
    inside = bits.reshape(g["n_layers"], g["ny"], wpr * 32)[..., :g["nx"]].astype(bool)
    assert np.array_equal(inside, s >= np.float32(cfg["C"]))


def test_bad_kernel_options_are_refused(c1):
    cfg, lat = c1
    cs = _cs()
    base = dict(z0=1.0, dz=0.4, n_layers=2, x0=0, y0=0, nx=20, ny=20, pixel=0.1, contours=False)
    for bad in (dict(tile=32, field_kernel="block"), dict(tile=24),
                dict(field_kernel="footprint", stage_records=48),
                dict(field_kernel="footprint", stage_records=2048)):
        with pytest.raises(cs.CslError, match="INVALID_ARG"):
            lat.slice(**base, **bad)


# ---- the fused field and contour pass: no Sigma plane, the same contours ----

def _same_contours(a, b):
    assert np.array_equal(a.layer_loop_off, b.layer_loop_off)
    assert np.array_equal(a.loop_vert_off, b.loop_vert_off)
    assert np.array_equal(a.edge_id, b.edge_id)
    assert np.array_equal(a.xy.view(np.uint32), b.xy.view(np.uint32))


@pytest.mark.parametrize("tile,slab", [(32, 8), (32, 2), (16, 4), (16, 1)])
def test_fused_pass_gives_the_unfused_contours(c1, c3s, tile, slab):
    """The fused pass's vertices are the same float expressions of the same
    Sigma values, read in shared memory instead of a plane: identical contours,
    ragged grids and odd origins included."""
    for cfg, lat, kw in ((c1[0], c1[1], {}), (c3s[0], c3s[1], {}),
                         (c1[0], c1[1], dict(nx=157, ny=93, x0=1.234, y0=-0.77, n_layers=7))):
        _, a, _ = _slice(lat, cfg, field_kernel="footprint", tile=tile, slab=slab, fused=True,
                         **kw)
        _, b, _ = _slice(lat, cfg, field_kernel="footprint", tile=tile, slab=slab, **kw)
        assert a.xy.shape[0] > 0
        _same_contours(a, b)


def test_fused_pass_against_the_oracle(c3s):
    cfg, lat = c3s
    g = dict(z0=cfg["z0"], dz=cfg["dz"], n_layers=cfg["n_layers"], x0=cfg["x0"], y0=cfg["y0"],
             nx=cfg["nx"], ny=cfg["ny"], pixel=cfg["pixel"])
    cont = lat.slice(**g, edge_ids=True, field_kernel="footprint", fused=True)   # no Sigma plane
    assert _contours_vs_oracle(cont, _oracle(cfg, g), cfg, g) > 0


def test_fused_bins_bit_exact_with_the_halo():
    """The fused pass bins each tile with its next column and row: the binner
    against its FP32 restatement with the one-pixel halo (on the jittered
    Freudenthal block; the graded lattice's dyadic node grid happens to put no
    box start within a pixel above a tile boundary)."""
    cfg = synth.config(2, small=True)
    lat = _cs().Lattice(cfg["nodes"], cfg["edges"], cfg["radius"], R=cfg["R"])
    for tile in (16, 32):
        off, ids = lat.slab_bins(z0=cfg["z0"], dz=cfg["dz"], first_layer=0, n_slab_layers=4,
                                 x0=cfg["x0"], y0=cfg["y0"], nx=cfg["nx"], ny=cfg["ny"],
                                 pixel=cfg["pixel"], tile=tile, halo=True)
        roff, rids = binning.bin_lists_fp32(cfg["nodes"], cfg["edges"], lat.R, z0=cfg["z0"],
                                            dz=cfg["dz"], first_layer=0, n_slab_layers=4,
                                            x0=cfg["x0"], y0=cfg["y0"], nx=cfg["nx"],
                                            ny=cfg["ny"], pixel=cfg["pixel"], tile=tile,
                                            halo=True)
        assert np.array_equal(off, roff) and np.array_equal(ids, rids)
        plain = lat.slab_bins(z0=cfg["z0"], dz=cfg["dz"], first_layer=0, n_slab_layers=4,
                              x0=cfg["x0"], y0=cfg["y0"], nx=cfg["nx"], ny=cfg["ny"],
                              pixel=cfg["pixel"], tile=tile)[1]
        assert ids.size > plain.size   # the halo adds entries


def test_fused_vertex_lists_grow_when_the_first_guess_is_short():
    """A field of thin vertical struts every 3 pixels has about one crossing
    per pixel, four times the first guess of the vertex lists' size: the chunk
    is run again with room for them, and the contours equal the unfused ones."""
    n, sp, px = 400, 0.15, 0.05
    xs = (np.arange(n) + 0.5) * sp
    X, Y = np.meshgrid(xs, xs)
    top = np.stack([X.ravel(), Y.ravel(), np.full(n * n, 1.0)], 1)
    bot = np.stack([X.ravel(), Y.ravel(), np.zeros(n * n)], 1)
    nodes = np.concatenate([bot, top]).astype(np.float32)
    edges = np.stack([np.arange(n * n), np.arange(n * n) + n * n], 1).astype(np.int32)
    radius = np.full(n * n, 0.035, np.float32)
    lat = _cs().Lattice(nodes, edges, radius, R=0.05)
    g = dict(z0=0.5, dz=0.1, n_layers=2, x0=0.0, y0=0.0, nx=1200, ny=1200, pixel=px)
    a = lat.slice(**g, edge_ids=True, field_kernel="footprint", fused=True)
    b = lat.slice(**g, edge_ids=True, field_kernel="footprint")
    assert a.xy.shape[0] > 2 * 1200 * 1200 // 4   # more than the first guess
    _same_contours(a, b)
