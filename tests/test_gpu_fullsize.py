"""Parity at the full configuration sizes, in the launch configuration the
benchmark times (default tile, slab of 8 layers, chunks of whole slabs).

The GPU slices a chunk-aligned range of layers of the full workload; the oracle
evaluates windows of 64 x 64 pixels of some of those layers, given the edges
whose swept sphere can reach the window (every other edge contributes 0 by
Eq. 8, so the window field is the same). Compared: the field on every window
pixel, and every contour loop that lies inside a window (its cells do not touch
the window's border ring, where the window's own padding differs from the
full grid)."""
import numpy as np
import pytest

import oracle
import synth
from tests import helpers

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

WIN = 64


def _edges_near(cfg, x0, y0, w, z_lo, z_hi):
    R = cfg["R"]
    nodes, edges = cfg["nodes"], cfg["edges"]
    a = nodes[edges[:, 0]].astype(np.float64)
    b = nodes[edges[:, 1]].astype(np.float64)
    lo, hi = np.minimum(a, b), np.maximum(a, b)
    keep = ((lo[:, 2] - R <= z_hi) & (hi[:, 2] + R >= z_lo) & (hi[:, 0] + R >= x0)
            & (lo[:, 0] - R <= x0 + w) & (hi[:, 1] + R >= y0) & (lo[:, 1] - R <= y0 + w))
    sel = np.nonzero(keep)[0]
    used = np.unique(edges[sel])
    remap = np.full(nodes.shape[0], -1, np.int64)
    remap[used] = np.arange(used.size)
    return nodes[used], remap[edges[sel]].astype(np.int32), cfg["radius"][sel], sel


def _check_windows(cfg, lat, first, n, n_windows, seed, win=WIN, at=()):
    """n_windows random windows, plus one at each (layer, i0, j0) of `at`."""
    nx, ny, px = cfg["nx"], cfg["ny"], cfg["pixel"]
    sig = torch.empty((n, ny, nx), dtype=torch.float32, device="cuda")
    z0 = cfg["z0"] + first * cfg["dz"]
    cont = lat.slice(z0=z0, dz=cfg["dz"], n_layers=n, x0=cfg["x0"], y0=cfg["y0"], nx=nx, ny=ny,
                     pixel=px, sigma_out=sig, edge_ids=True)
    torch.cuda.synchronize()
    r = np.random.default_rng(seed)
    W = nx + 2
    matched = 0
    places = [(int(r.integers(0, n)), int(r.integers(0, nx - win)), int(r.integers(0, ny - win)))
              for _ in range(n_windows)] + list(at)
    for k, i0, j0 in places:
        wx0, wy0 = cfg["x0"] + i0 * px, cfg["y0"] + j0 * px
        z = z0 + k * cfg["dz"]
        sn, se, sr, _ = _edges_near(cfg, wx0, wy0, win * px, z, z)
        ref = oracle.slice_sigma(sn, se, sr, R=cfg["R"], C=cfg["C"], z0=z, dz=1.0, n_layers=1,
                                 x0=wx0, y0=wy0, nx=win, ny=win, pixel=px)[0]
        got = sig[k, j0:j0 + win, i0:i0 + win].cpu().numpy()
        helpers.assert_field(got, ref, cfg["C"])
        # loops inside the window
        off, eid, xy = oracle.marching_squares(ref, x0=wx0, y0=wy0, pixel=px, C=cfg["C"])
        band = helpers.band_cells(ref, cfg["C"])
        gpu = {int(e[0]): (e, p) for e, p in cont.layer(k)}
        for li in range(len(off) - 1):
            le, lxy = eid[off[li]:off[li + 1]], xy[off[li]:off[li + 1]]
            s = le // 2
            I, J = s % (win + 2), s // (win + 2)
            if (I <= 1).any() or (J <= 1).any() or (I >= win).any() or (J >= win).any():
                continue   # touches the window's border cells
            cells = helpers._edge_cells(le, win)
            if band[cells[:, 1], cells[:, 0]].any():
                continue
            glob = 2 * ((J + j0) * W + (I + i0)) + (le % 2)
            assert int(glob[0]) in gpu, "loop missing on the GPU"
            ge, gxy = gpu[int(glob[0])]
            assert np.array_equal(ge, glob)
            d = np.max(np.hypot(gxy[:, 0] - lxy[:, 0], gxy[:, 1] - lxy[:, 1])) / px
            assert d <= helpers.VERTEX_TOL_PX
            matched += 1
    return matched


@pytest.fixture(scope="module")
def graded_100m():
    import paper_2101_05031_gb300 as cs
    cfg = synth.config(3)
    lat = cs.Lattice(cfg["nodes"], cfg["edges"], cfg["radius"], R=cfg["R"], C=cfg["C"])
    yield cfg, lat
    lat.close()


def _dense_band_window(cfg, win=WIN):
    """(i0, j0) of a window centred where the graded density rho(x) = 0.1 +
    0.3 (0.5 + 0.5 sin(2 pi x / 50) cos(2 pi y / 50)) peaks (x = 62.5, y = 100 mm)."""
    px = cfg["pixel"]
    return int((62.5 - cfg["x0"]) / px) - win // 2, int((100.0 - cfg["y0"]) / px) - win // 2


def test_graded_100M_windows(graded_100m):
    cfg, lat = graded_100m
    matched = _check_windows(cfg, lat, first=496, n=16, n_windows=6, seed=31)
    assert matched > 20


def test_graded_100M_lowest_and_highest_layers_and_the_dense_band(graded_100m):
    """The first and last 16 of the 1000 layers (where the lattice starts and
    ends), with random windows and one in the densest band of rho(x)."""
    cfg, lat = graded_100m
    i0, j0 = _dense_band_window(cfg)
    m = 0
    for first, seed in ((0, 35), (cfg["n_layers"] - 16, 36)):
        m += _check_windows(cfg, lat, first=first, n=16, n_windows=3, seed=seed,
                            at=[(3, i0, j0), (12, i0, j0)])
    assert m > 10


def test_graded_100M_fused_pass_equals_the_default(graded_100m):
    """The fused field and contour pass on 16 full layers of the 100M-strut
    workload: the same contours, bit for bit, as the default path."""
    cfg, lat = graded_100m
    kw = dict(z0=cfg["z0"] + 496 * cfg["dz"], dz=cfg["dz"], n_layers=16, x0=cfg["x0"],
              y0=cfg["y0"], nx=cfg["nx"], ny=cfg["ny"], pixel=cfg["pixel"], edge_ids=True,
              on_device=True)
    a = lat.slice(**kw, fused=True).to_host()
    b = lat.slice(**kw).to_host()
    assert a.xy.shape[0] > 1_000_000
    for x, y in ((a.layer_loop_off, b.layer_loop_off), (a.loop_vert_off, b.loop_vert_off),
                 (a.edge_id, b.edge_id)):
        assert np.array_equal(x, y)
    assert np.array_equal(a.xy.view(np.uint32), b.xy.view(np.uint32))


def test_freudenthal_430k_windows():
    import paper_2101_05031_gb300 as cs
    cfg = synth.config(2)
    lat = cs.Lattice(cfg["nodes"], cfg["edges"], cfg["radius"], R=cfg["R"], C=cfg["C"])
    # the holes of this dense lattice are ~50 px across: wider windows
    matched = _check_windows(cfg, lat, first=64, n=64, n_windows=4, seed=32, win=200)
    assert matched > 5


def test_volume_fraction_1M_sampled_cells():
    """Forward on sampled cells of the 64^3 grid, and the adjoint of a loss
    that weights only those cells."""
    import paper_2101_05031_gb300 as cs
    from paper_2101_05031_gb300 import volume_fraction, volume_fraction_backward
    cfg = synth.config(5)
    lat = cs.Lattice(cfg["nodes"], cfg["edges"], cfg["radius"], R=cfg["R"], C=cfg["C"])
    cells = cfg["cells"]
    d = cells["dims"]
    vf = volume_fraction(lat, cells).cpu().numpy().ravel()
    r = np.random.default_rng(33)
    # cells clustered in one corner block so that the oracle's edge subset stays small
    cx0, cy0, cz0 = (int(v) for v in r.integers(8, 48, 3))
    block = [((z * d[1] + y) * d[0] + x) for z in range(cz0, cz0 + 3) for y in range(cy0, cy0 + 3)
             for x in range(cx0, cx0 + 3)]
    ids = np.array(sorted(block), np.int64)
    o, h, R = cells["origin"], cells["h"], cfg["R"]
    bx0, by0, bz0 = o[0] + cx0 * h, o[1] + cy0 * h, o[2] + cz0 * h
    sn, se, sr, sel = _edges_near(cfg, bx0, by0, 3 * h, bz0, bz0 + 3 * h)
    ref = oracle.volume_fraction(sn, se, sr, cells, R=R, ids=ids)
    assert np.max(np.abs(vf[ids] - ref)) <= 3e-4
    g = np.zeros(vf.size, np.float32)
    g[ids] = r.normal(size=ids.size).astype(np.float32)
    gr, gn = volume_fraction_backward(lat, cells, torch.from_numpy(g.reshape(d[2], d[1], d[0])).cuda())
    gr = gr.cpu().numpy().astype(np.float64)
    ref_r, ref_n = oracle.vf_backward(sn, se, sr, cells, g[ids].astype(np.float64), R=R, ids=ids)
    outside = np.setdiff1d(np.arange(gr.size), sel)
    assert np.all(gr[outside] == 0.0)
    rel = np.linalg.norm(gr[sel] - ref_r) / np.linalg.norm(ref_r)
    assert rel <= 1e-4, rel
    # node gradients of the nodes the subset uses
    used = np.unique(cfg["edges"][sel])
    gn = gn.cpu().numpy().astype(np.float64)[used]
    reln = np.linalg.norm(gn - ref_n) / np.linalg.norm(ref_n)
    assert reln <= 1e-4, reln


def test_batched_64_lattices_windows():
    """The full 64-lattice batch (autotuned graph, as the benchmark runs it):
    sampled windows of four jobs against the oracle, and each job's loops
    inside its windows."""
    import paper_2101_05031_gb300 as cs
    cfg = synth.config(4)
    jobs = []
    for jb in cfg["jobs"]:
        lat = cs.Lattice(jb["nodes"], jb["edges"], jb["radius"], R=jb["R"], C=jb["C"])
        jobs.append((lat, dict(z0=jb["z0"], dz=jb["dz"], n_layers=jb["n_layers"], x0=jb["x0"],
                               y0=jb["y0"], nx=jb["nx"], ny=jb["ny"], pixel=jb["pixel"],
                               edge_ids=True)))
    b = cs.Batch(jobs, autotune=True)
    b.run()
    r = np.random.default_rng(34)
    matched = 0
    sizes = np.array([jb["edges"].shape[0] for jb in cfg["jobs"]])
    # the largest job, the smallest, and two in between
    order = np.argsort(sizes)
    for j in (int(order[-1]), int(order[0]), int(order[len(order) // 2]), int(order[10])):
        jb = cfg["jobs"][j]
        sig = b.sigma(j)
        cont = b.contours(j)
        nx, ny, px = jb["nx"], jb["ny"], jb["pixel"]
        W = nx + 2
        for _ in range(2):
            k = int(r.integers(0, jb["n_layers"]))
            win = min(200, nx - 2, ny - 2)
            i0 = int(r.integers(0, nx - win + 1))
            j0 = int(r.integers(0, ny - win + 1))
            wx0, wy0 = jb["x0"] + i0 * px, jb["y0"] + j0 * px
            z = jb["z0"] + k * jb["dz"]
            sn, se, sr, _ = _edges_near(jb, wx0, wy0, win * px, z, z)
            ref = oracle.slice_sigma(sn, se, sr, R=jb["R"], C=jb["C"], z0=z, dz=1.0, n_layers=1,
                                     x0=wx0, y0=wy0, nx=win, ny=win, pixel=px)[0]
            got = sig[k, j0:j0 + win, i0:i0 + win].cpu().numpy()
            helpers.assert_field(got, ref, jb["C"])
            off, eid, xy = oracle.marching_squares(ref, x0=wx0, y0=wy0, pixel=px, C=jb["C"])
            band = helpers.band_cells(ref, jb["C"])
            gpu = {int(e[0]): (e, p) for e, p in cont.layer(k)}
            for li in range(len(off) - 1):
                le, lxy = eid[off[li]:off[li + 1]], xy[off[li]:off[li + 1]]
                s_ = le // 2
                I, J = s_ % (win + 2), s_ // (win + 2)
                if (I <= 1).any() or (J <= 1).any() or (I >= win).any() or (J >= win).any():
                    continue
                cells = helpers._edge_cells(le, win)
                if band[cells[:, 1], cells[:, 0]].any():
                    continue
                glob = 2 * ((J + j0) * W + (I + i0)) + (le % 2)
                assert int(glob[0]) in gpu, "loop missing on the GPU"
                ge, gxy = gpu[int(glob[0])]
                assert np.array_equal(ge, glob)
                d = np.max(np.hypot(gxy[:, 0] - lxy[:, 0], gxy[:, 1] - lxy[:, 1])) / px
                assert d <= helpers.VERTEX_TOL_PX
                matched += 1
    assert matched >= 8
    b.close()
