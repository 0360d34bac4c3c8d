"""Density matching on the GPU (csl_density_match) against the FP64 oracle:
the subdivision (topology, bit-exact where no decision is a near tie), the
targets, rho*, the bisected ratios (compared through the densities they
reach, since a flat density leaves the ratio ill-conditioned), the voxel
ratios and the per-edge minimum rule."""
import itertools

import numpy as np
import pytest

import synth
from oracle import density as D

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

C, TEMP = 1.0, 0.01


def _run_gpu(cfg, **kw):
    import paper_2101_05031_gb300 as cs
    args = dict(r_min=cfg["r_min"], tet_n=cfg["tet_n"], vox_m=cfg["vox_m"],
                max_depth=cfg["max_depth"], iters=cfg["iters"])
    args.update(kw)
    return cs.density_match(cfg["nodes"], cfg["tets"], cfg["grid"], **args)


@pytest.fixture(scope="module")
def small():
    cfg = synth.density_config(small=True)
    ref = D.density_match(cfg["nodes"], cfg["tets"], cfg["grid"], r_min=cfg["r_min"],
                          tet_n=cfg["tet_n"], vox_m=cfg["vox_m"], max_depth=cfg["max_depth"],
                          iters=cfg["iters"])
    got = _run_gpu(cfg)
    return cfg, ref, got


def _ratio_close(rho, s_gpu, s_ref, tol_s=1e-4, tol_rho=5e-5):
    """Same ratio, or one the density cannot tell apart from it."""
    if abs(float(s_gpu) - float(s_ref)) <= tol_s:
        return True
    return abs(rho(float(s_gpu)) - rho(float(s_ref))) <= tol_rho


def test_subdivision_topology_matches(small):
    cfg, ref, got = small
    margins = np.array([abs(m) for _, m, _ in ref["decisions"]])
    assert margins.min() > 1e-4          # no near tie in this seeded case
    assert got["n_subdivided"] == sum(1 for *_, s in ref["decisions"] if s) > 0
    assert np.array_equal(got["nodes"], ref["nodes"])
    assert np.array_equal(got["edges"], ref["edges"])
    assert np.array_equal(got["tets"], ref["tets"])
    assert np.array_equal(got["depth"], ref["depth"])
    assert len(set(ref["depth"].tolist())) == 3   # all three levels occur


def test_medium_mesh_topology_matches():
    """A 4^3-cube mesh (384 tetrahedra): every input tetrahedron splits at
    level 0 and 32 of the children again at level 1, so edges split at an
    earlier level by a neighbour and faces shared by two splits of one level
    both occur; nodes, edges (creation order), leaves and depths bit-exact."""
    from synth.tets import SEED_BASE, graded_target_grid, kuhn_tet_mesh
    nodes, tets = kuhn_tet_mesh((4, 4, 4), 4.0, 0.1, seed=SEED_BASE + 9)
    grid = graded_target_grid((0.0, 0.0, 0.0), (16.0, 16.0, 16.0), 16.0 / 5.0,
                              scale=(0.03, 0.5), period=16.0)
    cfg = dict(nodes=nodes, tets=tets, grid=grid, r_min=0.1, tet_n=2, vox_m=2, max_depth=2,
               iters=24)
    ref = D.density_match(nodes, tets, grid, r_min=0.1, tet_n=2, vox_m=2, max_depth=2, iters=24)
    margins = np.array([abs(m) for _, m, _ in ref["decisions"]])
    assert margins.min() > 1e-4          # no near tie in this seeded case
    got = _run_gpu(cfg)
    assert got["n_subdivided"] == sum(1 for *_, s in ref["decisions"] if s) == 416
    assert np.array_equal(got["nodes"], ref["nodes"])
    assert np.array_equal(got["edges"], ref["edges"])
    assert np.array_equal(got["tets"], ref["tets"])
    assert np.array_equal(got["depth"], ref["depth"])
    assert np.bincount(got["depth"]).tolist() == [0, 3040, 256]


def test_targets_and_rho_star(small):
    cfg, ref, got = small
    assert np.max(np.abs(got["target"] - ref["target"])) <= 1e-12
    assert np.max(np.abs(got["rho_star"] - ref["rho_star"])) <= 2e-5


def test_tet_ratios_reach_the_same_densities(small):
    cfg, ref, got = small
    A = D.kuhn_coefficients(cfg["tet_n"])
    r0, R = ref["r0"], ref["R"]
    n_interior = 0
    for k, t in enumerate(ref["tets"]):
        rho = D.tet_density_fn(ref["nodes"][t].astype(np.float64), A, r0, R, C, TEMP * C)
        assert _ratio_close(rho, got["tet_ratio"][k], ref["tet_ratio"][k]), k
        n_interior += 0.5 < ref["tet_ratio"][k] < 2.0
    assert n_interior >= 20


def test_edge_ratios_take_the_smallest(small):
    """Step 3 per edge: bounded by the tetrahedra's differences; Step 4: the
    GPU's final ratio is exactly min(step-3 ratio, ratios of the voxels the
    edge meets), with the meets decided by the oracle's FP64 test."""
    cfg, ref, got = small
    lat = ref["lattice"]
    d_tet = np.abs(got["tet_ratio"].astype(np.float64) - ref["tet_ratio"])
    # per edge: the largest ratio difference of the leaves containing it
    seg_index = {e: i for i, e in enumerate(e for e in range(len(lat.edges))
                                            if lat.children[e] is None)}
    bound = np.zeros(len(seg_index))
    leaves = [t for t in range(len(lat.tets)) if lat.leaf[t]]
    for li, t in enumerate(leaves):
        for e in lat.tet_edges[t]:
            for s in lat.leaf_segments(e):
                bound[seg_index[s]] = max(bound[seg_index[s]], d_tet[li])
    assert np.all(np.abs(got["step3_ratio"] - ref["step3_ratio"]) <= bound + 1e-6)
    # the minimum rule, bit-exact on the GPU's own values
    grid = cfg["grid"]
    a = got["nodes"][got["edges"][:, 0]].astype(np.float64)
    b = got["nodes"][got["edges"][:, 1]].astype(np.float64)
    expect = got["step3_ratio"].copy()
    o, h = grid["origin"], grid["h"]
    nx, ny, nz = grid["dims"]
    for k, j, i in itertools.product(range(nz), range(ny), range(nx)):
        lo = (o[0] + h * i, o[1] + h * j, o[2] + h * k)
        hi = (o[0] + h * (i + 1), o[1] + h * (j + 1), o[2] + h * (k + 1))
        meets = np.array([D.seg_meets_box(a[e], b[e], lo, hi) for e in range(len(a))])
        assert np.isnan(got["voxel_ratio"][k, j, i]) == (not meets.any())
        if meets.any():
            expect[meets] = np.minimum(expect[meets], got["voxel_ratio"][k, j, i])
    assert np.array_equal(got["radius"], (np.float32(ref["r0"]) * expect).astype(np.float32))


def test_voxel_ratios_reach_the_same_densities(small):
    cfg, ref, got = small
    grid = cfg["grid"]
    seg_a = ref["nodes"][ref["edges"][:, 0]].astype(np.float64)
    seg_b = ref["nodes"][ref["edges"][:, 1]].astype(np.float64)
    nx, ny, nz = grid["dims"]
    n = 0
    for k, j, i in itertools.product(range(nz), range(ny), range(nx)):
        s_ref = ref["voxel_ratio"][k, j, i]
        if np.isnan(s_ref):
            assert np.isnan(got["voxel_ratio"][k, j, i])
            continue
        rho, _ = D.voxel_density_fn(grid, i, j, k, seg_a, seg_b, ref["step3_ratio"], ref["r0"],
                                    ref["R"], C, TEMP * C, cfg["vox_m"])
        # the GPU's fixed part uses its own step-3 ratios: allow their spread
        assert _ratio_close(rho, got["voxel_ratio"][k, j, i], s_ref, tol_s=2e-3, tol_rho=2e-4)
        n += 1
    assert n >= 10


def test_no_subdivision_and_flat_targets():
    """max_depth = 0 keeps the mesh; a target beyond reach takes the end points."""
    cfg = synth.density_config(small=True)
    grid = dict(cfg["grid"])
    for value, ratio in ((5.0, 2.0), (0.0, 0.5)):
        grid["target"] = np.full_like(cfg["grid"]["target"], value)
        got = _run_gpu(dict(cfg, grid=grid), max_depth=0)
        assert got["n_subdivided"] == 0 and got["tets"].shape == cfg["tets"].shape
        assert np.all(got["tet_ratio"] == ratio)
        assert np.all(got["voxel_ratio"][~np.isnan(got["voxel_ratio"])] == ratio)
        assert np.allclose(got["radius"], 2 * cfg["r_min"] * ratio)


def test_empty_mesh():
    cfg = synth.density_config(small=True)
    got = _run_gpu(dict(cfg, nodes=np.zeros((0, 3), np.float32), tets=np.zeros((0, 4), np.int32)))
    assert got["edges"].shape == (0, 2) and got["tets"].shape == (0, 4)
    assert np.all(np.isnan(got["voxel_ratio"]))


def test_full_workload_sampled_against_the_oracle():
    """The 93,750-tetrahedron workload. A leaf that was never subdivided is a
    tetrahedron of the mesh as given (the subdivision keeps node indices and
    vertex order), so 24 of them get their target, rho* and ratio recomputed
    by the oracle from the synthetic input alone. On every leaf, edge and
    voxel, without the oracle: the stopping rule (rho* >= target unless at the
    depth limit), ratios inside the bisection interval [1/2, 2] (voxels: or
    NaN), and radii between r0 / 2 and r0 times the edge's Step-3 ratio (the
    voxel check only lowers a ratio). Every step on oracle-made inputs is
    compared on the small case above."""
    cfg = synth.density_config()
    got = _run_gpu(cfg)
    assert got["n_subdivided"] > 0 and got["tets"].shape[0] > cfg["tets"].shape[0]
    n0 = cfg["nodes"].shape[0]
    assert np.array_equal(got["nodes"][:n0], cfg["nodes"].astype(np.float32))
    r0 = 2 * cfg["r_min"]
    R = 3 * r0
    A = D.kuhn_coefficients(cfg["tet_n"])
    orig = {tuple(sorted(t)): i for i, t in enumerate(cfg["tets"].tolist())}
    leaves0 = np.nonzero(got["depth"] == 0)[0]
    assert len(leaves0) > 1000
    r = synth.rng(17)
    for k in r.choice(leaves0, 24, replace=False):
        i = orig[tuple(sorted(got["tets"][k].tolist()))]
        assert np.array_equal(got["tets"][k], cfg["tets"][i])
        v = cfg["nodes"][cfg["tets"][i]].astype(np.float64)
        target = D.tet_target(cfg["grid"], v)
        assert abs(target - got["target"][k]) <= 1e-12
        rho = D.tet_density_fn(v, A, r0, R, C, TEMP * C)
        assert abs(rho(2.0) - got["rho_star"][k]) <= 2e-5
        s_ref = D.bisect_ratio(rho, target, cfg["iters"])
        assert _ratio_close(rho, got["tet_ratio"][k], s_ref)
    depth = got["depth"]
    assert depth.min() >= 0 and depth.max() <= cfg["max_depth"]
    inner = depth < cfg["max_depth"]
    assert np.all(got["rho_star"][inner] >= got["target"][inner] - 1e-6)
    for a in (got["tet_ratio"], got["step3_ratio"]):
        assert np.all((a >= 0.5 - 1e-6) & (a <= 2.0 + 1e-6))
    vr = got["voxel_ratio"]
    ok = np.isnan(vr) | ((vr >= 0.5 - 1e-6) & (vr <= 2.0 + 1e-6))
    assert np.all(ok) and np.count_nonzero(~np.isnan(vr)) > 0.5 * vr.size
    rad = got["radius"].astype(np.float64)
    assert np.all(rad >= 0.5 * r0 * (1 - 1e-6))
    assert np.all(rad <= r0 * got["step3_ratio"].astype(np.float64) * (1 + 1e-6))
