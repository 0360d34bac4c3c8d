"""Batched slicing (one CUDA graph over many jobs) against per-job slicing and
the FP64 oracle; replay stability, autotuning and the size-change check."""
import numpy as np
import pytest

import oracle
import synth
from tests import helpers

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _jobs(n_layers=12):
    """The small batched set (8 lattices, 1k-20k struts, 0.1 mm pixels) with
    12 layers each, plus two slab ranges of the first lattice."""
    import paper_2101_05031_gb300 as cs
    cfg = synth.config(4, small=True)
    jobs, specs = [], []
    for jb in cfg["jobs"]:
        lat = cs.Lattice(jb["nodes"], jb["edges"], jb["radius"], R=jb["R"], C=jb["C"])
        dz = jb["dz"] * jb["n_layers"] / n_layers
        d = dict(z0=jb["z0"] - jb["dz"] / 2 + dz / 2, dz=dz, n_layers=n_layers, x0=jb["x0"],
                 y0=jb["y0"], nx=jb["nx"], ny=jb["ny"], pixel=jb["pixel"], edge_ids=True)
        jobs.append((lat, d))
        specs.append(jb)
    lat0, d0 = jobs[0]
    for first, n in ((0, 5), (5, 7)):   # slab ranges of one lattice, ragged slabs
        d = dict(d0, z0=d0["z0"] + first * d0["dz"], n_layers=n)
        jobs.append((lat0, d))
        specs.append(specs[0])
    return jobs, specs


def _per_job(lat, d, slab, kernel="block", tile=16, stage=0):
    """Per-job slicing with the batch's field kernel and tile (default: the
    block kernel on 16-pixel tiles), so that both sum the same terms in the
    same order."""
    sig = torch.empty((d["n_layers"], d["ny"], d["nx"]), dtype=torch.float32, device="cuda")
    cont = lat.slice(z0=d["z0"], dz=d["dz"], n_layers=d["n_layers"], x0=d["x0"], y0=d["y0"],
                     nx=d["nx"], ny=d["ny"], pixel=d["pixel"], sigma_out=sig, edge_ids=True,
                     slab=slab, field_kernel=kernel, tile=tile, stage_records=stage)
    torch.cuda.synchronize()
    return sig, cont


def _same_contours(a, b):
    assert np.array_equal(a.layer_loop_off, b.layer_loop_off)
    assert np.array_equal(a.loop_vert_off, b.loop_vert_off)
    assert np.array_equal(a.xy, b.xy)
    assert np.array_equal(a.edge_id, b.edge_id)


@pytest.fixture(scope="module")
def job_set():
    return _jobs()


def test_batch_equals_per_job_slicing(job_set):
    """Same kernels, same terms in the same order: bit-identical Sigma and
    contours for every job, against per-job slicing at the same slab depth
    (the slab's first plane is the origin of the FP32 z coordinates)."""
    import paper_2101_05031_gb300 as cs
    jobs, _ = job_set
    for slab, ctas in ((8, 4), (2, 3)):
        ref = [_per_job(lat, d, slab) for lat, d in jobs]
        b = cs.Batch(jobs, slab=slab, ctas_per_sm=ctas, branches=3)
        b.run()
        info = b.info()
        assert info.slab == slab and info.ctas_per_sm == ctas and info.n_jobs == len(jobs)
        assert info.pixel_evals == sum(d["n_layers"] * d["nx"] * d["ny"] for _, d in jobs)
        assert info.n_crossings == sum(c.xy.shape[0] for _, c in ref)
        for j in range(len(jobs)):
            assert torch.equal(b.sigma(j), ref[j][0]), j
            _same_contours(b.contours(j), ref[j][1])
        b.close()


@pytest.mark.parametrize("tile,slab,stage", [(32, 8, 0), (16, 4, 128), (32, 2, 512)])
def test_footprint_batch_equals_per_job_slicing(job_set, tile, slab, stage):
    """The persistent footprint kernel over the batch's queue: the same sums
    as per-job slicing with the footprint kernel on the same tiles."""
    import paper_2101_05031_gb300 as cs
    jobs, _ = job_set
    ref = [_per_job(lat, d, slab, "footprint", tile, stage) for lat, d in jobs]
    b = cs.Batch(jobs, slab=slab, ctas_per_sm=2, branches=3, field_kernel="footprint",
                 tile=tile, stage_records=stage)
    b.run()
    info = b.info()
    assert (info.field_kernel, info.tile, info.slab) == (2, tile, slab)
    assert info.stage_records == (stage or 256)
    for j in range(len(jobs)):
        assert torch.equal(b.sigma(j), ref[j][0]), j
        _same_contours(b.contours(j), ref[j][1])
    b.close()


def test_batch_against_oracle(job_set):
    """One job's field and contours against the FP64 oracle (two layers)."""
    import paper_2101_05031_gb300 as cs
    jobs, specs = job_set
    # the smallest lattice keeps the oracle fast
    j = min(range(len(jobs) - 2), key=lambda i: specs[i]["edges"].shape[0])
    lat, d = jobs[j]
    sp = specs[j]
    b = cs.Batch(jobs, slab=4)
    b.run()
    sig = b.sigma(j).cpu().numpy()
    cont = b.contours(j)
    for k in (0, d["n_layers"] - 1):
        z = d["z0"] + k * d["dz"]
        ref = oracle.slice_sigma(sp["nodes"], sp["edges"], sp["radius"], R=sp["R"], C=sp["C"],
                                 z0=z, dz=1.0, n_layers=1, x0=d["x0"], y0=d["y0"], nx=d["nx"],
                                 ny=d["ny"], pixel=d["pixel"])[0]
        helpers.assert_field(sig[k], ref, sp["C"])
        m, x = helpers.compare_layer_contours(cont.layer(k), ref, x0=d["x0"], y0=d["y0"],
                                              pixel=d["pixel"], C=sp["C"])
        assert m > 0 and x <= 0.02 * (m + x) + 2


def test_replay_is_stable(job_set):
    import paper_2101_05031_gb300 as cs
    jobs, _ = job_set
    b = cs.Batch(jobs)
    b.run()
    first = [(b.sigma(j).clone(), b.contours(j)) for j in range(len(jobs))]
    for _ in range(3):
        b.run()
    for j in range(len(jobs)):
        assert torch.equal(b.sigma(j), first[j][0])
        _same_contours(b.contours(j), first[j][1])


def test_autotune_and_cache(job_set):
    """The staged search times the block kernel on 16-pixel tiles and the
    footprint kernel on 16- and 32-pixel tiles, then slab depth x CTAs per SM
    for the best, then (footprint) the staging chunk; the choice is the
    fastest candidate, is cached, and gives per-job slicing's results."""
    import paper_2101_05031_gb300 as cs
    jobs, _ = job_set
    b = cs.Batch(jobs[:3], autotune=True)
    info = b.info()
    n = info.n_candidates
    kname = {1: "block", 2: "footprint"}
    ref = [_per_job(lat, d, info.slab, kname[info.field_kernel], info.tile, info.stage_records)
           for lat, d in jobs[:3]]
    assert 8 <= n <= 16 and info.from_cache == 0
    shapes = {(int(info.cand_kernel[i]), int(info.cand_tile[i])) for i in range(n)}
    assert shapes >= {(1, 16), (2, 16), (2, 32)}
    assert len({int(info.cand_slab[i]) for i in range(n)}) >= 2
    if info.field_kernel == 2:
        assert {int(info.cand_stage[i]) for i in range(n)} == {128, 256, 512}
    ms = list(info.cand_ms)[:n]
    assert all(m > 0 for m in ms)
    best = int(np.argmin(ms))
    assert (info.cand_slab[best], info.cand_ctas[best], info.cand_kernel[best],
            info.cand_tile[best], info.cand_stage[best]) == \
        (info.slab, info.ctas_per_sm, info.field_kernel, info.tile, info.stage_records)
    b.run()
    for j in range(3):
        assert torch.equal(b.sigma(j), ref[j][0])
        _same_contours(b.contours(j), ref[j][1])
    b2 = cs.Batch(jobs[:3], autotune=True)
    i2 = b2.info()
    assert i2.from_cache == 1
    assert (i2.slab, i2.ctas_per_sm, i2.field_kernel, i2.tile, i2.stage_records) == \
        (info.slab, info.ctas_per_sm, info.field_kernel, info.tile, info.stage_records)


def test_changed_sizes_are_reported_and_recoverable():
    """Inputs whose counts differ from the plan: the run reports CAPACITY and
    writes nothing out of range; with the planned inputs back, it is exact."""
    import paper_2101_05031_gb300 as cs
    jobs, specs = _jobs(n_layers=6)
    jobs, specs = jobs[:3], specs[:3]
    ref = [_per_job(lat, d, 4) for lat, d in jobs]
    b = cs.Batch(jobs, slab=4, branches=2)
    lat, _ = jobs[1]
    sp = specs[1]
    r0 = torch.tensor(sp["radius"], device="cuda")
    n0 = torch.tensor(sp["nodes"], device="cuda")
    # thicker struts: other crossing counts (the bins depend only on R)
    lat.update(radius=torch.clamp(r0 * 1.25, max=0.95 * lat.R))
    with pytest.raises(cs.CslError) as e:
        b.run()
    assert e.value.code == 5
    lat.update(radius=r0)
    # moved nodes: other bins
    lat.update(nodes=n0 + 0.3)
    with pytest.raises(cs.CslError) as e:
        b.run()
    assert e.value.code == 5
    lat.update(nodes=n0)
    b.run()
    for j in range(3):
        assert torch.equal(b.sigma(j), ref[j][0])
        _same_contours(b.contours(j), ref[j][1])
