"""Host logic of the multi-rank benchmark path, as two gloo ranks on CPU:
each rank slices its own layer offset, the step time is the slowest rank's,
and the rate counts the units of every rank."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    cfg = dict(z0=0.1, dz=0.2, n_layers=10, x0=0.0, y0=0.0, nx=100, ny=80, pixel=0.05)
    kw = bench.slice_kwargs(cfg, rank, world)
    ms = 100.0 * (rank + 1)          # rank 1 is the slow one
    t_max = bench.max_over_ranks(ms, dist, "cpu")
    rate = bench.whole_job_rate(cfg["nx"] * cfg["ny"] * cfg["n_layers"], 3, world, t_max)
    out[rank] = (kw["z0"], t_max, rate)
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks():
    world = 2
    ctx = mp.get_context("spawn")
    with ctx.Manager() as m:
        out = m.dict()
        mp.start_processes(_rank_main, args=(world, _free_port(), out), nprocs=world,
                           join=True, start_method="spawn")
        res = dict(out)
    z = sorted(v[0] for v in res.values())
    assert z[0] == pytest.approx(0.1) and z[1] == pytest.approx(0.2)   # dz / world apart
    for _, t_max, rate in res.values():
        assert t_max == 200.0                       # the slowest rank
        assert rate == pytest.approx(8000 * 10 * 3 * 2 / 0.2)


def test_reference_arm_under_two_ranks():
    """bench.py --impl reference launched as two ranks (torch.distributed.run,
    on CPU): rank 0 times the oracle and prints one JSON line; the other rank
    exits 0 without work."""
    import json
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(_free_port()), "bench.py",
           "--impl", "reference", "--workload", "cubic-bcc-812", "--steps", "1", "--warmup", "1"]
    r = subprocess.run(cmd, cwd=root, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["value"] > 0
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["cpu_baseline"]["kind"] == "oracle"
