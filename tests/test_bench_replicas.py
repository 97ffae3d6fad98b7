"""The multi-replica host logic of bench.py (one process per GPU, independent replicas):
the job rate takes the slowest rank's time and the sum of all ranks' pixels, and the
reference arm runs on rank 0 only.  Two gloo processes on the CPU."""
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    # rank r took 10 (r + 1) ms per step for 1000 (r + 1) pixels
    ms, rate = bench.job_rate(10.0 * (rank + 1), 1000.0 * (rank + 1), world, dist, "cpu")
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, ms, rate))


def test_job_rate_two_gloo_ranks():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=10) for _ in range(world))
    for _, ms, rate in res:
        assert ms == pytest.approx(20.0)                       # the slowest rank
        assert rate == pytest.approx(3000.0 / 20e-3 / 1e6)     # all pixels / slowest time


def test_job_rate_single_rank():
    sys.path.insert(0, ROOT)
    import bench
    ms, rate = bench.job_rate(5.0, 262144, 1)
    assert ms == 5.0 and rate == pytest.approx(262144 / 5e-3 / 1e6)


def test_reference_arm_runs_on_rank_zero_only(monkeypatch, capsys):
    sys.path.insert(0, ROOT)
    import bench

    class Args:
        steps, warmup, gpus = 1, 3, 2
    monkeypatch.setenv("RANK", "1")
    called = []
    monkeypatch.setattr(bench, "run_cpu", lambda *a, **k: called.append(a))
    assert bench.run_reference(Args()) == 0
    assert not called and capsys.readouterr().out == ""


def test_gpus_flag_starts_its_own_ranks():
    """`bench.py --gpus 2` without a launcher starts two ranks itself (torch.distributed.run
    on 127.0.0.1); the reference arm needs no GPU, runs on rank 0 and prints one line."""
    import json
    import subprocess
    env = dict(os.environ)
    for v in ("WORLD_SIZE", "RANK", "LOCAL_RANK", "MASTER_ADDR", "MASTER_PORT"):
        env.pop(v, None)
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--gpus", "2", "--steps", "1", "--warmup", "3"],
                       capture_output=True, text=True, env=env, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    line = json.loads(lines[0])
    assert line["impl"] == "reference" and line["n_gpus"] == 2 and line["value"] > 0
