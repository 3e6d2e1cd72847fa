"""bench.py's multi-rank logic on CPU: two gloo ranks take the maximum of
their timings and report the whole-job rate; non-zero ranks of the oracle
(reference) arm exit at once without output."""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _rank(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    mine = [1.0 + rank, 10.0 - rank, 3.0 * (rank + 1)]
    got = bench.max_over_ranks(mine, world, "cpu")
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, got, bench.whole_job_rate(1000, world, got[0])))


def test_max_over_ranks_gloo():
    import multiprocessing as mp
    import socket
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, got, rate in res:
        assert got == [2.0, 10.0, 6.0]                  # element-wise max over the two ranks
        assert rate == pytest.approx(2 * 1000 / 2e-3)  # both ranks' units over the slowest time


def test_reference_arm_other_ranks_exit():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2"],
                       env=env, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0
    assert r.stdout.strip() == ""


def bench_cores():
    sys.path.insert(0, ROOT)
    import bench
    return bench.host_cores()


def test_reference_arm_json_line():
    """Rank 0 of the oracle (reference) arm prints one JSON line with the
    contract's keys: the native arm's metric and config, the oracle's own
    cpu_baseline, and an e2e object that moves no device bytes."""
    import json
    env = dict(os.environ)
    for k in ("RANK", "WORLD_SIZE", "LOCAL_RANK"):
        env.pop(k, None)
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "3", "--ref-step-s", "0.2", "--workload", "lognormal_3m"],
                       env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference"
    assert d["metric"] == "tets assembled+condensed/s" and d["unit"] == "tets/s" and d["higher_is_better"] is True
    assert d["steps"] == 1 and d["warmup"] == 3 and d["n_gpus"] == 1 and d["value"] > 0
    assert d["config"]["workload"] == "lognormal_3m" and d["config"]["nE"] == 3359232
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] == bench_cores() and cb["value"] == d["value"] and cb["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": "tets/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
