"""The benchmark's multi-rank logic on CPU (gloo, world size 2): the barrier,
the max-over-ranks reduction of the timed region and the whole-job value,
and that under torchrun only rank 0 of the reference arm prints its line."""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    sys.path.insert(0, ROOT)
    import torch.distributed as tdist
    import bench
    tdist.init_process_group("gloo", rank=rank, world_size=world)
    bench.rank_barrier()
    ms = bench.max_over_ranks(10.0 + 5.0 * rank)  # rank 1 is the slow one
    q.put((rank, ms, bench.job_value(world, 8192, 100, ms)))
    bench.rank_barrier()
    tdist.destroy_process_group()


def test_max_over_ranks_and_job_value_gloo():
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [o[1] for o in out] == [15.0, 15.0]
    assert out[0][2] == out[1][2] == pytest.approx(2 * 8192 * 100 / 15e-3)


def test_single_process_helpers_need_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    bench.rank_barrier()
    assert bench.max_over_ranks(3.5) == 3.5
    assert bench.job_value(1, 10, 2, 1000.0) == 20.0


def test_reference_arm_under_torchrun_prints_once():
    """Two ranks: rank 0 times the oracle and prints one JSON line, rank 1
    exits 0 without work."""
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(_free_port()),
           "bench.py", "--impl", "reference", "--workload", "shear", "--steps", "2", "--warmup", "3"]
    r = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [json.loads(l) for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    assert lines[0]["impl"] == "reference" and lines[0]["n_gpus"] == 2 and lines[0]["value"] > 0
