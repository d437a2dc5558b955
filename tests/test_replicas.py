"""The replica runs' host logic on CPU with a two-rank gloo process group:
per-rank seeds, the max-over-ranks timing reduction, the whole-job
throughput, and the reference arm's non-zero ranks exiting without work."""
from __future__ import annotations

import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    from paper_2111_14704_gb300.replicas import job_throughput, reduce_max, replica_seed
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    local = [10.0 + 5.0 * rank, 1.0 - 0.25 * rank]          # rank 1 slower, rank 0 slower e2e
    ms_max, e2e_max = reduce_max(local, world)
    dist.barrier()
    out.put((rank, replica_seed(2, rank), ms_max, e2e_max, job_throughput(world, 1000, 4, ms_max)))
    dist.destroy_process_group()


def test_two_rank_gloo_reduction_and_throughput():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, s0, m0, e0, v0), (r1, s1, m1, e1, v1) = res
    assert (s0, s1) == (2, 3)                  # independent boxes
    assert m0 == m1 == 15.0 and e0 == e1 == 1.0
    assert v0 == v1 == pytest.approx(2 * 1000 * 4 / 15e-3)


def test_single_rank_is_identity():
    from paper_2111_14704_gb300.replicas import job_throughput, reduce_max
    assert reduce_max([3.0, 4.0], 1) == [3.0, 4.0]
    assert job_throughput(1, 10, 2, 1.0) == pytest.approx(20000.0)


def test_reference_arm_other_ranks_exit_without_work():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--gpus", "2", "--steps", "1", "--warmup", "1"],
                       capture_output=True, text=True, env=env, timeout=120, cwd=ROOT)
    assert r.returncode == 0 and r.stdout.strip() == ""
