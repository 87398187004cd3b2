"""The benchmark's multi-rank bookkeeping on CPU: two `gloo` ranks agree on the slowest rank's
time, the whole-job rate counts every rank's share against it, and the CPU reference arm does
no work on ranks other than 0.  (The GPU arm runs the same helpers over NCCL, one rank per GPU.)"""
import multiprocessing as mp
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402

torch = pytest.importorskip("torch")


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        slowest = bench.max_over_ranks(10.0 * (rank + 1), dist, "cpu")  # rank r took 10 (r + 1) ms
        q.put((rank, slowest))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_agree_on_the_slowest_time():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = dict(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert got == {0: 20.0, 1: 20.0}
    # each rank searched 1,000 queries; the job did 2,000 in the slowest rank's 20 ms
    assert bench.whole_job_rate(1000, 2, got[0]) == pytest.approx(100_000.0)


def test_single_process_is_its_own_maximum():
    assert bench.max_over_ranks(3.5) == 3.5


def test_reference_arm_does_nothing_off_rank_0(monkeypatch):
    monkeypatch.setenv("RANK", "1")
    args = bench.argparse.Namespace(gpus=2, steps=1, warmup=3)
    assert bench.run_reference(args) == 0
