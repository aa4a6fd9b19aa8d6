"""The bench's N > 1 path (replicas, one independent system per rank) on CPU: two gloo ranks
check the slowest-rank time, the whole-job throughput and the per-rank seeds, and the
reference arm's rank rule (rank 0 alone prints)."""
import multiprocessing as mp
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    sys.path.insert(0, ROOT)
    import torch.distributed as dist

    import bench
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        local_ms = [5.0, 7.5][rank]
        ms = bench.max_over_ranks(local_ms, dist, "cpu")
        value = bench.job_throughput(world, bench.flops(16384, 1), ms * 1e-3)
        q.put((rank, ms, value, bench.rank_seed(rank)))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_replicas_take_the_slowest_rank_and_add_the_work():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    import bench
    assert [o[1] for o in out] == [7.5, 7.5]
    assert out[0][2] == pytest.approx(2 * bench.flops(16384, 1) / 7.5e-3)
    assert out[0][3] != out[1][3]   # each replica solves its own system


def test_single_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.25, None, "cpu") == 3.25
    assert bench.job_throughput(1, 10.0, 2.0) == 5.0


def test_reference_arm_prints_on_rank_zero_only(capsys):
    sys.path.insert(0, ROOT)
    import bench
    a = bench.parse(["--impl", "reference", "--gpus", "2"])
    bench.run_reference(a, rank=1, world=2)   # a non-zero rank does no work and prints nothing
    assert capsys.readouterr().out == ""
