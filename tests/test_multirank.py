"""The replicas path of bench.py (one independent problem per rank, no
collective on the data path) as two gloo ranks on the CPU: the rank seeds,
the slowest-rank time reduction, the whole-job value, and the reference arm
that only rank 0 runs."""
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


def _rank_main(rank, world, port, times, out):
    sys.path.insert(0, ROOT)
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port), "RANK": str(rank),
                       "WORLD_SIZE": str(world)})
    import torch.distributed as dist
    import bench
    from paper_2410_09663_b300 import workloads
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        wl = bench.replica_workload(workloads.small_16(), rank)
        t = bench.max_over_ranks(times[rank], world)
        out.put((rank, wl.seed, t, bench.job_value(7, world, t[0])))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_reduce_to_the_slowest_replica():
    world, port = 2, _free_port()
    times = [[1.5, 0.25], [0.75, 2.0]]
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, times, out)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(out.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, s0, t0, v0), (r1, s1, t1, v1) = res
    assert (r0, r1) == (0, 1)
    assert s1 == s0 + 1                              # independent problem per rank
    assert t0 == t1 == [1.5, 2.0]                    # element-wise max over ranks
    assert v0 == v1 == pytest.approx(2 * 7 / 1.5)    # all ranks' steps over the slowest time


def test_single_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks([3.0, 4.0], 1) == [3.0, 4.0]
    assert bench.job_value(10, 1, 2.0) == 5.0


def test_reference_arm_runs_on_rank_zero_only(monkeypatch, capsys):
    """Under torchrun the oracle arm is timed on rank 0; the other ranks
    exit 0 at once, without work and without output."""
    sys.path.insert(0, ROOT)
    import bench
    from paper_2410_09663_b300 import workloads
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    args = bench.main.__globals__["argparse"].Namespace(steps=1, warmup=3, gpus=2)
    assert bench.run_reference(args, workloads.small_16()) == 0
    assert capsys.readouterr().out == ""
