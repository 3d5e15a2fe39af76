"""The multi-GPU form of the benchmark is independent replicas (the update
does not shard): every rank runs its own graph, and the job's time is the
slowest rank's.  Its host logic -- replica seeds, the max over ranks, the
whole-job rate, rank 0 alone printing the reference arm -- runs here as two
gloo ranks on the CPU."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
torch = pytest.importorskip("torch")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    sys.path.insert(0, ROOT)
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        local_ms = [120.0, 95.5][rank]
        ms = bench.max_over_ranks(local_ms, world, "cpu")
        rate = bench.job_rate(world, 20, ms)
        seed = bench.replica_seed(2000, rank)
        dist.barrier()
        with open(os.path.join(out_dir, "rank%d.txt" % rank), "w") as f:
            f.write("%r %r %r\n" % (ms, rate, seed))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time(tmp_path):
    import torch.multiprocessing as mp
    world = 2
    mp.start_processes(_rank_main, args=(world, _free_port(), str(tmp_path)), nprocs=world, start_method="spawn")
    got = [open(tmp_path / ("rank%d.txt" % r)).read().split() for r in range(world)]
    for ms, rate, _ in got:
        assert float(ms) == 120.0                        # every rank sees the slowest time
        assert float(rate) == pytest.approx(2 * 20 / 0.120)
    assert got[0][2] != got[1][2]                         # each replica draws its own graph


def test_single_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(7.5, 1, "cpu") == 7.5
    assert bench.job_rate(1, 10, 500.0) == 20.0


def test_reference_arm_runs_on_rank_zero_only(capsys):
    """Under torchrun every rank but 0 leaves the reference arm at once,
    without running the oracle or printing."""
    sys.path.insert(0, ROOT)
    import bench
    old = sys.argv
    sys.argv = ["bench.py", "--impl", "reference"]
    try:
        a = bench.parse()
    finally:
        sys.argv = old
    assert bench.run_reference(a, 1, 2) is None
    assert capsys.readouterr().out == ""
