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


def test_reference_arm_line_on_one_rank():
    """The reference arm (the oracle, every host core) prints one JSON line
    with the benchmark's metric and unit, impl "reference", a cpu_baseline
    naming its sample and cores, and an e2e entry of its own value with no
    host-device traffic (here on a small graph: R-MAT scale 12)."""
    import json
    import subprocess
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--scale", "12",
                          "--steps", "2", "--warmup", "1"], capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [l for l in out.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    line = json.loads(lines[0])
    assert line["impl"] == "reference"
    assert line["unit"] == "updates/s" and line["higher_is_better"] is True
    assert line["steps"] == 2 and line["warmup"] == 1 and line["value"] > 0
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == line["value"] and cb["sample"]
    assert line["e2e"] == {"value": line["value"], "unit": "updates/s", "h2d_bytes_per_step": 0,
                           "d2h_bytes_per_step": 0}
