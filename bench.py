"""Benchmark: DF-P batch updates on an R-MAT scale-25 graph on GB300.

One step = one batch update of the hot path: pr_apply_batch (in-place edit of
the CSR and its transpose, effective change) followed by pr_update with DF-P
(initial marking, frontier sweeps with expansion and pruning, convergence),
for a random 80/20 batch of 1e-4 |E| edges (Sec. 5.2.2 of the paper) on a
synthetic R-MAT graph with 2^25 vertices and 2^30 drawn edges (Table 2
stand-in).  Batches follow one another on the evolving graph.

value  = batch updates per second, inputs resident in HBM (device batches,
         pr_apply_batch_device + pr_update).
e2e    = the same through host buffers: pinned host batches in, ranks of all
         vertices back to host memory (pr_apply_batch, pr_update, pr_ranks).
roofline: the DF-P rank-sweep kernel, algorithmic bytes (12 B per processed
         in-edge + 60 B per processed vertex) over its CUDA-event time.

cpu_baseline / parity: before the timed steps, the CPU oracle (the plain C
reference of the method, built with OpenMP over the host cores) runs one
apply + DF-P update of the same workload at full size from its own Static
ranks, which the GPU also takes; the GPU's ranks are compared with it
element by element and the oracle's update is timed.

--impl reference times the same oracle on a bounded sample of the workload
(1/16 of the drawn edges per step) on the host cores.
"""
from __future__ import annotations

import argparse
import dataclasses
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "DF-P batch-update time & HBM GB/s; served updates/s, p50/p99 vs plain launches"
ALPHA, TAU = 0.85, 1e-10
SWEEP_BYTES_PER_EDGE = 12
SWEEP_BYTES_PER_VERTEX = 60
# DRAM bytes (read + write) of one pull-form DF-P sweep (k_gather_rows + k_finish_pull) on the
# default workload, from the ncu capture of the current kernels under profiles/ (R-MAT scale 24,
# scaled by the in-edges walked), keyed by the gather setting (threads, quads per lane, hub vertices,
# fused epilogue, ranges); a setting without a capture of the current kernels reports null
SWEEP_DRAM_BYTES_RMAT25 = {(1024, 2, 0, 0, 1): 11.45e9, (512, 2, 0, 0, 1): 11.45e9}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--scale", type=int, default=25)
    ap.add_argument("--edge-factor", type=int, default=32)
    ap.add_argument("--batch-frac", type=float, default=1e-4)
    ap.add_argument("--seed", type=int, default=2000)
    ap.add_argument("--e2e-steps", type=int, default=5)
    ap.add_argument("--async-steps", type=int, default=5,
                    help="large: DF-P steps in the asynchronous order after the timed ones (reported in detail)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--workload", default="large",
                    choices=["large", "batched", "serving", "methods", "temporal", "tolerances", "orders", "settings"],
                    help="large: one R-MAT scale-25 graph (default); batched: a group of R-MAT graphs updated "
                         "together; serving: Poisson request arrivals for resident graphs")
    ap.add_argument("--rates", default="50,200,500,1000,2000", help="serving: arrival rates (requests/s)")
    ap.add_argument("--max-requests", type=int, default=400, help="serving: requests per rate at most")
    ap.add_argument("--batch-fracs", default="1e-7,1e-6,1e-5,1e-4,1e-3,1e-2,1e-1",
                    help="methods: batch sizes as fractions of |E|")
    ap.add_argument("--reps", type=int, default=1, help="methods: batches per size")
    ap.add_argument("--temporal-batches", type=int, default=100, help="temporal: consecutive batches per size")
    ap.add_argument("--tolerance-batches", type=int, default=10, help="tolerances: consecutive batches")
    ap.add_argument("--graphs", type=int, default=64, help="batched: graphs in the group")
    ap.add_argument("--tune", default="auto",
                    help="large: setting of the every-vertex sweeps: auto (pr_autotune on the first warm-up "
                         "update), default, or threads,quads_per_lane,hub_vertices,fused_epilogue[,ranges]; "
                         "batched: auto, default, or the group's quads_per_lane,steps_per_unit,chunks_per_unit")
    ap.add_argument("--group-loop", default="device", choices=["device", "host"],
                    help="batched: iteration loop of the group update (host: kernels launched one by one)")
    return ap.parse_args()


def workload_name(a):
    return ("R-MAT scale %d (2^%d vertices, %d x 2^%d drawn edges, a,b,c,d=.57,.19,.19,.05), self-loops, "
            "DF-P after each random 80/20 batch of %g |E|" % (a.scale, a.scale, a.edge_factor, a.scale, a.batch_frac))


# ------------------------------------------------------------------ clocks

class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        time.sleep(0.3)

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.2)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 8:
                rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[0]) for r in rows if r[0].replace(".", "").isdigit()]
        mx = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[4 + i].lower() == "active"})
        loaded = [s for s in sm if mx and s > 0.5 * max(mx)] or sm
        return {"sm_mhz": statistics.median(loaded) if loaded else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


# ------------------------------------------------------------------ CPU oracle

REF_SAMPLE_SCALE_DROP = 4   # the reference arm's per-step sample: 1/16 of the drawn edges


def cpu_model():
    """The host CPU's model name (lscpu, else /proc/cpuinfo)."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=20).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return "unknown"


def full_size_parity(a, G, n, src_host, dst_host, batch_host):
    """Parity and CPU baseline on the benchmark workload itself.

    The oracle (the same C source built with OpenMP, every host core, the
    same bits as its single-threaded build) builds the graph from the same
    drawn edges and computes R_{t-1} by Static at tau = 1e-10.  Both sides take
    those ranks (the GPU through pr_set_ranks), apply the same batch and run
    DF-P; the GPU's ranks are compared with the oracle's element by element.
    The oracle's apply + DF-P is the timed CPU baseline."""
    import numpy as np

    import oracle
    t0 = time.perf_counter()
    O = oracle.Graph(n, src_host, dst_host, parallel=True)
    t_create = time.perf_counter() - t0
    t0 = time.perf_counter()
    r0, st_static = O.update("static", alpha=ALPHA, tau=TAU)
    t_static = time.perf_counter() - t0
    G.set_ranks(r0)
    G.apply_batch(*batch_host)
    gst = G.update("dfp", alpha=ALPHA, tau=TAU)
    r_gpu = G.ranks()
    t0 = time.perf_counter()
    O.apply_batch(*batch_host)
    t_apply = time.perf_counter() - t0
    ref, ost = O.update("dfp", alpha=ALPHA, tau=TAU, r_prev=r0)
    t_update = time.perf_counter() - t0
    linf = float(np.max(np.abs(r_gpu - ref)))
    m_graph = O.m
    del O
    threads = oracle.threads()
    same = (gst.iterations, gst.vertices_ever_affected, gst.vertices_processed) == \
        (ost.iterations, ost.vertices_ever_affected, ost.vertices_processed)
    parity = {
        "what": "DF-P ranks of the whole graph after one batch of the benchmark workload, GPU against the oracle "
                "from the same R_{t-1} (the oracle's Static, tau=1e-10), element by element",
        "linf": linf, "tol": 1e-9, "pass": linf < 1e-9 and gst.iterations == ost.iterations,
        "iterations": [gst.iterations, ost.iterations],
        "vertices_ever_affected": [gst.vertices_ever_affected, ost.vertices_ever_affected],
        "vertex_updates": [gst.vertices_processed, ost.vertices_processed],
        "same_decisions": same,
        # the nearest expand / prune / stop decision to its threshold (relative): where it is far below
        # the GPU's relative error on those quantities, a decision may go the other way
        "oracle_nearest_tie_rel": ost.tie_rel,
        "oracle_static_iterations": st_static.iterations,
        "oracle_seconds": {"create": t_create, "static": t_static, "apply": t_apply, "apply_dfp": t_update},
    }
    cb = {"value": 1.0 / t_update, "unit": "updates/s", "cores": threads, "kind": "oracle",
          "cpu_model": cpu_model(),
          "sample": "the whole workload, one update: oracle (plain C, the same source built with OpenMP, %d threads) "
                    "apply + DF-P of one %d-edge batch on the full graph (%d vertices, %d edges) from its own "
                    "Static ranks; %.1f s (apply %.1f s), not scaled"
                    % (threads, len(batch_host[0]) + len(batch_host[2]), n, m_graph, t_update, t_apply)}
    return parity, cb


def reference_sample(a, steps):
    """The reference arm's steps: the oracle (OpenMP build, every host core)
    on R-MAT scale a.scale - REF_SAMPLE_SCALE_DROP with the same edge factor
    and batch fraction, one apply + DF-P per step on the evolving graph;
    returns (seconds per step, edges, scale)."""
    import oracle
    import synth
    sc = max(1, a.scale - REF_SAMPLE_SCALE_DROP)
    n = 1 << sc
    src, dst = synth.rmat(sc, a.edge_factor << sc, a.seed)
    g = oracle.Graph(n, src, dst, parallel=True)
    r, _ = g.update("static", alpha=ALPHA, tau=TAU)
    size = max(1, int(round(a.batch_frac * g.m)))
    times = []
    for i in range(steps):
        b = synth.batch(n, src, dst, size, a.seed + 1 + i)
        t0 = time.perf_counter()
        g.apply_batch(*b)
        r, _ = g.update("dfp", alpha=ALPHA, tau=TAU, r_prev=r)
        times.append(time.perf_counter() - t0)
    return times, g.m, sc


def replica_seed(seed, rank):
    """Seed of rank `rank`'s replica: every rank draws its own graph and batches."""
    return seed + 7919 * rank


def max_over_ranks(x, world, device):
    """The largest of every rank's x (a time): the job is as slow as its
    slowest replica.  With one rank, x itself."""
    if world <= 1:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def job_rate(world, units_per_rank, ms):
    """Whole-job throughput: the units all ranks processed over the slowest
    rank's time."""
    return world * units_per_rank / (ms / 1000.0)


def run_reference(a, rank, world):
    if rank != 0:
        return
    import oracle
    times, m_sample, sc = reference_sample(a, a.warmup + a.steps)
    timed = times[a.warmup:] or times
    per = statistics.median(timed)
    ratio = 2.0 ** (sc - a.scale)
    value = ratio / per
    cb = {"value": value, "unit": "updates/s", "cores": oracle.threads(), "kind": "oracle", "cpu_model": cpu_model(),
          "sample": "oracle (plain C, the same source built with OpenMP, %d threads) apply + DF-P per step on R-MAT "
                    "scale %d (%d edges, the same edge factor and batch fraction), %d timed steps; median %.3f s per "
                    "update, scaled by the drawn-edge ratio 2^%d to the full workload (one full-size update is "
                    "measured by the GPU arm's cpu_baseline)" % (oracle.threads(), sc, m_sample, len(timed), per,
                                                                  sc - a.scale)}
    line = {"metric": METRIC, "value": value, "unit": "updates/s", "n_gpus": world, "steps": len(timed),
            "warmup": a.warmup, "ms_per_step": 1000.0 * per / ratio, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": workload_name(a), "inputs": "larger than L2", "sample_scale": sc},
            "impl": "reference", "cpu_baseline": cb,
            "e2e": {"value": value, "unit": "updates/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ GPU arm

def run_gpu(a, rank, world, local_rank):
    import numpy as np
    import torch

    import paper_2401_15870_gb300 as pr
    import synth.gpu as sg

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    stream = torch.cuda.current_stream()
    n = 1 << a.scale
    seed = replica_seed(a.seed, rank)    # independent replica per rank
    src, dst = sg.rmat(a.scale, a.edge_factor << a.scale, seed)
    G = pr.Graph.from_edges(n, src, dst, device=True, stream=stream)
    m0 = G.m
    st0 = G.update("static", alpha=ALPHA, tau=TAU, time_sweeps=True)
    full_sweep_ms = st0.ms_sweep / max(st0.sweeps, 1)
    size = max(1, int(round(a.batch_frac * m0)))
    nb = a.warmup + a.steps
    dev_batches = [sg.batch(n, src, dst, size, seed + 1 + i) for i in range(nb)]
    async_batches = [sg.batch(n, src, dst, size, seed + 300001 + i) for i in range(a.async_steps)]
    host_batches = []
    for i in range(a.e2e_steps):
        bt = sg.batch(n, src, dst, size, seed + 100001 + i)
        host_batches.append([t.cpu().pin_memory() for t in bt])
    parity_inputs = None
    if not a.no_cpu_baseline and world == 1:
        # the same drawn edges and one more batch, for the oracle
        parity_inputs = (src.cpu().numpy(), dst.cpu().numpy(),
                         [t.cpu().numpy() for t in sg.batch(n, src, dst, size, seed + 200001)])
    torch.cuda.synchronize()
    del src, dst
    parity = cpu_base = None
    if parity_inputs is not None:
        parity, cpu_base = full_size_parity(a, G, n, *parity_inputs)
        del parity_inputs

    sweep_records = []

    def step(b, log=False):
        G.apply_batch_device(*b)
        st = G.update("dfp", alpha=ALPHA, tau=TAU, time_sweeps=True)
        if log:
            sweep_records.extend(G.sweep_log())
        return st

    # the first warm-up step tunes the sweep setting on its own update: every
    # candidate runs that DF-P update from the same ranks (same bits each time)
    first = 0
    if a.tune == "auto" and a.warmup > 0:
        G.apply_batch_device(*dev_batches[0])
        tuning = G.autotune("dfp", alpha=ALPHA, tau=TAU)
        first = 1
    else:
        if a.tune not in ("auto", "default"):
            G.set_tuning(*[int(x) for x in a.tune.split(",")])
        tuning = G.tuning()
    for i in range(first, a.warmup):
        step(dev_batches[i])
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    clocks = ClockSampler(local_rank)
    clocks.start()
    l0 = pr.pr_kernel_launches()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    ev0.record(stream)
    stats = [step(dev_batches[a.warmup + i], log=True) for i in range(a.steps)]
    ev1.record(stream)
    torch.cuda.synchronize()
    launches = pr.pr_kernel_launches() - l0
    clk = clocks.stop()
    ms = max_over_ranks(ev0.elapsed_time(ev1), world, dev)
    value = job_rate(world, a.steps, ms)

    sweep_ms = sum(s.ms_sweep for s in stats)
    sweeps = sum(s.sweeps for s in stats)
    # the dominant kernel: the every-vertex (pull) sweep, k_gather_rows + k_finish_pull; the list (push)
    # sweeps of the first iterations are another kernel, reported beside it
    def alg_bytes(recs):
        return sum(SWEEP_BYTES_PER_EDGE * r[3] + SWEEP_BYTES_PER_VERTEX * r[4] for r in recs)
    pull = [r for r in sweep_records if r[1] == pr.PR_SWEEP_EVERY_VERTEX]
    push = [r for r in sweep_records if r[1] == pr.PR_SWEEP_LIST]
    pull_ms = sum(r[2] for r in pull)
    push_ms = sum(r[2] for r in push)
    achieved = alg_bytes(pull) / (pull_ms / 1000.0) / 1e9 if pull_ms > 0 else 0.0
    all_gbs = (alg_bytes(sweep_records) / ((pull_ms + push_ms) / 1000.0) / 1e9) if pull_ms + push_ms > 0 else 0.0
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        pass
    peak = float(peaks.get("hbm_gbs", 6800.0))
    peak_src = "measured" if "hbm_gbs" in peaks else "fallback"

    # end to end through host buffers: batch in from pinned memory, all ranks out
    r_host = torch.empty(n, dtype=torch.float64).pin_memory()
    r_np = r_host.numpy()
    e2e_ms = None
    h2d = d2h = 0
    if a.e2e_steps > 0:
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for b in host_batches:
            arrs = [t.numpy() for t in b]
            G.apply_batch(*arrs)
            G.update("dfp", alpha=ALPHA, tau=TAU)
            G.ranks(r_np)
        torch.cuda.synchronize()
        e2e_ms = (time.perf_counter() - t0) * 1000.0
        h2d = sum(t.numel() * 4 for t in host_batches[0])
        d2h = n * 8
        e2e_ms = max_over_ranks(e2e_ms, world, dev)
    # the asynchronous order of Alg. 1 (PR_OPT_ASYNC: eight vertex ranges in turn) on the same kind of
    # steps, after everything timed: a reported alternative, not the headline (the synchronous order
    # is the library's canonical reading)
    async_detail = None
    if a.async_steps > 0:
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        ast = []
        for b in async_batches:
            G.apply_batch_device(*b)
            ast.append(G.update("dfp", alpha=ALPHA, tau=TAU, order="async"))
        e1.record(stream)
        torch.cuda.synchronize()
        async_detail = {"updates_per_s": a.async_steps / (e0.elapsed_time(e1) / 1000.0),
                        "iterations_mean": statistics.mean(s.iterations for s in ast),
                        "ms_update_mean": statistics.mean(s.ms_update for s in ast)}
    # one every-vertex sweep with the tuned setting (after everything timed)
    st_nd = G.update("nd", alpha=ALPHA, tau=TAU, max_iter=2, time_sweeps=True, loop="host")
    if rank != 0:
        return
    line = {
        "metric": METRIC, "value": value, "unit": "updates/s", "n_gpus": world, "steps": a.steps,
        "warmup": a.warmup, "ms_per_step": ms / a.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": workload_name(a), "vertices": n, "edges": m0, "batch_edges": size,
                   "inputs": "larger than L2 (graph ~%.0f GB resident)" % (m0 * 8 * 1.2 / 1e9),
                   "parallelism": "replicas" if world > 1 else "single GPU"},
        "roofline": {"bound": "hbm", "kernel": "DF-P every-vertex (pull) rank sweep: k_gather_rows + k_finish_pull, "
                               "one launch pair per iteration", "launches": len(pull),
                     "ms_per_launch": pull_ms / max(len(pull), 1), "achieved": achieved, "peak": peak,
                     "unit": "GB/s", "frac": achieved / peak,
                     "traffic": SWEEP_DRAM_BYTES_RMAT25.get((tuning.threads, tuning.quads_per_lane, tuning.hub_vertices,
                                                             tuning.fused_epilogue, tuning.ranges))
                     if (a.scale, a.edge_factor, a.batch_frac) == (25, 32, 1e-4) else None,
                     "peak_source": peak_src + " (MEASURED_PEAKS.json hbm_gbs)" if peak_src == "measured" else
                     "fallback 6800 GB/s"},
        "e2e": {"value": job_rate(world, a.e2e_steps, e2e_ms) if e2e_ms else None, "unit": "updates/s",
                "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
        "gpu_launches": launches,
        "clocks": clk,
        "detail": {
            "iterations_mean": statistics.mean(s.iterations for s in stats),
            "ms_apply_mean": statistics.mean(s.ms_apply for s in stats),
            "ms_update_mean": statistics.mean(s.ms_update for s in stats),
            "sweep_ms_mean_per_launch": sweep_ms / max(sweeps, 1),
            "sweep_share_of_step": sweep_ms / ms if ms else None,
            "list_sweeps": {"launches": len(push), "ms": push_ms,
                            "gbs": alg_bytes(push) / (push_ms / 1000.0) / 1e9 if push_ms > 0 else None},
            "all_sweeps_gbs": all_gbs,
            "pull_sweep_edges_share": (sum(r[3] for r in pull) / len(pull) / m0) if pull else None,
            "vertices_ever_affected_mean": statistics.mean(s.vertices_ever_affected for s in stats),
            "edges_processed_mean": statistics.mean(s.edges_processed for s in stats),
            "eff_ins_mean": statistics.mean(s.eff_insertions for s in stats),
            "eff_del_mean": statistics.mean(s.eff_deletions for s in stats),
            "gather_setting": dataclasses.asdict(tuning),
            "static_iterations": st0.iterations,
            "full_sweep_ms_default_setting": full_sweep_ms,
            "full_sweep_ms": st_nd.ms_sweep / max(st_nd.sweeps, 1),
            "full_sweep_gbs": (SWEEP_BYTES_PER_EDGE * st_nd.edges_processed + 40 * st_nd.vertices_processed)
            / (st_nd.ms_sweep / 1000.0) / 1e9 if st_nd.ms_sweep else None,
            "async_order": async_detail,
        },
    }
    if cpu_base is not None:
        line["cpu_baseline"] = cpu_base
        line["parity"] = parity
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ batched workload

def batched_specs(a):
    """Graph sizes of the batched workload: scale uniform over the integers
    12..21 (vertex counts log-uniform in 2^12 .. 2^21), edge factor uniform in
    8..32, one seed per graph."""
    import numpy as np
    rng = np.random.default_rng(a.seed)
    return [(int(rng.integers(12, 22)), int(rng.integers(8, 33)), a.seed + 1000 * (i + 1)) for i in range(a.graphs)]


def batched_name(a):
    return ("%d R-MAT graphs (scales 12..21 uniform, edge factor 8..32 uniform, a,b,c,d=.57,.19,.19,.05), "
            "self-loops, each DF-P-updated after its own random 80/20 batch of %g |E|; one group update "
            "(pr_group_update) per step" % (a.graphs, a.batch_frac))


def run_batched(a, rank, world, local_rank):
    import torch

    import paper_2401_15870_gb300 as pr
    import synth.gpu as sg

    torch.cuda.set_device(local_rank)
    stream = torch.cuda.current_stream()
    specs = batched_specs(a)
    graphs, batches, host_batches, sizes = [], [], [], []
    nb = a.warmup + a.steps
    for scale, ef, seed in specs:
        n = 1 << scale
        src, dst = sg.rmat(scale, ef << scale, replica_seed(seed, rank))
        G = pr.Graph.from_edges(n, src, dst, device=True, stream=stream)
        size = max(1, int(round(a.batch_frac * G.m)))
        # batches for the group steps, then as many for the plain steps, then
        # one for tuning
        batches.append([sg.batch(n, src, dst, size, seed + 1 + i) for i in range(2 * nb + 1)])
        host_batches.append([[t.cpu().pin_memory() for t in sg.batch(n, src, dst, size, seed + 50001 + i)]
                             for i in range(a.e2e_steps)])
        graphs.append(G)
        sizes.append((n, G.m, size))
        del src, dst
    torch.cuda.synchronize()
    grp = pr.Group(graphs, stream=stream)
    grp.update("static", alpha=ALPHA, tau=TAU)
    # tuning, before anything is timed: the group's unit sizes on group DF-P
    # updates, and every graph's own settings on its DF-P updates (for the
    # per-graph baseline), all on one extra batch per graph
    gtune, ptune = grp.tuning(), []
    if a.tune not in ("auto", "default"):
        # explicit group unit sizes (quads per lane, warp steps per unit, chunks per unit); graphs untuned
        q, steps, chunks = (int(x) for x in a.tune.split(","))
        grp.set_tuning(quads_per_lane=q, chunks_per_unit=chunks, steps_per_unit=steps)
        gtune = grp.tuning()
    elif a.tune == "auto":
        for G, b in zip(graphs, batches):
            G.apply_batch_device(*b[2 * nb])
        gtune = grp.autotune("dfp", alpha=ALPHA, tau=TAU)
        ptune = [G.autotune("dfp", alpha=ALPHA, tau=TAU) for G in graphs]
        grp.update("dfp", alpha=ALPHA, tau=TAU)

    def group_step(i):
        grp.apply_batches_device([b[i] for b in batches])
        return grp.update("dfp", alpha=ALPHA, tau=TAU, loop=a.group_loop)

    def plain_step(i):
        out = []
        for G, b in zip(graphs, batches):
            G.apply_batch_device(*b[i])
            out.append(G.update("dfp", alpha=ALPHA, tau=TAU))
        return out

    def timed(fn, first):
        for i in range(a.warmup):
            fn(first + i)
        torch.cuda.synchronize()
        l0 = pr.pr_kernel_launches()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        st = [fn(first + a.warmup + i) for i in range(a.steps)]
        ev1.record(stream)
        torch.cuda.synchronize()
        return ev0.elapsed_time(ev1), st, pr.pr_kernel_launches() - l0

    clocks = ClockSampler(local_rank)
    clocks.start()
    ms_g, st_g, launches_g = timed(group_step, 0)
    clk = clocks.stop()
    ms_p, st_p, launches_p = timed(plain_step, nb)
    value = len(graphs) * a.steps / (ms_g / 1000.0)
    plain = len(graphs) * a.steps / (ms_p / 1000.0)

    # end to end through host buffers: every graph's batch from pinned memory,
    # every graph's ranks back to host memory
    e2e_ms, h2d, d2h = None, 0, 0
    if a.e2e_steps > 0:
        r_host = [torch.empty(n, dtype=torch.float64).pin_memory() for n, _, _ in sizes]
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for i in range(a.e2e_steps):
            grp.apply_batches([[t.numpy() for t in hb[i]] for hb in host_batches])
            grp.update("dfp", alpha=ALPHA, tau=TAU)
            for G, r in zip(graphs, r_host):
                G.ranks(r.numpy())
        torch.cuda.synchronize()
        e2e_ms = (time.perf_counter() - t0) * 1000.0
        h2d = sum(sum(t.numel() * 4 for t in hb[0]) for hb in host_batches)
        d2h = sum(n * 8 for n, _, _ in sizes)

    # group sweep loop against HBM: algorithmic bytes of the sweeps over the
    # group update's time (which also holds its init, marking and control)
    flat = [s for step in st_g for s in step]
    upd_ms = sum(step[0].ms_update for step in st_g)
    sweep_bytes = sum(SWEEP_BYTES_PER_EDGE * s.edges_processed + SWEEP_BYTES_PER_VERTEX * s.vertices_processed
                      for s in flat)
    achieved = sweep_bytes / (upd_ms / 1000.0) / 1e9 if upd_ms else 0.0
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        pass
    peak = float(peaks.get("hbm_gbs", 6800.0))
    if rank != 0:
        return
    m_tot = sum(m for _, m, _ in sizes)
    line = {
        "metric": METRIC, "value": value, "unit": "graph updates/s", "n_gpus": world, "steps": a.steps,
        "warmup": a.warmup, "ms_per_step": ms_g / a.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": batched_name(a), "graphs": len(graphs), "vertices": sum(n for n, _, _ in sizes),
                   "edges": m_tot, "batch_edges": sum(b for _, _, b in sizes),
                   "inputs": "larger than L2 (graphs ~%.1f GB resident)" % (m_tot * 8 * 1.2 / 1e9),
                   "parallelism": "single GPU"},
        "plain": {"value": plain, "unit": "graph updates/s", "ms_per_step": ms_p / a.steps,
                  "gpu_launches": launches_p,
                  "what": "the same steps with one pr_apply_batch_device + pr_update per graph"},
        "speedup_vs_plain": value / plain,
        "roofline": {"bound": "hbm", "kernel": "group DF-P loop (k_g_gather + k_g_finish, with init / mark / control)",
                     "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak, "traffic": None},
        "e2e": {"value": len(graphs) * a.e2e_steps / (e2e_ms / 1000.0) if e2e_ms else None,
                "unit": "graph updates/s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
        "gpu_launches": launches_g,
        "clocks": clk,
        "detail": {
            "apply": "pr_apply_batches_device: every graph's batch queued before the host waits",
            "group_unit_sizes": dataclasses.asdict(gtune),
            "per_graph_settings": {"threads": sorted(set(t.threads for t in ptune)),
                                   "quads_per_lane": sorted(set(t.quads_per_lane for t in ptune)),
                                   "hub_vertices": sorted(set(t.hub_vertices for t in ptune)),
                                   "fused_epilogue": sorted(set(t.fused_epilogue for t in ptune)),
                                   "ranges": sorted(set(t.ranges for t in ptune))},
            "group_update_ms_mean": upd_ms / a.steps,
            # in-edges of frontier rows over the in-edges the group's pull sweeps walk
            # (every slot of a live graph per pass)
            "processed_share_of_walked": sum(s.edges_processed for s in flat) /
            max(1, sum(s.iterations * m for step in st_g for s, (_, m, _) in zip(step, sizes))),
            "iterations_max_mean": statistics.mean(max(s.iterations for s in step) for step in st_g),
            "iterations_mean": statistics.mean(s.iterations for s in flat),
            # the batch chains of the graphs overlap on the library's streams, so the
            # edit time of a step is its time less the group update's
            "ms_apply_step_mean": (ms_g - upd_ms) / a.steps,
            "plain_update_ms_sum_mean": statistics.mean(sum(s.ms_update for s in step) for step in st_p),
        },
    }
    print(json.dumps(line), flush=True)
    grp.close()


# ------------------------------------------------------------------ serving workload

# scales of the 16 resident graphs of the serving workload: 18..24 with edge
# factor 16, 16 x sum(2^s) = 2.56e9 drawn edges in all
SERVING_SCALES = [24] * 8 + [23, 23, 22, 21, 20, 19, 18, 18]


def serving_name(a):
    return ("16 resident R-MAT graphs (scales 18..24, edge factor 16, 2.56e9 drawn edges in all), requests with "
            "Poisson arrivals for a uniformly drawn graph, batch sizes log-uniform in 10..1e5 edges (80/20), DF-P; "
            "server (pr_server, grouped: coalescing, solo updates and group updates overlapping batch edits) vs one "
            "pr_apply_batch + pr_update per request")


def run_serving(a, rank, world, local_rank):
    import threading

    import numpy as np
    import torch

    import paper_2401_15870_gb300 as pr
    import synth.gpu as sg

    torch.cuda.set_device(local_rank)
    rng = np.random.default_rng(a.seed + 5)
    specs = [(int(sc), 16, a.seed + 3000 + 17 * i) for i, sc in enumerate(rng.permutation(SERVING_SCALES))]
    graphs, cands = [], []
    for scale, ef, seed in specs:
        n = 1 << scale
        src, dst = sg.rmat(scale, ef << scale, seed)
        graphs.append(pr.Graph.from_edges(n, src, dst, device=True))
        cands.append((n, src, dst))
    torch.cuda.synchronize()
    grp = pr.Group(graphs)
    grp.update("static", alpha=ALPHA, tau=TAU)
    grp.close()
    rates = [float(x) for x in a.rates.split(",")]

    def requests(rate, k0):
        """Poisson arrivals: (arrival offset s, graph, host batch).  The arrival
        times, graphs and sizes depend on the rate only; the edges on k0, so each
        arm gets batches of its own (a batch applied twice changes nothing)."""
        r2 = np.random.default_rng(a.seed + int(rate))
        count = min(a.max_requests, max(400, int(rate * 1.0)))
        t = np.cumsum(r2.exponential(1.0 / rate, count))
        out = []
        for i in range(count):
            g = int(r2.integers(0, len(graphs)))
            size = int(round(10 ** r2.uniform(1, 5)))
            n, src, dst = cands[g]
            b = sg.batch(n, src, dst, size, k0 + i)
            out.append((float(t[i]), g, [x.cpu().numpy() for x in b]))
        return out

    def serve(mode, reqs):
        srv = pr.Server(graphs, mode=mode, method="dfp", alpha=ALPHA, tau=TAU)
        tickets = []
        t0 = pr.pr_server_clock()

        def submitter():
            for at, g, b in reqs:
                dt = t0 + at - pr.pr_server_clock()
                if dt > 0:
                    time.sleep(dt)
                tickets.append(srv.submit(g, *b))
        th = threading.Thread(target=submitter)
        th.start()
        th.join()
        srv.drain(3600)
        infos = [srv.wait(t, 60) for t in tickets]
        srv.close()
        lat = np.array([i.t_done - i.t_submit for i in infos]) * 1000.0
        span = max(i.t_done for i in infos) - t0
        rounds = len({i.round for i in infos})
        return {"updates_per_s": len(infos) / span, "p50_ms": float(np.percentile(lat, 50)),
                "p99_ms": float(np.percentile(lat, 99)), "requests": len(infos), "rounds": rounds,
                "mean_merged": float(np.mean([i.merged for i in infos])),
                "iterations_mean": float(np.mean([i.stats.iterations for i in infos])),
                "eff_edges_mean": float(np.mean([i.stats.eff_insertions + i.stats.eff_deletions for i in infos])),
                "failed": int(sum(1 for i in infos if i.status != 0))}

    rows = []
    l0 = pr.pr_kernel_launches()
    for k, rate in enumerate(rates):
        row = {"rate_per_s": rate}
        for j, mode in enumerate(("grouped", "plain")):
            reqs = requests(rate, a.seed + 100000 * (k + 1) + 50000 * j)
            row["batch_edges_mean"] = float(np.mean([len(b[0]) + len(b[2]) for _, _, b in reqs]))
            row[mode] = serve(mode, reqs)
        rows.append(row)
    launches = pr.pr_kernel_launches() - l0
    if rank != 0:
        return
    top = rows[-1]
    line = {
        "metric": METRIC, "value": top["grouped"]["updates_per_s"], "unit": "served updates/s", "n_gpus": world,
        "steps": sum(r["grouped"]["requests"] for r in rows), "warmup": 0, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": serving_name(a), "graphs": len(graphs), "scales": [s for s, _, _ in specs],
                   "edges": sum(g.m for g in graphs), "inputs": "host batches through pr_server_submit; ranks "
                   "ready on the device at completion", "parallelism": "single GPU"},
        "p50_ms": top["grouped"]["p50_ms"], "p99_ms": top["grouped"]["p99_ms"],
        "plain": {"value": top["plain"]["updates_per_s"], "p50_ms": top["plain"]["p50_ms"],
                  "p99_ms": top["plain"]["p99_ms"]},
        "rates": rows, "gpu_launches": launches,
    }
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ every method over batch sizes

def run_methods(a, rank, world, local_rank):
    """Static, ND, DT, DF and DF-P from the same previous ranks after one batch
    of each size: apply and update times, updated edges/s, iterations, share
    of vertices processed, bytes moved per second, and the L1 error against a
    Static solve of 500 iterations at tau = 0 (the paper's reference solve).
    The graph is put back after every batch by applying its inverse (the
    effective insertions deleted, the effective deletions re-inserted).  On
    graphs of at most 2^16 vertices the CPU oracle runs the same methods on the
    same batch beside it."""
    import numpy as np
    import torch

    import paper_2401_15870_gb300 as pr
    import synth.gpu as sg

    torch.cuda.set_device(local_rank)
    n = 1 << a.scale
    src, dst = sg.rmat(a.scale, a.edge_factor << a.scale, a.seed)
    G = pr.Graph.from_edges(n, src, dst, device=True)
    m0 = G.m
    st0 = G.update("static", alpha=ALPHA, tau=TAU)
    r_prev = G.ranks()
    O = None
    if a.scale <= 16:
        import oracle
        O = oracle.Graph(n, src.cpu().numpy(), dst.cpu().numpy())
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        pass
    peak = float(peaks.get("hbm_gbs", 6800.0))
    rows = []
    for frac in [float(x) for x in a.batch_fracs.split(",")]:
        size = max(1, int(round(frac * m0)))
        for rep in range(a.reps):
            b = sg.batch(n, src, dst, size, a.seed + 1 + rep + int(round(1e9 * frac)) % 100003)
            torch.cuda.synchronize()
            G.set_ranks(r_prev)
            G.apply_batch_device(*b)
            if O is not None:
                O.apply_batch(*[x.cpu().numpy() for x in b])
            ref = G.update("static", alpha=ALPHA, tau=0.0, max_iter=500)
            r_ref = G.ranks()
            for method in ("static", "nd", "dt", "df", "dfp"):
                G.set_ranks(r_prev)
                st = G.update(method, alpha=ALPHA, tau=TAU)
                r = G.ranks()
                eff = st.eff_insertions + st.eff_deletions
                row = {"batch_frac": frac, "batch_edges": size, "effective_edges": eff, "method": method,
                       "ms_apply": st.ms_apply, "ms_update": st.ms_update,
                       "updated_edges_per_s": eff / ((st.ms_apply + st.ms_update) / 1000.0),
                       "iterations": st.iterations, "converged": st.converged,
                       "affected_share": st.vertices_ever_affected / n,
                       "gbs": (SWEEP_BYTES_PER_EDGE * st.edges_processed +
                               (40 if method in ("static", "nd") else SWEEP_BYTES_PER_VERTEX) *
                               st.vertices_processed) / (st.ms_update / 1000.0) / 1e9,
                       "l1_error": float(np.abs(r - r_ref).sum()), "linf_error": float(np.abs(r - r_ref).max())}
                row["hbm_frac"] = row["gbs"] / peak
                if O is not None:
                    t0 = time.perf_counter()
                    ro, ost = O.update(method, alpha=ALPHA, tau=TAU, r_prev=None if method == "static" else r_prev)
                    row["oracle_ms"] = (time.perf_counter() - t0) * 1000.0
                    row["oracle_linf_diff"] = float(np.abs(r - ro).max())
                    row["oracle_iterations"] = ost.iterations
                rows.append(row)
            row_ref = {"batch_frac": frac, "method": "reference static (500 iterations, tau = 0)",
                       "iterations": ref.iterations, "ms_update": ref.ms_update}
            rows.append(row_ref)
            # put the graph back
            dm, dp = G.effective_delta()
            G.apply_batch(dp[:, 0], dp[:, 1], dm[:, 0], dm[:, 1])
            if O is not None:
                O.apply_batch(dp[:, 0], dp[:, 1], dm[:, 0], dm[:, 1])
    if rank != 0:
        return
    dfp = [r for r in rows if r.get("method") == "dfp"]
    line = {
        "metric": METRIC, "value": statistics.mean(r["ms_apply"] + r["ms_update"] for r in dfp),
        "unit": "ms per DF-P batch update (mean over batch sizes)", "n_gpus": world, "higher_is_better": False,
        "dtype": "f64", "data": "synthetic",
        "config": {"workload": "R-MAT scale %d, edge factor %d; every method after one random 80/20 batch per size"
                   % (a.scale, a.edge_factor), "vertices": n, "edges": m0, "static_iterations": st0.iterations},
        "peak_gbs": peak, "rows": rows,
    }
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ temporal stream

def run_temporal(a, rank, world, local_rank):
    """A temporal edge stream of 2.6M vertices and 63M timestamped edges with
    repeats (copying / preferential attachment): the first 90% is the base
    graph; then consecutive insertion-only batches of 1e-5, 1e-4 and 1e-3 |E_T|
    in timestamp order, each followed by DF-P from the previous ranks.  Every
    tenth batch also runs DF and Static from the same previous ranks and a
    Static solve of 500 iterations at tau = 0 as the reference for the L1 error."""
    import numpy as np
    import torch

    import paper_2401_15870_gb300 as pr
    import synth

    torch.cuda.set_device(local_rank)
    n, m_t = 2_600_000, 63_000_000
    t0 = time.perf_counter()
    src, dst = synth.temporal(n, m_t, a.seed + 77)
    gen_s = time.perf_counter() - t0
    base = int(0.9 * m_t)
    out = []
    for frac in (1e-5, 1e-4, 1e-3):
        size = int(round(frac * m_t))
        G = pr.Graph.from_edges(n, src[:base], dst[:base])
        base_m = G.m
        G.update("static", alpha=ALPHA, tau=TAU)
        rec = {"batch_frac": frac, "batch_edges": size, "apply_ms": [], "dfp_ms": [], "dfp_iterations": [],
               "eff_edges": [], "affected_share": [], "checks": []}
        pos = base
        for k in range(a.temporal_batches):
            if pos + size > m_t:
                break
            bs, bd = src[pos:pos + size], dst[pos:pos + size]
            pos += size
            r_prev = G.ranks()
            G.apply_batch(ins_src=bs, ins_dst=bd)
            st = G.update("dfp", alpha=ALPHA, tau=TAU)
            rec["apply_ms"].append(st.ms_apply)
            rec["dfp_ms"].append(st.ms_update)
            rec["dfp_iterations"].append(st.iterations)
            rec["eff_edges"].append(st.eff_insertions)
            rec["affected_share"].append(st.vertices_ever_affected / n)
            if k % 10 == 9:
                r_dfp = G.ranks()
                chk = {"batch": k}
                G.update("static", alpha=ALPHA, tau=0.0, max_iter=500)
                r_ref = G.ranks()
                chk["dfp_l1"] = float(np.abs(r_dfp - r_ref).sum())
                for method in ("df", "static"):
                    G.set_ranks(r_prev)
                    s2 = G.update(method, alpha=ALPHA, tau=TAU)
                    chk[method + "_ms"] = s2.ms_update
                    chk[method + "_iterations"] = s2.iterations
                    chk[method + "_l1"] = float(np.abs(G.ranks() - r_ref).sum())
                rec["checks"].append(chk)
                G.set_ranks(r_dfp)   # the stream goes on from the DF-P ranks
        G.close()
        summ = {"batch_frac": frac, "batch_edges": size, "batches": len(rec["dfp_ms"]),
                "apply_ms_mean": statistics.mean(rec["apply_ms"]), "dfp_ms_mean": statistics.mean(rec["dfp_ms"]),
                "dfp_iterations_mean": statistics.mean(rec["dfp_iterations"]),
                "effective_edges_mean": statistics.mean(rec["eff_edges"]),
                "affected_share_mean": statistics.mean(rec["affected_share"]),
                "updated_edges_per_s": sum(rec["eff_edges"]) / ((sum(rec["apply_ms"]) + sum(rec["dfp_ms"])) / 1e3),
                "static_ms_mean": statistics.mean(c["static_ms"] for c in rec["checks"]),
                "df_ms_mean": statistics.mean(c["df_ms"] for c in rec["checks"]),
                "dfp_l1_mean": statistics.mean(c["dfp_l1"] for c in rec["checks"]),
                "df_l1_mean": statistics.mean(c["df_l1"] for c in rec["checks"]),
                "static_l1_mean": statistics.mean(c["static_l1"] for c in rec["checks"])}
        summ["dfp_speedup_vs_static"] = summ["static_ms_mean"] / summ["dfp_ms_mean"]
        out.append(summ)
    if rank != 0:
        return
    line = {"metric": METRIC, "value": out[1]["dfp_ms_mean"], "unit": "ms per DF-P update (1e-4 |E_T| batches)",
            "n_gpus": world, "higher_is_better": False, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "temporal stream (copying / preferential attachment with repeats), %d vertices, "
                       "%d timestamped edges, base = first 90%%, consecutive insertion-only batches" % (n, m_t),
                       "generation_s": gen_s, "base_edges_with_self_loops": base_m},
            "sizes": out}
    print(json.dumps(line), flush=True)


def run_tolerances(a, rank, world, local_rank):
    """The experiments of Sec. 4.3 and Sec. 4.4 (figures adjust-frontier and
    adjust-prune) on the temporal stream: consecutive insertion-only batches of
    1e-5 |E_T| after a base of the first 90%.  For every batch, every setting
    runs from the same previous ranks (a Static solve of G_{t-1} to its exact
    fixed point) and is timed against Static at tau = 1e-10; the error is the
    L1 distance to the exact fixed point of G_t.
      frontier: DF with each measure -- relative change at tau_f = 0.1 ...
        1e-6, rank change and contribution-factor change at tau_f = tau ...
        tau / 1e5;
      prune: DF-P with the relative change, tau_f in {1e-6, 1e-7, 1e-8},
        tau_p = tau_f ... tau_f / 1e4."""
    import numpy as np
    import torch

    import paper_2401_15870_gb300 as pr
    import synth

    torch.cuda.set_device(local_rank)
    n, m_t = 2_600_000, 63_000_000
    src, dst = synth.temporal(n, m_t, a.seed + 77)
    base = int(0.9 * m_t)
    size = int(round(1e-5 * m_t))
    settings = [("df", "relative", 10.0 ** -k, 10.0 ** -k) for k in range(1, 7)]
    settings += [("df", ms, TAU / 10.0 ** k, TAU / 10.0 ** k) for ms in ("absolute", "contrib") for k in range(0, 6)]
    settings += [("dfp", "relative", tf, tf / 10.0 ** k) for tf in (1e-6, 1e-7, 1e-8) for k in range(0, 5)]
    G = pr.Graph.from_edges(n, src[:base], dst[:base])
    G.update("static", alpha=ALPHA, tau=0.0, max_iter=500)
    r_prev = G.ranks()
    acc = {i: {"ms": [], "l1": [], "share": [], "iters": []} for i in range(len(settings))}
    static = {"ms": [], "l1": [], "iters": []}
    pos = base
    for k in range(a.tolerance_batches):
        G.apply_batch(ins_src=src[pos:pos + size], ins_dst=dst[pos:pos + size])
        pos += size
        G.update("static", alpha=ALPHA, tau=0.0, max_iter=500)
        r_ref = G.ranks()
        s0 = G.update("static", alpha=ALPHA, tau=TAU)
        static["ms"].append(s0.ms_update)
        static["iters"].append(s0.iterations)
        static["l1"].append(float(np.abs(G.ranks() - r_ref).sum()))
        for i, (method, measure, tf, tp) in enumerate(settings):
            G.set_ranks(r_prev)
            st = G.update(method, alpha=ALPHA, tau=TAU, tau_f=tf, tau_p=tp, measure=measure)
            acc[i]["ms"].append(st.ms_update)
            acc[i]["iters"].append(st.iterations)
            acc[i]["share"].append(st.vertices_ever_affected / n)
            acc[i]["l1"].append(float(np.abs(G.ranks() - r_ref).sum()))
        G.set_ranks(r_ref)
        r_prev = r_ref
    if rank != 0:
        return
    rows = []
    for i, (method, measure, tf, tp) in enumerate(settings):
        speed = [s / m for s, m in zip(static["ms"], acc[i]["ms"])]
        rows.append({"method": method, "measure": measure, "tau_f": tf, "tau_p": tp,
                     "speedup_vs_static_mean": statistics.mean(speed),
                     "ms_mean": statistics.mean(acc[i]["ms"]), "iterations_mean": statistics.mean(acc[i]["iters"]),
                     "affected_share_mean": statistics.mean(acc[i]["share"]),
                     "l1_error_mean": statistics.mean(acc[i]["l1"])})
    best = min((r for r in rows if r["l1_error_mean"] <= statistics.mean(static["l1"])),
               key=lambda r: r["ms_mean"], default=None)
    line = {"metric": METRIC, "value": best["speedup_vs_static_mean"] if best else None,
            "unit": "mean speedup over Static of the fastest setting whose error stays at or below Static's",
            "n_gpus": world, "higher_is_better": True, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "temporal stream (copying / preferential attachment with repeats), %d vertices, "
                       "%d timestamped edges, base = first 90%%, %d consecutive insertion-only batches of "
                       "1e-5 |E_T| (%d edges); every setting from the exact fixed point of G_{t-1}"
                       % (n, m_t, a.tolerance_batches, size)},
            "best": best,
            "static": {"ms_mean": statistics.mean(static["ms"]), "iterations_mean": statistics.mean(static["iters"]),
                       "l1_error_mean": statistics.mean(static["l1"])},
            "settings": rows}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ sweep settings

SETTINGS_TABLE = [(256, 4, 0, 0, 1), (512, 4, 0, 0, 1), (1024, 2, 0, 0, 1), (512, 2, 0, 0, 1), (1024, 4, 0, 0, 1),
                  (1024, 4, 13824, 0, 1), (1024, 4, 0, 1, 1), (1024, 2, 0, 1, 1), (1024, 2, 0, 0, 2),
                  (1024, 2, 0, 0, 4)]


def run_settings(a, rank, world, local_rank):
    """Time the every-vertex sweep under fixed settings of pr_set_tuning
    (threads per block, quads per lane, hub vertices, epilogue in the gather
    kernel, vertex ranges) on the benchmark graph: ND sweeps (mean of 3) and the
    pull-form sweeps of one DF-P update (per-sweep trace) after one random
    batch, the same batch and previous ranks for every setting."""
    import numpy as np
    import torch

    import paper_2401_15870_gb300 as pr
    import synth.gpu as sg

    torch.cuda.set_device(local_rank)
    n = 1 << a.scale
    src, dst = sg.rmat(a.scale, a.edge_factor << a.scale, a.seed)
    G = pr.Graph.from_edges(n, src, dst, device=True)
    G.update("static", alpha=ALPHA, tau=TAU)
    size = max(1, int(round(a.batch_frac * G.m)))
    G.apply_batch_device(*sg.batch(n, src, dst, size, a.seed + 1))
    del src, dst
    r0 = torch.empty(n, dtype=torch.float64, device="cuda")
    G.ranks_device(r0)
    rows = []
    for t, q, hub, fused, ranges in SETTINGS_TABLE:
        G.set_tuning(t, q, hub, fused, ranges)
        G.set_ranks_device(r0)
        G.update("nd", alpha=ALPHA, tau=TAU, max_iter=1, time_sweeps=True, loop="host")   # warm-up
        G.set_ranks_device(r0)
        st = G.update("nd", alpha=ALPHA, tau=0.0, max_iter=3, time_sweeps=True, loop="host")
        nd_ms = st.ms_sweep / max(st.sweeps, 1)
        G.set_ranks_device(r0)
        G.update("dfp", alpha=ALPHA, tau=TAU, time_sweeps=True, direction="pull")
        pull = [r[2] for r in G.sweep_log() if r[1] == pr.PR_SWEEP_EVERY_VERTEX and r[3] > 0]
        rows.append({"threads": t, "quads_per_lane": q, "hub_vertices": hub, "fused_epilogue": fused,
                     "ranges": ranges, "nd_sweep_ms": nd_ms, "dfp_pull_sweep_ms": float(np.mean(pull)),
                     "dfp_sweeps": len(pull)})
    if rank != 0:
        return
    best = min(rows, key=lambda r: r["dfp_pull_sweep_ms"])
    line = {"metric": METRIC, "value": best["dfp_pull_sweep_ms"], "unit": "ms per DF-P pull sweep, best setting",
            "n_gpus": world, "higher_is_better": False, "dtype": "f64", "data": "synthetic",
            "config": {"workload": workload_name(a), "edges": G.m}, "settings": rows}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ synchronous and asynchronous order

def run_orders(a, rank, world, local_rank):
    """Sec. 4.4: the synchronous order (every vertex of a sweep reads the ranks
    of the start of the sweep) against the asynchronous one (PR_OPT_ASYNC: eight
    vertex ranges swept in turn, each reading the ranks of the ranges before it
    as updated in the sweep) on the temporal stream: 2.6M vertices, 63M
    timestamped edges, base = first 90%, then a.reps consecutive insertion-only
    batches of each size 1e-5, 1e-4, 1e-3 |E_T|.  Every method starts from the
    exact fixed point of G_{t-1} (Static at tau = 0, 500 iterations) and is
    compared in L1 with the exact fixed point of G_t.  Beside it, the oracle's
    three orders (sync; async: ascending id, one vertex at a time; ranges: the
    GPU's asynchronous schedule) on a 20,000-vertex, 400,000-edge stream of the
    same kind, three batches of 400 insertions."""
    import numpy as np
    import torch

    import oracle
    import paper_2401_15870_gb300 as pr
    import synth

    torch.cuda.set_device(local_rank)
    n, m_t = 2_600_000, 63_000_000
    src, dst = synth.temporal(n, m_t, a.seed + 77)
    base = int(0.9 * m_t)
    G = pr.Graph.from_edges(n, src[:base], dst[:base])
    G.update("static", alpha=ALPHA, tau=0.0, max_iter=500)
    r_prev = G.ranks()
    methods = ("static", "nd", "df", "dfp")
    rows = []
    pos = base
    for frac in (1e-5, 1e-4, 1e-3):
        size = int(round(frac * m_t))
        acc = {(mth, o): {"ms": [], "l1": [], "iters": []} for mth in methods for o in ("sync", "async")}
        for k in range(a.reps):
            G.apply_batch(ins_src=src[pos:pos + size], ins_dst=dst[pos:pos + size])
            pos += size
            G.update("static", alpha=ALPHA, tau=0.0, max_iter=500)
            r_ref = G.ranks()
            for mth in methods:
                for o in ("sync", "async"):
                    G.set_ranks(r_prev)
                    st = G.update(mth, alpha=ALPHA, tau=TAU, loop="host", order=o)
                    acc[(mth, o)]["ms"].append(st.ms_update)
                    acc[(mth, o)]["iters"].append(st.iterations)
                    acc[(mth, o)]["l1"].append(float(np.abs(G.ranks() - r_ref).sum()))
            G.set_ranks(r_ref)
            r_prev = r_ref
        for (mth, o), v in acc.items():
            rows.append({"batch_frac": frac, "batch": size, "method": mth, "order": o,
                         "ms_mean": statistics.mean(v["ms"]), "iterations_mean": statistics.mean(v["iters"]),
                         "l1_error_mean": statistics.mean(v["l1"])})
    # the oracle's orders on a small stream of the same kind
    on, om = 20000, 400000
    s_, d_ = synth.temporal(on, om, 5)
    ob = int(0.9 * om)
    og = oracle.Graph(on, s_[:ob], d_[:ob])
    orp, _ = og.update("static", tau=0.0, max_iter=500)
    orows = []
    opos = ob
    for k in range(3):
        og.apply_batch([], [], s_[opos:opos + 400], d_[opos:opos + 400])
        opos += 400
        oref, _ = og.update("static", tau=0.0, max_iter=500)
        for mth in ("nd", "df", "dfp"):
            for o in ("sync", "async", "ranges"):
                r, st = og.update(mth, r_prev=orp, order=o)
                orows.append({"batch": k, "method": mth, "order": o, "l1_error": float(np.abs(r - oref).sum()),
                              "iterations": st.iterations, "vertex_updates": st.vertices_processed})
        orp = oref
    if rank != 0:
        return
    dfp = {r["order"]: r for r in rows if r["method"] == "dfp" and r["batch_frac"] == 1e-4}
    line = {"metric": METRIC, "value": dfp["async"]["l1_error_mean"], "unit": "DF-P L1 error, asynchronous order, "
            "1e-4 |E_T| batches", "n_gpus": world, "higher_is_better": False, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "temporal stream (copying / preferential attachment with repeats), %d vertices, "
                       "%d timestamped edges, base = first 90%%, %d consecutive insertion-only batches per size; "
                       "every method from the exact fixed point of G_{t-1}" % (n, m_t, a.reps)},
            "gpu": rows, "oracle_20k": orows}
    print(json.dumps(line), flush=True)


def main():
    a = parse()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", str(a.gpus)))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if a.impl == "reference":
        run_reference(a, rank, world if "WORLD_SIZE" in os.environ else a.gpus)
        return
    if world > 1:
        import torch
        torch.cuda.set_device(local_rank)
        torch.distributed.init_process_group("nccl")
    try:
        if a.workload == "batched":
            run_batched(a, rank, world, local_rank)
        elif a.workload == "serving":
            run_serving(a, rank, world, local_rank)
        elif a.workload == "methods":
            run_methods(a, rank, world, local_rank)
        elif a.workload == "temporal":
            run_temporal(a, rank, world, local_rank)
        elif a.workload == "tolerances":
            run_tolerances(a, rank, world, local_rank)
        elif a.workload == "orders":
            run_orders(a, rank, world, local_rank)
        elif a.workload == "settings":
            run_settings(a, rank, world, local_rank)
        else:
            run_gpu(a, rank, world, local_rank)
    finally:
        if world > 1:
            import torch
            torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
