// tune.cu -- the autotuner of the every-vertex rank sweep (pr_autotune).
//
// The gather phase of a sweep over every vertex (Static, ND, the pull form of
// DF / DF-P) is bound by the memory system's throughput for scattered 8-byte
// contribution reads: about one L1TEX wavefront each, and one 32-byte L2
// sector each when it misses L1.  Three knobs change how much of that a sweep
// needs and how well its latency is hidden, and the best setting depends on
// the graph's size and degree skew:
//   - threads per block (256, 512, 1024);
//   - quads per lane per warp step (2, 4, 8: loads in flight per lane);
//   - the hub threshold: the contributions of the vertices of highest
//     out-degree (internal ids [0, hub), ordered by decreasing out-degree) are
//     staged in shared memory by every block, so gathers from them cost a few
//     bank wavefronts per warp instead of one L1TEX wavefront per lane.  It is
//     a degree threshold: vertices of out-degree >= odeg[hub - 1] are staged.
// pr_autotune times every candidate on the graph itself (every-vertex sweeps,
// or whole DF / DF-P updates, on the graph's stream, CUDA events) and keeps
// the fastest.  The choice changes
// no result: the fixed-point sums are exact, so every configuration gives the
// same bits.
#include <algorithm>
#include <vector>
#include "dfpr.h"
#include "handle.cuh"
#include "prim.cuh"
#include "frontier.cuh"

using namespace dfpr;

namespace {

// hub sizes tried (clamped to n + 1): none, and sizes that leave 8 and 2
// blocks of shared memory per SM (larger hubs leave too little L1 for the
// misses in flight on large graphs, and cover every vertex of small ones)
constexpr int32_t HUB_CANDIDATES[] = {0, 3072, 13824};

bool same_cfg(const GatherCfg& a, const GatherCfg& b) {
  return a.threads == b.threads && a.qpt == b.qpt && a.hub == b.hub && a.fused == b.fused && a.parts == b.parts;
}

pr_status read_tuning(pr_graph* h, pr_tuning* out) {
  Graph* g = &h->g;
  out->threads = h->gcfg.threads;
  out->quads_per_lane = h->gcfg.qpt;
  out->hub_vertices = std::min<int32_t>(h->gcfg.hub, g->n);
  out->fused_epilogue = h->gcfg.fused;
  out->ranges = h->gcfg.parts;
  out->hub_min_degree = 0;
  if (out->hub_vertices > 0) {
    int32_t d = 0;
    if (cudaMemcpyAsync(&d, g->out.deg + (out->hub_vertices - 1), sizeof(int32_t), cudaMemcpyDeviceToHost,
                        g->stream) != cudaSuccess ||
        cudaStreamSynchronize(g->stream) != cudaSuccess)
      return (pr_status)cuda_fail(g, cudaGetLastError(), "pr_get_tuning");
    out->hub_min_degree = d;
  }
  out->ms_gather = h->gcfg_ms;
  out->candidates = h->gcfg_trials;
  return PR_OK;
}

// candidate settings: every thread count, quads per lane and hub size in
// HUB_CANDIDATES (clamped to n + 1), epilogue inside or after the gather, and
// 1, 2, 4 or 8 vertex ranges (separate epilogue only)
std::vector<GatherCfg> candidates(int32_t n) {
  std::vector<GatherCfg> cands;
  for (int t : {256, 512, 1024})
    for (int q : {2, 4, 8})
      for (int32_t hb : HUB_CANDIDATES)
        for (int f : {0, 1})
          for (int pt : {1, 2, 4, 8}) {
            GatherCfg c;
            c.threads = t;
            c.qpt = q;
            c.hub = std::min<int32_t>(hb, n + 1);
            c.fused = f;
            c.parts = pt;
            bool dup = false;
            for (const GatherCfg& o : cands) dup = dup || same_cfg(o, c);
            if (!dup && gather_cfg_valid(c)) cands.push_back(c);
          }
  return cands;
}

// Static / ND: one Eq. 1 sweep over every vertex per trial, from the current
// contributions.  A trial writes the next contribution buffer (scratch between
// updates) and R in place, so R is saved first and restored at the end; every
// update resets the control block the sweeps add their totals to.
pr_status tune_sweeps(pr_graph* h, double alpha, int32_t reps, GatherCfg* best, float* best_ms, int32_t* trials) {
  Graph* g = &h->g;
  cudaStream_t s = g->stream;
  if (g->tab_alpha != alpha) {
    cudaError_t e = launch_tables(g->tab_sc, g->tab_ab, alpha, g->n, s);
    if (e != cudaSuccess) return (pr_status)cuda_fail(g, e, "pr_autotune");
    g->tab_alpha = alpha;
  }
  SweepParams p = base_params(g, alpha, 1e-6, 1e-6);
  p.Ccur = g->C[g->ccur];
  p.Cnext = g->C[1 - g->ccur];
  p.ntiles_host = g->in.cap >> 2;
  cudaError_t e = cudaMemcpyAsync(h->vec_tmp, g->R, sizeof(double) * (size_t)g->n, cudaMemcpyDeviceToDevice, s);
  if (e != cudaSuccess) return (pr_status)cuda_fail(g, e, "pr_autotune");
  cudaEvent_t e0 = h->ev[4], e1 = h->ev[5];
  auto sweep = [&](const GatherCfg& c) {
    const SweepAux* aux = nullptr;
    cudaError_t ae = sweep_aux(h, c, &aux);
    return ae == cudaSuccess ? launch_full_sweep(SWEEP_FULL, p, c, g->rowbits, g->rowbase, g->anyb, g->done, aux, s)
                             : ae;
  };
  for (const GatherCfg& c : candidates(g->n)) {
    // one untimed sweep (also raises the kernel's shared memory limit), then
    // reps timed ones
    if (sweep(c) != cudaSuccess) {
      cudaGetLastError();   // a configuration this device cannot run is skipped
      continue;
    }
    bool ok = cudaEventRecord(e0, s) == cudaSuccess;
    for (int r = 0; ok && r < reps; r++) ok = sweep(c) == cudaSuccess;
    ok = ok && cudaEventRecord(e1, s) == cudaSuccess && cudaEventSynchronize(e1) == cudaSuccess;
    float ms = 0.f;
    if (!ok || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
      cudaError_t err = cudaGetLastError();
      cudaMemcpyAsync(g->R, h->vec_tmp, sizeof(double) * (size_t)g->n, cudaMemcpyDeviceToDevice, s);
      return (pr_status)cuda_fail(g, err != cudaSuccess ? err : cudaErrorUnknown, "pr_autotune");
    }
    ms /= (float)reps;
    ++*trials;
    if (*best_ms < 0.f || ms < *best_ms) {
      *best_ms = ms;
      *best = c;
    }
  }
  e = cudaMemcpyAsync(g->R, h->vec_tmp, sizeof(double) * (size_t)g->n, cudaMemcpyDeviceToDevice, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  return e == cudaSuccess ? PR_OK : (pr_status)cuda_fail(g, e, "pr_autotune");
}

// DF / DF-P: reps whole updates per trial (host loop, sweep kernels timed with
// events), each from the ranks the graph had on entry and with its last batch;
// those ranks are put back at the end.
pr_status tune_updates(pr_graph* h, int method, double alpha, double tau, int32_t reps, GatherCfg* best,
                       float* best_ms, int32_t* trials) {
  Graph* g = &h->g;
  cudaStream_t s = g->stream;
  double* saved = nullptr;
  cudaError_t e = dev_malloc((void**)&saved, sizeof(double) * (size_t)g->n);
  if (e != cudaSuccess) return (pr_status)cuda_fail(g, e, "pr_autotune");
  e = cudaMemcpyAsync(saved, g->R, sizeof(double) * (size_t)g->n, cudaMemcpyDeviceToDevice, s);
  const GatherCfg keep = h->gcfg;
  pr_status st = e == cudaSuccess ? PR_OK : (pr_status)cuda_fail(g, e, "pr_autotune");
  for (const GatherCfg& c : candidates(g->n)) {
    if (st != PR_OK) break;
    h->gcfg = c;
    double ms = 0.0;
    for (int r = 0; r < reps && st == PR_OK; r++) {
      e = cudaMemcpyAsync(g->R, saved, sizeof(double) * (size_t)g->n, cudaMemcpyDeviceToDevice, s);
      if (e == cudaSuccess) e = launch_contrib_all(g->R, g->C[g->ccur], g->out.deg, g->tab_sc, g->n, s);
      if (e != cudaSuccess) {
        st = (pr_status)cuda_fail(g, e, "pr_autotune");
        break;
      }
      pr_stats out{};
      st = run_update(h, method, alpha, tau, 1e-6, 1e-6, 500, PR_OPT_TIME_SWEEPS | PR_OPT_HOST_LOOP, &out);
      ms += out.ms_sweep;
    }
    if (st != PR_OK) break;
    ++*trials;
    if (*best_ms < 0.f || ms / reps < *best_ms) {
      *best_ms = (float)(ms / reps);
      *best = c;
    }
  }
  h->gcfg = keep;
  if (st == PR_OK) {
    e = cudaMemcpyAsync(g->R, saved, sizeof(double) * (size_t)g->n, cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess) e = launch_contrib_all(g->R, g->C[g->ccur], g->out.deg, g->tab_sc, g->n, s);
    if (e != cudaSuccess) st = (pr_status)cuda_fail(g, e, "pr_autotune");
  }
  cudaStreamSynchronize(s);
  cudaFree(saved);
  return st;
}

}  // namespace

extern "C" {

pr_status pr_autotune(pr_graph* h, pr_method method, double alpha, double tau, int32_t reps, pr_tuning* out) {
  if (!h || reps < 0 || reps > 100) return PR_EINVAL;
  if (!(alpha >= 0.0 && alpha < 1.0) || !(tau >= 0.0)) return PR_EINVAL;
  Graph* g = &h->g;
  g->err.clear();
  const bool sweeps = method == PR_STATIC || method == PR_NAIVE_DYNAMIC;
  if (!sweeps && method != PR_DF && method != PR_DFP) return PR_EINVAL;
  if (!sweeps && !g->has_ranks)
    return (pr_status)set_error(g, ENORANKS_, "pr_autotune: DF / DF-P trials need ranks");
  if (reps == 0) reps = sweeps ? 3 : 1;
  GatherCfg best = h->gcfg;
  float best_ms = -1.f;
  int32_t trials = 0;
  pr_status st = sweeps ? tune_sweeps(h, alpha, reps, &best, &best_ms, &trials)
                        : tune_updates(h, (int)method, alpha, tau, reps, &best, &best_ms, &trials);
  if (st != PR_OK) return st;
  if (best_ms < 0.f) return (pr_status)set_error(g, PR_ECUDA, "pr_autotune: no configuration could be launched");
  h->gcfg = best;
  h->gcfg_ms = best_ms;
  h->gcfg_trials = trials;
  // graphs that pr_update runs with the loop on the device use the group
  // kernels of a one-graph group: tune its unit sizes too
  if (g->in.cap < PR_DEVICE_LOOP_SLOTS && g->has_ranks) {
    if (!h->solo) {
      pr_graph* one[1] = {h};
      st = pr_group_create(1, one, g->stream, &h->solo);
      if (st != PR_OK) return st;
    }
    st = pr_group_autotune(h->solo, method, alpha, tau, 1, nullptr);
    if (st != PR_OK) return st;
  }
  return out ? read_tuning(h, out) : PR_OK;
}

pr_status pr_get_tuning(const pr_graph* hc, pr_tuning* out) {
  if (!hc || !out) return PR_EINVAL;
  return read_tuning(const_cast<pr_graph*>(hc), out);
}

pr_status pr_set_tuning(pr_graph* h, const pr_tuning* in) {
  if (!h || !in) return PR_EINVAL;
  GatherCfg c;
  c.threads = in->threads;
  c.qpt = in->quads_per_lane;
  c.hub = in->hub_vertices;
  c.fused = in->fused_epilogue;
  c.parts = in->ranges;
  if (c.hub < 0 || !gather_cfg_valid(c)) return PR_EINVAL;
  c.hub = std::min<int32_t>(c.hub, h->g.n + 1);
  h->gcfg = c;
  h->gcfg_ms = 0.f;
  h->gcfg_trials = 0;
  return PR_OK;
}

}  // extern "C"
