// handle.cuh -- the opaque pr_graph handle of the C ABI: one graph and the
// host-side scratch of its drivers.
#pragma once
#include <vector>
#include "dfpr.h"
#include "graph.cuh"
#include "sweep.cuh"

struct pr_graph {
  dfpr::Graph g;
  cudaEvent_t ev[6] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
  double ms_apply = 0.0;
  int32_t* lbits_tmp = nullptr;   // bits_to_list scratch
  int64_t* ls_tmp = nullptr;      // list scan scratch
  int64_t tiles_cap = 0;          // capacity of the tile tables
  double* vec_tmp = nullptr;      // n doubles (rank import / export)
  struct pr_group* solo = nullptr;  // one-graph group behind the device loop of pr_update
  dfpr::GatherCfg gcfg;            // gather configuration of every-vertex sweeps (pr_autotune)
  dfpr::SweepAux saux;             // second stream and events of sweeps in several ranges (made on first use)
  float gcfg_ms = 0.f;              // its measured gather time (0: not measured)
  int32_t gcfg_trials = 0;          // configurations the last pr_autotune timed
  std::vector<pr_sweep_record> sweep_log;   // per-sweep trace of the last timed host-loop update
};

namespace dfpr {
// sweep parameters of a graph's current state (api.cu)
SweepParams base_params(Graph* g, double alpha, double tau_f, double tau_p);
// the graph's sweep auxiliary, created on first use for a setting with
// several ranges (api.cu); NULL when the setting has one range
cudaError_t sweep_aux(pr_graph* h, const GatherCfg& c, const SweepAux** out);
// one update with the iteration loop on the host (api.cu); the arguments are
// validated by the caller
pr_status run_update(pr_graph* h, int method, double alpha, double tau, double tau_f, double tau_p, int32_t max_iter,
                     int32_t flags, pr_stats* out);
}
