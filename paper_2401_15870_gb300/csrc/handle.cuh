// handle.cuh -- the opaque pr_graph handle of the C ABI: one graph and the
// host-side scratch of its drivers.
#pragma once
#include "graph.cuh"

struct pr_graph {
  dfpr::Graph g;
  cudaEvent_t ev[6] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
  double ms_apply = 0.0;
  int32_t* lbits_tmp = nullptr;   // bits_to_list scratch
  int64_t* ls_tmp = nullptr;      // list scan scratch
  int64_t tiles_cap = 0;          // capacity of the tile tables
  double* vec_tmp = nullptr;      // n doubles (rank import / export)
  struct pr_group* solo = nullptr;  // one-graph group behind the device loop of pr_update
};
