// batch.cuh -- in-place batch edit of the device graph (Sec. 3.2).
#pragma once
#include "graph.cuh"

namespace dfpr {

// endpoint arrays are device pointers in user ids; validated unless `validated`
int apply_batch_device(Graph* g, const int32_t* ds, const int32_t* dd, int64_t nd, const int32_t* is,
                       const int32_t* id, int64_t ni, bool validated);

// the same in two phases, so that the batches of many graphs are queued before
// the host waits for any: a small batch (at most 4096 edges) is queued by
// apply_batch_launch and finished by apply_batch_complete (which waits for the
// graph's stream); a larger one is applied whole by apply_batch_launch.
struct SmallApply {
  struct SmallBufs* B = nullptr;   // set while a small batch is pending
  int32_t* S[2] = {nullptr, nullptr};
  int64_t cap[2] = {0, 0};
  int64_t nk = 0;
};
int apply_batch_launch(Graph* g, const int32_t* ds, const int32_t* dd, int64_t nd, const int32_t* is,
                       const int32_t* id, int64_t ni, bool validated, SmallApply* pending);
int apply_batch_complete(Graph* g, SmallApply* pending);

}  // namespace dfpr
