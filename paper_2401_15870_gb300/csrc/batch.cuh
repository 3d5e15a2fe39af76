// batch.cuh -- in-place batch edit of the device graph (Sec. 3.2).
#pragma once
#include "graph.cuh"

namespace dfpr {

// endpoint arrays are device pointers in user ids; validated unless `validated`
int apply_batch_device(Graph* g, const int32_t* ds, const int32_t* dd, int64_t nd, const int32_t* is,
                       const int32_t* id, int64_t ni, bool validated);

}  // namespace dfpr
