// noalloc.cu -- one synchronous rank sweep (Eq. 1) over a caller-provided
// in-CSR, for callers that must not allocate device memory.
//
// The regular entry points keep their working memory in the graph handle,
// which pr_graph_create* allocates with cudaMalloc.  Some callers cannot do
// that: code that runs where a device allocation is not allowed or would
// stall other work (cudaMalloc may synchronize the device), for example a
// serving loop whose memory budget is owned by another allocator, or an
// embedding application that hands out all device memory itself.
// pr_sweep_noalloc gives them the rank sweep with no allocation at all: its
// one piece of scratch memory -- the fixed-point contribution of every vertex
// and the L-infinity accumulator -- lives in the file-scope device array
// below, which exists on every GPU that loads this library, from load until
// process exit.
//
// Properties a caller must know:
//   * Size limit: n <= PR_NOALLOC_MAX_N (header); larger n is rejected with
//     PR_EINVAL before any device work.  The array holds PR_NOALLOC_MAX_N + 2
//     int64 values (about 4 MB) whatever n is.
//   * r_out must not overlap r_in: each vertex's change is measured against
//     r_in after r_out is written, so overlapping buffers are rejected.
//   * The first call on a device looks up the array's device address with
//     cudaGetSymbolAddress (once per device, with that device current).  Make
//     that first call before any stream capture on the device.
//   * Every call uses the same array and leaves its contents behind; each
//     call overwrites the contributions and clears the accumulator first.
//     Calls whose work overlaps on the GPU (different streams, or different
//     host threads on one device) race on the array and give wrong results:
//     serialize them.
#include <mutex>
#include "dfpr.h"
#include "common.cuh"
#include "prim.cuh"

namespace {

constexpr int32_t NA_MAX_N = PR_NOALLOC_MAX_N;
constexpr int NA_MAX_DEV = 64;

// [0 .. NA_MAX_N] fixed-point contributions (entry n unused), then the
// accumulator of the L-infinity change as the bit pattern of a non-negative double
struct NoAllocScratch {
  long long contrib[NA_MAX_N + 1];
  unsigned long long delta_bits;
};

__device__ __align__(256) NoAllocScratch na_scratch;

std::mutex na_mu;
NoAllocScratch* na_addr[NA_MAX_DEV] = {nullptr};

// contributions R[u] / |out(u)| in 2^-61 fixed point, exactly as the graph's
// own sweep computes them (2^61 / d, product rounded to nearest); clears the
// accumulator
__global__ void k_na_contrib(int32_t n, const double* __restrict__ r, const int32_t* __restrict__ out_deg,
                             NoAllocScratch* s) {
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
    int32_t d = out_deg[v];
    s->contrib[v] = d > 0 ? __double2ll_rn(r[v] * (dfpr::FIX_ONE / (double)d)) : 0;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) s->delta_bits = 0ull;
}

// one warp per vertex: exact sum of its in-neighbours' contributions, Eq. 1
__global__ void k_na_sweep(int32_t n, const int64_t* __restrict__ in_off, const int32_t* __restrict__ in_src,
                           const double* __restrict__ r_in, double* __restrict__ r_out, double alpha, double C0,
                           NoAllocScratch* s) {
  int lane = threadIdx.x & 31;
  int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  double dmax = 0.0;
  for (int64_t v = warp; v < n; v += nw) {
    long long sum = 0;
    for (int64_t j = in_off[v] + lane; j < in_off[v + 1]; j += 32) sum += s->contrib[in_src[j]];
    sum = dfpr::warp_sum_ll(sum);
    double r = C0 + alpha * ((double)sum * dfpr::FIX_INV);
    if (lane == 0) {
      r_out[v] = r;
      dmax = fmax(dmax, fabs(r - r_in[v]));
    }
  }
  dmax = dfpr::warp_max(dmax);
  if (lane == 0 && dmax > 0.0) dfpr::atomic_max_nonneg(&s->delta_bits, dmax);
}

__global__ void k_na_delta(const NoAllocScratch* s, double* out) { *out = __longlong_as_double((long long)s->delta_bits); }

// device address of the array on the current device, looked up once per device
cudaError_t na_scratch_ptr(NoAllocScratch** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= NA_MAX_DEV) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(na_mu);
  if (!na_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, na_scratch);
    if (e != cudaSuccess) return e;
    na_addr[dev] = (NoAllocScratch*)p;
  }
  *out = na_addr[dev];
  return cudaSuccess;
}

}  // namespace

extern "C" pr_status pr_sweep_noalloc(int32_t n, const int64_t* in_off, const int32_t* in_src, const int32_t* out_deg,
                                      const double* r_in, double* r_out, double alpha, double* delta_out,
                                      void* stream) {
  if (n < 1 || n > NA_MAX_N) return PR_EINVAL;
  if (!in_off || !in_src || !out_deg || !r_in || !r_out || !delta_out) return PR_EINVAL;
  // the sweep measures each vertex's change against r_in after writing r_out
  if ((const void*)r_out < (const void*)(r_in + n) && (const void*)r_in < (const void*)(r_out + n)) return PR_EINVAL;
  if (!(alpha >= 0.0 && alpha < 1.0)) return PR_EINVAL;
  NoAllocScratch* s = nullptr;
  if (na_scratch_ptr(&s) != cudaSuccess) return PR_ECUDA;
  cudaStream_t st = (cudaStream_t)stream;
  int grid = dfpr::grid_for(n, 256);
  dfpr::note_launch();
  k_na_contrib<<<grid, 256, 0, st>>>(n, r_in, out_deg, s);
  int wgrid = dfpr::grid_for((int64_t)n * 32, 256);
  dfpr::note_launch();
  k_na_sweep<<<wgrid, 256, 0, st>>>(n, in_off, in_src, r_in, r_out, alpha, (1.0 - alpha) / (double)n, s);
  dfpr::note_launch();
  k_na_delta<<<1, 1, 0, st>>>(s, delta_out);
  return cudaGetLastError() == cudaSuccess ? PR_OK : PR_ECUDA;
}
