// common.cuh -- shared definitions of the GB300 DF / DF-P PageRank library.
//
// Data layout in HBM (internal vertex ids, see graph.cu for the relabelling):
//   out-CSR  oo[n+1] int64 row starts (capacity, multiple of 4 slots, so every
//            row starts 16-byte aligned), od[n] int32 out-degree (self-loop
//            included), oc[oo[n]] int32 targets, each row sorted ascending;
//            slots between od[v] and the row's capacity hold SENT (= n).
//   in-CSR   io / id / ic, the same for in-edges (sources sorted ascending).
//   R[n]     FP64 ranks.
//   C[2][n+1] int64 contributions R[u] / |out(u)| in 2^-61 fixed point
//            (C[.][n] = 0, so SENT slots add nothing); two buffers so a full
//            synchronous sweep can write the next contributions while the
//            current ones are still being gathered.
#pragma once
#include <cstdint>
#include <cstddef>
#include <cuda_runtime.h>

namespace dfpr {

// Device allocations of the library go through dev_malloc so that a test can
// make the k-th one fail as if the device were out of memory
// (pr_debug_fail_alloc), with no fault on the GPU.
cudaError_t dev_malloc_raw(void** p, size_t bytes);
void arm_alloc_failure(long long k);
template <class T>
inline cudaError_t dev_malloc(T** p, size_t bytes) {
  return dev_malloc_raw(reinterpret_cast<void**>(p), bytes);
}

// process-wide count of kernel launches made by this library (pr_kernel_launches)
void note_launch();
void note_launches(unsigned long long k);   // kernels run by a CUDA graph launch
unsigned long long launches_so_far();

// fixed-point scale of the contribution sums: value = integer * 2^-FIX_BITS
constexpr int FIX_BITS = 61;
constexpr double FIX_ONE = 2305843009213693952.0;          // 2^61
constexpr double FIX_INV = 1.0 / 2305843009213693952.0;    // 2^-61, exact

constexpr int WARP = 32;

// ---------------------------------------------------------------- error codes
// (mirrors pr_status in include/dfpr.h; kept here so device code needs no C header)
enum Status : int { OK = 0, EINVAL_ = 1, ERANGE_ = 2, ENOMEM_ = 3, ENORANKS_ = 4, ECUDA_ = 5, ETIMEOUT_ = 6 };

// ---------------------------------------------------------------- small device helpers

__device__ __forceinline__ unsigned lanemask_lt() {
  unsigned r;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(r));
  return r;
}

__device__ __forceinline__ int lane_id() { return threadIdx.x & (WARP - 1); }

// Append `want` (per lane) items to a global counter with one atomic per warp.
// Returns this lane's slot (valid only where want).
__device__ __forceinline__ int warp_append(int* counter, bool want) {
  unsigned act = __activemask();
  unsigned m = __ballot_sync(act, want);
  if (m == 0) return -1;
  int leader = __ffs(m) - 1;
  int base = 0;
  if (lane_id() == leader) base = atomicAdd(counter, __popc(m));
  base = __shfl_sync(act, base, leader);
  return base + __popc(m & lanemask_lt());
}

// test-and-set one bit; true if this call set it
__device__ __forceinline__ bool bit_tas(uint32_t* bits, int v) {
  uint32_t mask = 1u << (v & 31);
  uint32_t* w = bits + (v >> 5);
  if (__ldcg(w) & mask) return false;
  return (atomicOr(w, mask) & mask) == 0;
}

__device__ __forceinline__ bool bit_get(const uint32_t* bits, int v) {
  return (__ldcg(bits + (v >> 5)) >> (v & 31)) & 1u;
}

// atomic max of a non-negative double through its bit pattern
__device__ __forceinline__ void atomic_max_nonneg(unsigned long long* p, double x) {
  atomicMax(p, (unsigned long long)__double_as_longlong(x));
}

__device__ __forceinline__ double warp_max(double x) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x = fmax(x, __shfl_xor_sync(0xffffffffu, x, o));
  return x;
}

__device__ __forceinline__ long long warp_sum_ll(long long x) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
  return x;
}

__host__ __device__ __forceinline__ int64_t round4(int64_t x) { return (x + 3) & ~(int64_t)3; }
__host__ __device__ __forceinline__ int64_t cdiv(int64_t a, int64_t b) { return (a + b - 1) / b; }

// convert rank r of a vertex with out-degree d into its fixed-point contribution
__device__ __forceinline__ long long to_fix(double r, double inv_d_scaled) {
  return __double2ll_rn(r * inv_d_scaled);
}

}  // namespace dfpr
