// prim.cu -- scan, radix sort, compaction and fills (see prim.cuh).
#include <atomic>
#include <mutex>
#include "prim.cuh"

namespace dfpr {

static std::atomic<unsigned long long> g_launches{0};
void note_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
void note_launches(unsigned long long k) { g_launches.fetch_add(k, std::memory_order_relaxed); }
unsigned long long launches_so_far() { return g_launches.load(std::memory_order_relaxed); }

// allocations until the injected failure (0: none armed)
static std::atomic<long long> g_fail_in{0};

void arm_alloc_failure(long long k) { g_fail_in.store(k > 0 ? k : 0); }

cudaError_t dev_malloc_raw(void** p, size_t bytes) {
  if (g_fail_in.load(std::memory_order_relaxed) > 0 && g_fail_in.fetch_sub(1) == 1) {
    *p = nullptr;
    return cudaErrorMemoryAllocation;
  }
  return cudaMalloc(p, bytes);
}

static int g_sms = 0;

int num_sms() {
  if (g_sms == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&g_sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || g_sms <= 0) g_sms = 152;
  }
  return g_sms;
}

int grid_for(int64_t n, int block) {
  int64_t want = cdiv(n > 0 ? n : 1, block);
  int64_t cap = (int64_t)num_sms() * 16;
  return (int)(want < cap ? want : cap);
}

// ================================================================== scan

constexpr int SC_THREADS = 256;
constexpr int SC_ITEMS = 8;
constexpr int SC_CHUNK = SC_THREADS * SC_ITEMS;  // 2048

int64_t scan_tmp_elems(int64_t n) { return cdiv(n > 0 ? n : 1, SC_CHUNK) + 1; }

// inclusive block scan of one value per thread; returns the inclusive prefix,
// *total receives the block total
template <typename T>
__device__ __forceinline__ T block_incl_scan(T x, T* total) {
  __shared__ T wsum[SC_THREADS / WARP];
  int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    T y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) wsum[w] = x;
  __syncthreads();
  if (w == 0) {
    T s = lane < SC_THREADS / WARP ? wsum[lane] : T(0);
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      T y = __shfl_up_sync(0xffffffffu, s, o);
      if (lane >= o) s += y;
    }
    if (lane < SC_THREADS / WARP) wsum[lane] = s;
  }
  __syncthreads();
  T add = w > 0 ? wsum[w - 1] : T(0);
  *total = wsum[SC_THREADS / WARP - 1];
  __syncthreads();
  return x + add;
}

template <typename T>
__global__ void k_scan_reduce(const T* __restrict__ in, int64_t n, T* __restrict__ sums) {
  int64_t base = (int64_t)blockIdx.x * SC_CHUNK + (int64_t)threadIdx.x * SC_ITEMS;
  T s = 0;
#pragma unroll
  for (int i = 0; i < SC_ITEMS; i++) {
    int64_t j = base + i;
    if (j < n) s += in[j];
  }
  T tot;
  block_incl_scan<T>(s, &tot);
  if (threadIdx.x == 0) sums[blockIdx.x] = tot;
}

// one block: exclusive scan of sums[0..nb) in place, sums[nb] = total
template <typename T>
__global__ void k_scan_top(T* sums, int64_t nb) {
  T carry = 0;
  for (int64_t base = 0; base < nb; base += SC_THREADS) {
    int64_t j = base + threadIdx.x;
    T x = j < nb ? sums[j] : T(0);
    T tot;
    T inc = block_incl_scan<T>(x, &tot);
    if (j < nb) sums[j] = carry + inc - x;
    carry += tot;
  }
  if (threadIdx.x == 0) sums[nb] = carry;
}

template <typename T>
__global__ void k_scan_down(const T* in, int64_t n, const T* __restrict__ sums, T* out, int64_t nb) {
  int64_t base = (int64_t)blockIdx.x * SC_CHUNK + (int64_t)threadIdx.x * SC_ITEMS;
  T v[SC_ITEMS];
  T s = 0;
#pragma unroll
  for (int i = 0; i < SC_ITEMS; i++) {
    int64_t j = base + i;
    v[i] = j < n ? in[j] : T(0);
    s += v[i];
  }
  T tot;
  T inc = block_incl_scan<T>(s, &tot);
  T run = sums[blockIdx.x] + inc - s;
#pragma unroll
  for (int i = 0; i < SC_ITEMS; i++) {
    int64_t j = base + i;
    if (j < n) out[j] = run;
    run += v[i];
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) out[n] = sums[nb];
}

template <typename T>
cudaError_t scan_excl(const T* in, T* out, int64_t n, T* tmp, cudaStream_t s) {
  int64_t nb = cdiv(n > 0 ? n : 1, SC_CHUNK);
  if (n == 0) return cudaMemsetAsync(out, 0, sizeof(T), s);
  note_launch(); k_scan_reduce<T><<<(unsigned)nb, SC_THREADS, 0, s>>>(in, n, tmp);
  note_launch(); k_scan_top<T><<<1, SC_THREADS, 0, s>>>(tmp, nb);
  note_launch(); k_scan_down<T><<<(unsigned)nb, SC_THREADS, 0, s>>>(in, n, tmp, out, nb);
  return cudaGetLastError();
}

template cudaError_t scan_excl<int32_t>(const int32_t*, int32_t*, int64_t, int32_t*, cudaStream_t);
template cudaError_t scan_excl<int64_t>(const int64_t*, int64_t*, int64_t, int64_t*, cudaStream_t);

// ================================================================== radix sort

constexpr int RS_THREADS = 512;
constexpr int RS_WARPS = RS_THREADS / WARP;
constexpr int RS_ITEMS = 16;
constexpr int RS_KPW = WARP * RS_ITEMS;       // keys per warp
constexpr int RS_TILE = RS_WARPS * RS_KPW;    // 8192 keys per tile
// digits of RS_BITS bits: the 2 x 25-bit edge keys of a 2^25-vertex graph
// take 5 passes instead of the 7 of 8-bit digits
constexpr int RS_BITS = 10;
constexpr int RS_BINS = 1 << RS_BITS;

static int64_t rs_tiles(int64_t n) { return cdiv(n > 0 ? n : 1, RS_TILE); }

size_t radix_tmp_bytes(int64_t n) {
  int64_t cnt = (int64_t)RS_BINS * rs_tiles(n);
  return sizeof(int32_t) * (size_t)(cnt + 1 + scan_tmp_elems(cnt));
}

__global__ void __launch_bounds__(RS_THREADS) k_rs_hist(const uint64_t* __restrict__ keys, int64_t n, int shift,
                                                        int32_t* __restrict__ counts, int64_t ntiles) {
  __shared__ int hist[RS_BINS];
  for (int i = threadIdx.x; i < RS_BINS; i += RS_THREADS) hist[i] = 0;
  __syncthreads();
  int64_t base = (int64_t)blockIdx.x * RS_TILE;
  for (int i = threadIdx.x; i < RS_TILE; i += RS_THREADS) {
    int64_t j = base + i;
    if (j < n) atomicAdd(&hist[(int)((keys[j] >> shift) & (RS_BINS - 1))], 1);
  }
  __syncthreads();
  for (int d = threadIdx.x; d < RS_BINS; d += RS_THREADS) counts[(int64_t)d * ntiles + blockIdx.x] = hist[d];
}

// stable scatter: a warp owns a contiguous run of RS_KPW keys of the tile and
// ranks its keys item by item, so (warp, item, lane) order is input order.
// The tile's keys are first placed in shared memory in digit order (each at
// its position among the tile's keys of its digit), then written out by
// consecutive threads, so the keys of one digit leave as one coalesced run
// instead of each warp's 32 keys going to up to 32 places.
// dynamic shared memory of k_rs_scatter: the staged tile, the per-warp digit
// counts and the digit starts
constexpr size_t RS_STAGE_BYTES =
    sizeof(uint64_t) * RS_TILE + sizeof(int) * (size_t)RS_WARPS * RS_BINS + sizeof(int) * (size_t)RS_BINS;

__global__ void __launch_bounds__(RS_THREADS) k_rs_scatter(const uint64_t* __restrict__ keys, uint64_t* __restrict__ out,
                                                           int64_t n, int shift, const int32_t* __restrict__ offs,
                                                           int64_t ntiles) {
  extern __shared__ uint64_t stage[];   // RS_TILE keys, then wcnt and dstart
  int (*wcnt)[RS_BINS] = reinterpret_cast<int (*)[RS_BINS]>(stage + RS_TILE);
  int* dstart = reinterpret_cast<int*>(stage + RS_TILE) + RS_WARPS * RS_BINS;   // first position of each digit
  int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int i = threadIdx.x; i < RS_WARPS * RS_BINS; i += RS_THREADS) (&wcnt[0][0])[i] = 0;
  __syncthreads();
  const int64_t tile0 = (int64_t)blockIdx.x * RS_TILE;
  int64_t base = tile0 + (int64_t)w * RS_KPW;
  uint64_t k[RS_ITEMS];
  int rank[RS_ITEMS];
  unsigned lt = lanemask_lt();
#pragma unroll
  for (int i = 0; i < RS_ITEMS; i++) {
    int64_t j = base + i * WARP + lane;
    bool valid = j < n;
    k[i] = valid ? keys[j] : 0;
    int d = valid ? (int)((k[i] >> shift) & (RS_BINS - 1)) : RS_BINS;
    unsigned peers = __match_any_sync(0xffffffffu, d);
    int before = valid ? wcnt[w][d] : 0;
    rank[i] = before + __popc(peers & lt);
    __syncwarp();
    if (valid && lane == __ffs(peers) - 1) wcnt[w][d] = before + __popc(peers);
    __syncwarp();
  }
  __syncthreads();
  // per digit: the warps' counts turned into offsets within the digit, and
  // the digit's total
  for (int d = threadIdx.x; d < RS_BINS; d += RS_THREADS) {
    int run = 0;
    for (int ww = 0; ww < RS_WARPS; ww++) {
      int t = wcnt[ww][d];
      wcnt[ww][d] = run;
      run += t;
    }
    dstart[d] = run;
  }
  __syncthreads();
  // exclusive scan of the digit totals by warp 0 (RS_BINS / 32 digits per lane)
  if (w == 0) {
    constexpr int PER = RS_BINS / WARP;
    int sum = 0;
    for (int q = 0; q < PER; q++) sum += dstart[lane * PER + q];
    int incl = sum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int t = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += t;
    }
    int run = incl - sum;
    for (int q = 0; q < PER; q++) {
      const int v = dstart[lane * PER + q];
      dstart[lane * PER + q] = run;
      run += v;
    }
  }
  __syncthreads();
#pragma unroll
  for (int i = 0; i < RS_ITEMS; i++) {
    int64_t j = base + i * WARP + lane;
    if (j < n) {
      int d = (int)((k[i] >> shift) & (RS_BINS - 1));
      stage[dstart[d] + wcnt[w][d] + rank[i]] = k[i];
    }
  }
  __syncthreads();
  const int valid_keys = (int)(n - tile0 < RS_TILE ? n - tile0 : RS_TILE);
  for (int t = threadIdx.x; t < valid_keys; t += RS_THREADS) {
    const uint64_t key = stage[t];
    const int d = (int)((key >> shift) & (RS_BINS - 1));
    out[(int64_t)offs[(int64_t)d * ntiles + blockIdx.x] + (t - dstart[d])] = key;
  }
}

cudaError_t radix_sort_u64(uint64_t* keys, uint64_t* alt, int64_t n, int nbits, void* tmp, cudaStream_t s) {
  if (n <= 1 || nbits <= 0) return cudaSuccess;
  if (n >= (int64_t(1) << 31)) return cudaErrorInvalidValue;
  static std::once_flag smem_set;
  static cudaError_t smem_err = cudaSuccess;
  std::call_once(smem_set, [] {
    smem_err = cudaFuncSetAttribute(k_rs_scatter, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)RS_STAGE_BYTES);
  });
  if (smem_err != cudaSuccess) return smem_err;
  int64_t ntiles = rs_tiles(n);
  int64_t cnt = (int64_t)RS_BINS * ntiles;
  int32_t* counts = (int32_t*)tmp;
  int32_t* scratch = counts + cnt + 1;
  uint64_t* src = keys;
  uint64_t* dst = alt;
  for (int shift = 0; shift < nbits; shift += RS_BITS) {
    note_launch(); k_rs_hist<<<(unsigned)ntiles, RS_THREADS, 0, s>>>(src, n, shift, counts, ntiles);
    cudaError_t e = scan_excl<int32_t>(counts, counts, cnt, scratch, s);
    if (e != cudaSuccess) return e;
    note_launch(); k_rs_scatter<<<(unsigned)ntiles, RS_THREADS, RS_STAGE_BYTES, s>>>(src, dst, n, shift, counts, ntiles);
    uint64_t* t = src;
    src = dst;
    dst = t;
  }
  if (src != keys) return cudaMemcpyAsync(keys, src, sizeof(uint64_t) * (size_t)n, cudaMemcpyDeviceToDevice, s);
  return cudaGetLastError();
}

// ================================================================== compaction

size_t compact_tmp_bytes(int64_t n) { return sizeof(int64_t) * (size_t)(n + 1 + scan_tmp_elems(n)); }

__global__ void k_flag_to_i64(const uint8_t* __restrict__ f, int64_t n, int64_t* __restrict__ x) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    x[i] = f[i] ? 1 : 0;
}

__global__ void k_compact_scatter(const uint64_t* __restrict__ in, const uint8_t* __restrict__ f,
                                  const int64_t* __restrict__ pos, int64_t n, uint64_t* __restrict__ out,
                                  int64_t* count_dev) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    if (f[i]) out[pos[i]] = in[i];
  if (blockIdx.x == 0 && threadIdx.x == 0) *count_dev = pos[n];
}

cudaError_t compact_u64(const uint64_t* in, const uint8_t* flag, int64_t n, uint64_t* out, int64_t* count_dev,
                        void* tmp, cudaStream_t s) {
  if (n == 0) return cudaMemsetAsync(count_dev, 0, sizeof(int64_t), s);
  int64_t* pos = (int64_t*)tmp;
  int64_t* scr = pos + n + 1;
  note_launch(); k_flag_to_i64<<<grid_for(n, 256), 256, 0, s>>>(flag, n, pos);
  cudaError_t e = scan_excl<int64_t>(pos, pos, n, scr, s);
  if (e != cudaSuccess) return e;
  note_launch(); k_compact_scatter<<<grid_for(n, 256), 256, 0, s>>>(in, flag, pos, n, out, count_dev);
  return cudaGetLastError();
}

__global__ void k_flag_unique(const uint64_t* __restrict__ k, int64_t n, uint8_t* __restrict__ f) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    f[i] = (i == 0 || k[i] != k[i - 1]) ? 1 : 0;
}

cudaError_t flag_unique_sorted(const uint64_t* k, int64_t n, uint8_t* flag, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  note_launch(); k_flag_unique<<<grid_for(n, 256), 256, 0, s>>>(k, n, flag);
  return cudaGetLastError();
}

// ================================================================== fills

template <typename T>
__global__ void k_fill(T* p, T v, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) p[i] = v;
}
__global__ void k_iota(int32_t* p, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    p[i] = (int32_t)i;
}

cudaError_t fill_i32(int32_t* p, int32_t v, int64_t n, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  note_launch(); k_fill<int32_t><<<grid_for(n, 256), 256, 0, s>>>(p, v, n);
  return cudaGetLastError();
}
cudaError_t fill_i64(int64_t* p, int64_t v, int64_t n, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  note_launch(); k_fill<int64_t><<<grid_for(n, 256), 256, 0, s>>>(p, v, n);
  return cudaGetLastError();
}
cudaError_t iota_i32(int32_t* p, int64_t n, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  note_launch(); k_iota<<<grid_for(n, 256), 256, 0, s>>>(p, n);
  return cudaGetLastError();
}

}  // namespace dfpr
