// synth_cuda.cu -- the generators of synth.c on the GPU, for graphs too large
// to draw on the host (R-MAT scale 25: 2^30 edges).  Same counter-based
// definitions, same integer arithmetic, so equal arguments give equal arrays.
// Holds none of the PageRank arithmetic.
#include <cstdint>
#include <cuda_runtime.h>

namespace {

__device__ __forceinline__ uint64_t mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
  return z ^ (z >> 31);
}

__device__ __forceinline__ uint64_t draw(uint64_t seed, uint64_t stream, uint64_t ctr) {
  return mix64(mix64(seed ^ (stream << 56)) + ctr * 0x9E3779B97F4A7C15ULL);
}

__device__ __forceinline__ uint32_t scale32(uint32_t u, uint32_t range) {
  return (uint32_t)(((uint64_t)u * range) >> 32);
}
__device__ __forceinline__ uint64_t scale64(uint64_t u, uint64_t range) { return __umul64hi(u, range); }

struct PermKeys {
  uint64_t mask, k1, k2, k3;
  int sh;
};

__device__ __forceinline__ uint32_t perm_pow2(uint32_t x, const PermKeys& k) {
  uint64_t y = x;
  y = (y * k.k1) & k.mask;
  y ^= y >> k.sh;
  y = (y + k.k2) & k.mask;
  y = (y * k.k3) & k.mask;
  y ^= y >> k.sh;
  return (uint32_t)y;
}

__global__ void k_rmat(int scale, int64_t m, uint64_t seed, uint64_t t1, uint64_t t2, uint64_t t3, PermKeys pk,
                       int32_t* __restrict__ src, int32_t* __restrict__ dst) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < m; e += (int64_t)gridDim.x * blockDim.x) {
    uint32_t u = 0, v = 0;
    uint64_t w = 0;
    for (int l = 0; l < scale; l++) {
      if ((l & 1) == 0) w = draw(seed, 1, (uint64_t)e * 16 + (uint64_t)(l >> 1));
      uint64_t r = (l & 1) ? (w >> 32) : (w & 0xffffffffULL);
      uint32_t rb, cb;
      if (r < t1) { rb = 0; cb = 0; }
      else if (r < t2) { rb = 0; cb = 1; }
      else if (r < t3) { rb = 1; cb = 0; }
      else { rb = 1; cb = 1; }
      u = (u << 1) | rb;
      v = (v << 1) | cb;
    }
    src[e] = (int32_t)perm_pow2(u, pk);
    dst[e] = (int32_t)perm_pow2(v, pk);
  }
}

__global__ void k_batch(int32_t n, const int32_t* __restrict__ cs, const int32_t* __restrict__ cd, int64_t n_cand,
                        int64_t n_del, int64_t n_ins, uint64_t seed, int32_t* __restrict__ ds, int32_t* __restrict__ dd,
                        int32_t* __restrict__ is, int32_t* __restrict__ id) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n_del + n_ins;
       i += (int64_t)gridDim.x * blockDim.x) {
    if (i < n_del) {
      if (n_cand > 0) {
        uint64_t j = scale64(draw(seed, 3, (uint64_t)i), (uint64_t)n_cand);
        ds[i] = cs[j];
        dd[i] = cd[j];
      }
    } else {
      int64_t k = i - n_del;
      uint64_t w = draw(seed, 2, (uint64_t)k);
      uint32_t u = scale32((uint32_t)(w >> 32), (uint32_t)n);
      uint32_t v = scale32((uint32_t)(w & 0xffffffffULL), (uint32_t)n);
      if (v == u) v = (u + 1) % (uint32_t)n;
      is[k] = (int32_t)u;
      id[k] = (int32_t)v;
    }
  }
}

uint64_t host_mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
  return z ^ (z >> 31);
}
uint64_t host_draw(uint64_t seed, uint64_t stream, uint64_t ctr) {
  return host_mix64(host_mix64(seed ^ (stream << 56)) + ctr * 0x9E3779B97F4A7C15ULL);
}

int grid_for(int64_t n) {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (sms <= 0) sms = 132;
  int64_t want = (n + 255) / 256;
  int64_t cap = (int64_t)sms * 16;
  return (int)(want < 1 ? 1 : (want < cap ? want : cap));
}

}  // namespace

extern "C" int sy_rmat_device(int scale, int64_t m, uint64_t seed, int32_t a, int32_t b, int32_t c, int32_t* src,
                              int32_t* dst, void* stream) {
  if (scale < 1 || scale > 31 || m < 0) return 1;
  PermKeys pk;
  pk.mask = (1ULL << scale) - 1;
  pk.k1 = (host_draw(seed, 7, 0) | 1) & pk.mask;
  pk.k2 = host_draw(seed, 7, 1) & pk.mask;
  pk.k3 = (host_draw(seed, 7, 2) | 1) & pk.mask;
  pk.sh = (scale + 1) / 2;
  uint64_t t1 = ((uint64_t)a << 32) / 10000;
  uint64_t t2 = ((uint64_t)(a + b) << 32) / 10000;
  uint64_t t3 = ((uint64_t)(a + b + c) << 32) / 10000;
  if (m == 0) return 0;
  k_rmat<<<grid_for(m), 256, 0, (cudaStream_t)stream>>>(scale, m, seed, t1, t2, t3, pk, src, dst);
  return cudaGetLastError() == cudaSuccess ? 0 : 2;
}

extern "C" int sy_batch_device(int32_t n, const int32_t* cand_src, const int32_t* cand_dst, int64_t n_cand,
                               int64_t n_del, int64_t n_ins, uint64_t seed, int32_t* del_src, int32_t* del_dst,
                               int32_t* ins_src, int32_t* ins_dst, void* stream) {
  if (n < 1 || n_del < 0 || n_ins < 0) return 1;
  if (n_del + n_ins == 0) return 0;
  k_batch<<<grid_for(n_del + n_ins), 256, 0, (cudaStream_t)stream>>>(n, cand_src, cand_dst, n_cand, n_del, n_ins, seed,
                                                                      del_src, del_dst, ins_src, ins_dst);
  return cudaGetLastError() == cudaSuccess ? 0 : 2;
}
