// frontier.cu -- initial marking (Alg. 1), reachability helpers (Sec. 3.3.2),
// per-iteration bookkeeping, contribution refresh.
#include "frontier.cuh"
#include "sweep.cuh"
#include "prim.cuh"

namespace dfpr {

#define GRID_STRIDE(i, n) \
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < (n); i += (int64_t)gridDim.x * blockDim.x)

// The loops below call warp_append, so every lane of a warp must run the same
// number of trips: they iterate to a warp-uniform bound and mask the tail.
#define WARP_UNIFORM_STRIDE(i, n)                                                                     \
  for (int64_t i##_base = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) & ~(int64_t)31,            \
                    i = i##_base + (threadIdx.x & 31);                                                \
       i##_base < (n); i##_base += (int64_t)gridDim.x * blockDim.x, i = i##_base + (threadIdx.x & 31))

__global__ void k_mark_sources(const uint64_t* __restrict__ a, int64_t na, const uint64_t* __restrict__ b, int64_t nb,
                               int bits, uint32_t* seen, int32_t* list, int32_t* count) {
  int64_t tot = na + nb;
  WARP_UNIFORM_STRIDE(i, tot) {
    bool add = false;
    int32_t u = 0;
    if (i < tot) {
      uint64_t key = i < na ? a[i] : b[i - na];
      u = (int32_t)(key >> bits);
      add = bit_tas(seen, u);
    }
    int slot = warp_append(count, add);
    if (add) list[slot] = u;
  }
}

cudaError_t launch_mark_sources(const uint64_t* a, int64_t na, const uint64_t* b, int64_t nb, int id_bits,
                                uint32_t* seen, int32_t* list, int32_t* count, cudaStream_t s) {
  if (na + nb == 0) return cudaSuccess;
  note_launch(); k_mark_sources<<<grid_for(na + nb, 256), 256, 0, s>>>(a, na, b, nb, id_bits, seen, list, count);
  return cudaGetLastError();
}

__global__ void k_mark_targets(const uint64_t* __restrict__ d, int64_t nd, int bits, uint32_t* bm, uint32_t* ever,
                               int32_t* list, int32_t* count) {
  uint64_t mask = (1ull << bits) - 1;
  WARP_UNIFORM_STRIDE(i, nd) {
    bool add = false;
    int32_t w = 0;
    if (i < nd) {
      w = (int32_t)(d[i] & mask);
      add = bit_tas(bm, w);
    }
    int slot = warp_append(count, add);
    if (add) {
      list[slot] = w;
      if (ever) atomicOr(ever + (w >> 5), 1u << (w & 31));
    }
  }
}

cudaError_t launch_mark_targets(const uint64_t* d, int64_t nd, int id_bits, uint32_t* bits, uint32_t* ever,
                                int32_t* list, int32_t* count, cudaStream_t s) {
  if (nd == 0) return cudaSuccess;
  note_launch(); k_mark_targets<<<grid_for(nd, 256), 256, 0, s>>>(d, nd, id_bits, bits, ever, list, count);
  return cudaGetLastError();
}

__global__ void k_follow_edges(const uint64_t* __restrict__ d, int64_t nd, int bits, uint32_t* vis, int32_t* list,
                               int32_t* count) {
  uint64_t mask = (1ull << bits) - 1;
  WARP_UNIFORM_STRIDE(i, nd) {
    bool add = false;
    int32_t w = 0;
    if (i < nd) {
      int32_t u = (int32_t)(d[i] >> bits);
      w = (int32_t)(d[i] & mask);
      add = bit_get(vis, u) && bit_tas(vis, w);
    }
    int slot = warp_append(count, add);
    if (add) list[slot] = w;
  }
}

cudaError_t launch_follow_edges(const uint64_t* d, int64_t nd, int id_bits, uint32_t* vis, int32_t* list,
                                int32_t* count, cudaStream_t s) {
  if (nd == 0) return cudaSuccess;
  note_launch(); k_follow_edges<<<grid_for(nd, 256), 256, 0, s>>>(d, nd, id_bits, vis, list, count);
  return cudaGetLastError();
}

__global__ void k_source_bits(const uint64_t* __restrict__ d, int64_t nd, int bits, uint32_t* bm) {
  GRID_STRIDE(i, nd) {
    int32_t u = (int32_t)(d[i] >> bits);
    atomicOr(bm + (u >> 5), 1u << (u & 31));
  }
}

cudaError_t launch_source_bits(const uint64_t* d, int64_t nd, int id_bits, uint32_t* bits, cudaStream_t s) {
  if (nd == 0) return cudaSuccess;
  note_launch(); k_source_bits<<<grid_for(nd, 256), 256, 0, s>>>(d, nd, id_bits, bits);
  return cudaGetLastError();
}

// ---- bitset -> ascending list

int64_t bits_to_list_tmp(int32_t n) {
  int64_t words = cdiv((int64_t)n, 32);
  return words + 1 + scan_tmp_elems(words);
}

__global__ void k_word_pop(const uint32_t* __restrict__ a, const uint32_t* __restrict__ b, int64_t words, int32_t n,
                           int32_t* __restrict__ pc) {
  GRID_STRIDE(w, words) {
    uint32_t x = a[w] | (b ? b[w] : 0u);
    int64_t hi = (w + 1) * 32;
    if (hi > n) x &= (n - w * 32 >= 32) ? 0xffffffffu : ((1u << (n - w * 32)) - 1u);
    pc[w] = __popc(x);
  }
}

__global__ void k_word_emit(const uint32_t* __restrict__ a, const uint32_t* __restrict__ b, int64_t words, int32_t n,
                            const int32_t* __restrict__ pos, int32_t* __restrict__ list, int32_t* count) {
  GRID_STRIDE(w, words) {
    uint32_t x = a[w] | (b ? b[w] : 0u);
    int64_t hi = (w + 1) * 32;
    if (hi > n) x &= (n - w * 32 >= 32) ? 0xffffffffu : ((1u << (n - w * 32)) - 1u);
    int32_t p = pos[w];
    while (x) {
      int bit = __ffs(x) - 1;
      list[p++] = (int32_t)(w * 32 + bit);
      x &= x - 1;
    }
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) *count = pos[words];
}

cudaError_t launch_bits_to_list(const uint32_t* a, const uint32_t* b, int32_t n, int32_t* list, int32_t* count,
                                int32_t* tmp, cudaStream_t s) {
  int64_t words = cdiv((int64_t)n, 32);
  int32_t* pc = tmp;
  int32_t* scr = tmp + words + 1;
  note_launch(); k_word_pop<<<grid_for(words, 256), 256, 0, s>>>(a, b, words, n, pc);
  cudaError_t e = scan_excl<int32_t>(pc, pc, words, scr, s);
  if (e != cudaSuccess) return e;
  note_launch(); k_word_emit<<<grid_for(words, 256), 256, 0, s>>>(a, b, words, n, pc, list, count);
  return cudaGetLastError();
}

__global__ void k_popcount(const uint32_t* __restrict__ a, int64_t words, long long* out) {
  long long c = 0;
  GRID_STRIDE(w, words) c += __popc(a[w]);
  c = warp_sum_ll(c);
  if ((threadIdx.x & 31) == 0 && c) atomicAdd((unsigned long long*)out, (unsigned long long)c);
}

// out = a | b, word by word
__global__ void k_bits_or(const uint32_t* __restrict__ a, const uint32_t* __restrict__ b, uint32_t* __restrict__ out,
                          int64_t words) {
  GRID_STRIDE(w, words) out[w] = a[w] | b[w];
}

cudaError_t launch_bits_or(const uint32_t* a, const uint32_t* b, uint32_t* out, int64_t words, cudaStream_t s) {
  if (words == 0) return cudaSuccess;
  note_launch(); k_bits_or<<<grid_for(words, 256), 256, 0, s>>>(a, b, out, words);
  return cudaGetLastError();
}

cudaError_t launch_popcount(const uint32_t* a, int64_t words, long long* out, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(out, 0, sizeof(long long), s);
  if (e != cudaSuccess) return e;
  if (words == 0) return cudaSuccess;
  note_launch(); k_popcount<<<grid_for(words, 256), 256, 0, s>>>(a, words, out);
  return cudaGetLastError();
}

// ---- bookkeeping

__global__ void k_control(Ctl* ctl, int frontier) {
  ctl->dR_last = ctl->dR;
  ctl->dR = 0ull;
  ctl->iter += 1;
  if (frontier) {
    int c = ctl->cur;
    ctl->count[c] = 0;
    ctl->cur = 1 - c;
    ctl->nexp_last = ctl->nexp;
    ctl->nexp = 0;
  }
}

cudaError_t launch_control(Ctl* ctl, int frontier, cudaStream_t s) {
  note_launch(); k_control<<<1, 1, 0, s>>>(ctl, frontier);
  return cudaGetLastError();
}

__global__ void k_tables(double* tab_sc, double2* tab_ab, double alpha, int32_t n) {
  GRID_STRIDE(d, TAB) {
    if (d == 0) {
      tab_sc[0] = 0.0;
      if (tab_ab) tab_ab[0] = make_double2(0.0, 0.0);
    } else {
      tab_sc[d] = FIX_ONE / (double)d;
      if (tab_ab) tab_ab[d] = closed_coeffs(alpha, n, (int32_t)d);
    }
  }
}

cudaError_t launch_tables(double* tab_sc, double2* tab_ab, double alpha, int32_t n, cudaStream_t s) {
  note_launch(); k_tables<<<cdiv(TAB, 256), 256, 0, s>>>(tab_sc, tab_ab, alpha, n);
  return cudaGetLastError();
}

__device__ __forceinline__ long long contrib_of(double r, int32_t d, const double* tab_sc) {
  double sc = d < TAB ? tab_sc[d] : FIX_ONE / (double)d;
  return __double2ll_rn(r * sc);
}

__global__ void k_init_uniform(double* R, long long* C, const int32_t* odeg, const double* tab_sc, int32_t n) {
  double r = 1.0 / (double)n;
  GRID_STRIDE(v, n) {
    R[v] = r;
    C[v] = contrib_of(r, odeg[v], tab_sc);
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) C[n] = 0;
}

cudaError_t launch_init_uniform(double* R, long long* C, const int32_t* odeg, const double* tab_sc, int32_t n,
                                cudaStream_t s) {
  note_launch(); k_init_uniform<<<grid_for(n, 256), 256, 0, s>>>(R, C, odeg, tab_sc, n);
  return cudaGetLastError();
}

__global__ void k_contrib_all(const double* R, long long* C, const int32_t* odeg, const double* tab_sc, int32_t n) {
  GRID_STRIDE(v, n) C[v] = contrib_of(R[v], odeg[v], tab_sc);
  if (blockIdx.x == 0 && threadIdx.x == 0) C[n] = 0;
}

cudaError_t launch_contrib_all(const double* R, long long* C, const int32_t* odeg, const double* tab_sc, int32_t n,
                               cudaStream_t s) {
  note_launch(); k_contrib_all<<<grid_for(n, 256), 256, 0, s>>>(R, C, odeg, tab_sc, n);
  return cudaGetLastError();
}

__global__ void k_contrib_list(const int32_t* list, const int32_t* count, const double* R, long long* C,
                               const int32_t* odeg, const double* tab_sc) {
  int32_t K = *count;
  GRID_STRIDE(k, K) {
    int32_t v = list[k];
    C[v] = contrib_of(R[v], odeg[v], tab_sc);
  }
}

cudaError_t launch_contrib_list(const int32_t* list, const int32_t* count, const double* R, long long* C,
                                const int32_t* odeg, const double* tab_sc, int32_t n, cudaStream_t s) {
  note_launch(); k_contrib_list<<<grid_for(n, 256), 256, 0, s>>>(list, count, R, C, odeg, tab_sc);
  return cudaGetLastError();
}

__global__ void k_gather_f64(const double* __restrict__ in, const int32_t* __restrict__ idx, double* __restrict__ out,
                             int32_t n) {
  GRID_STRIDE(i, n) out[i] = in[idx[i]];
}
__global__ void k_scatter_f64(const double* __restrict__ in, const int32_t* __restrict__ idx, double* __restrict__ out,
                              int32_t n) {
  GRID_STRIDE(i, n) out[idx[i]] = in[i];
}

cudaError_t launch_gather_f64(const double* in, const int32_t* idx, double* out, int32_t n, cudaStream_t s) {
  note_launch(); k_gather_f64<<<grid_for(n, 256), 256, 0, s>>>(in, idx, out, n);
  return cudaGetLastError();
}
cudaError_t launch_scatter_f64(const double* in, const int32_t* idx, double* out, int32_t n, cudaStream_t s) {
  note_launch(); k_scatter_f64<<<grid_for(n, 256), 256, 0, s>>>(in, idx, out, n);
  return cudaGetLastError();
}

}  // namespace dfpr
