// sweep.cu -- pull rank sweep with the fused DF / DF-P epilogue, frontier
// expansion, commit, and the list scan that balances them.
//
// Every kernel here walks a "list" of vertices flattened into 16-byte quads of
// their CSR rows (4 int32 ids per quad).  A tile is 1024 consecutive quads of
// that flattened space, so work is balanced by edges, not by vertices: a
// vertex with 10^6 in-edges spans ~245 tiles, a run of degree-1 vertices shares
// one.  Inside a tile each thread takes quads tid, tid+256, ... (lanes read
// consecutive quads of a row: coalesced 128-bit loads), finds the quad's owner
// by binary search over the tile's item starts in shared memory, gathers the
// four contributions and reduces them per owner with a segmented warp
// reduction.  Owners whose row crosses a tile edge add their partial sum to a
// global accumulator; the tile that completes the row (ticket counter) runs the
// epilogue.  Contributions are 2^-61 fixed-point integers, so every partial
// order of additions gives the same bits: the result does not depend on the
// tiling, and integer adds run on GB300's integer pipes (FP64 adds are ~36x
// slower there).
#include <climits>
#include "sweep.cuh"
#include "prim.cuh"

namespace dfpr {

// ------------------------------------------------------------------ helpers

template <typename T>
__device__ __forceinline__ T block_incl_scan256(T x, T* total, T* wsum /* >= 8 */) {
  int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    T y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) wsum[w] = x;
  __syncthreads();
  if (w == 0) {
    T s = lane < 8 ? wsum[lane] : T(0);
#pragma unroll
    for (int o = 1; o < 8; o <<= 1) {
      T y = __shfl_up_sync(0xffffffffu, s, o);
      if (lane >= o) s += y;
    }
    if (lane < 8) wsum[lane] = s;
  }
  __syncthreads();
  T add = w > 0 ? wsum[w - 1] : T(0);
  *total = wsum[7];
  __syncthreads();
  return x + add;
}

__device__ __forceinline__ void block_flush_stats(double dmax, long long edges, long long verts, Ctl* ctl) {
  __shared__ double s_d[SW_THREADS / WARP];
  __shared__ long long s_e[SW_THREADS / WARP], s_v[SW_THREADS / WARP];
  dmax = warp_max(dmax);
  edges = warp_sum_ll(edges);
  verts = warp_sum_ll(verts);
  int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (lane == 0) {
    s_d[w] = dmax;
    s_e[w] = edges;
    s_v[w] = verts;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double d = 0;
    long long e = 0, v = 0;
    for (int i = 0; i < SW_THREADS / WARP; i++) {
      d = fmax(d, s_d[i]);
      e += s_e[i];
      v += s_v[i];
    }
    if (d > 0) atomic_max_nonneg(&ctl->dR, d);
    if (e) atomicAdd((unsigned long long*)&ctl->edges, (unsigned long long)e);
    if (v) atomicAdd((unsigned long long*)&ctl->verts, (unsigned long long)v);
  }
}

// owner of local quad q: largest i in [0, nitems) with lstart[i] <= q (lstart[0] == 0)
__device__ __forceinline__ int tile_owner(const int32_t* lstart, int nitems, int q) {
  int lo = 0, hi = nitems - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (lstart[mid] <= q) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

// ------------------------------------------------------------------ sweep

template <int MODE>
__device__ __forceinline__ void finalize(const SweepParams& p, int32_t k, int32_t v, long long sum, double& dmax,
                                         long long& edges, long long& verts) {
  double Rv = p.R[v];
  int32_t d = p.odeg[v];
  double r;
  if (MODE == SWEEP_DFP) {
    // Eq. 2: K = sum over in-neighbours minus the vertex's own self-loop term,
    // r = (C0 + alpha K) / (1 - alpha/d); the self term is removed exactly in
    // fixed point
    long long K = sum - p.Ccur[v];
    double Kd = (double)K * FIX_INV;
    double f = d < TAB ? p.tab_cl[d] : 1.0 / (1.0 - p.alpha / (double)d);
    r = f * (p.C0 + p.alpha * Kd);
  } else {
    // Eq. 1: r = C0 + alpha c
    double c = (double)sum * FIX_INV;
    r = p.C0 + p.alpha * c;
  }
  double dr = fabs(r - Rv);
  dmax = fmax(dmax, dr);
  edges += p.ideg[v];
  verts += 1;
  if (MODE == SWEEP_FULL) {
    p.R[v] = r;
    double sc = d < TAB ? p.tab_sc[d] : FIX_ONE / (double)d;
    p.Cnext[v] = __double2ll_rn(r * sc);
    return;
  }
  p.rnew[k] = r;
  if (MODE == SWEEP_DF || MODE == SWEEP_DFP) {
    // Alg. 1: prune when dr / max(r, R[v]) <= tau_p (DF-P), expand when it is
    // > tau_f; both compared without the division, in FP64
    double mr = fmax(r, Rv);
    bool stay = (MODE == SWEEP_DF) || !(dr <= p.tau_p * mr);
    bool expand = dr > p.tau_f * mr;
    bool add = stay && bit_tas(p.bits_next, v);
    int slot = warp_append(p.cnt_next, add);
    if (add) {
      p.wl_next[slot] = v;
      if (p.ever) atomicOr(p.ever + (v >> 5), 1u << (v & 31));
    }
    int xs = warp_append(p.cnt_x, expand);
    if (expand) p.xl[xs] = v;
  }
}

template <int MODE>
__global__ void __launch_bounds__(SW_THREADS) k_sweep(SweepParams p) {
  __shared__ int32_t s_lstart[SW_MAX_ITEMS + 1];
  __shared__ long long s_adj[SW_MAX_ITEMS];
  __shared__ long long s_acc[SW_MAX_ITEMS];
  __shared__ int32_t s_v[SW_MAX_ITEMS];
  __shared__ int32_t s_nt[SW_MAX_ITEMS];

  constexpr bool ident = MODE == SWEEP_FULL;
  const int64_t ntiles = ident ? p.ntiles_host : *p.ntiles_dev;
  const int32_t K = ident ? p.n : *p.count;
  const int64_t Qtot = ident ? (p.ioff[p.n] >> 2) : p.qs[K];
  double dmax = 0.0;
  long long edges = 0, verts = 0;
  const int lane = threadIdx.x & 31;

  for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const int64_t T0 = t * SW_TILE_Q;
    const int64_t T1 = min(T0 + (int64_t)SW_TILE_Q, Qtot);
    const int32_t k_lo = p.tfirst[t];
    int32_t k_hi = p.tfirst[t + 1];
    if (k_hi > K - 1) k_hi = K - 1;
    int nitems = k_hi - k_lo + 1;
    if (nitems > SW_MAX_ITEMS || nitems < 1) {   // cannot happen for a well-formed tile table
      if (threadIdx.x == 0) p.ctl->status = 1;
      break;
    }
    for (int i = threadIdx.x; i < nitems; i += SW_THREADS) {
      int32_t k = k_lo + i;
      int32_t v = ident ? k : p.list[k];
      int64_t q0 = ident ? (p.ioff[v] >> 2) : p.qs[k];
      int64_t q1 = ident ? (p.ioff[v + 1] >> 2) : p.qs[k + 1];
      s_v[i] = v;
      s_lstart[i] = (int32_t)(max(q0, T0) - T0);
      s_adj[i] = p.ioff[v] - 4 * q0 + 4 * T0;
      int nt;
      if (q0 >= T1 || q1 <= T0) nt = -1;
      else if (q0 >= T0 && q1 <= T1) nt = 0;
      else nt = (int)((q1 - 1) / SW_TILE_Q - q0 / SW_TILE_Q + 1);
      s_nt[i] = nt;
      s_acc[i] = 0;
    }
    if (threadIdx.x == 0) s_lstart[nitems] = INT_MAX;
    __syncthreads();
    const int nq = (int)(T1 - T0);
#pragma unroll
    for (int j = 0; j < SW_QPT; j++) {
      const int q = threadIdx.x + j * SW_THREADS;
      const bool valid = q < nq;
      int owner = SW_MAX_ITEMS;
      long long sum = 0;
      if (valid) {
        owner = tile_owner(s_lstart, nitems, q);
        int4 c = __ldg(reinterpret_cast<const int4*>(p.icol + s_adj[owner] + 4 * (int64_t)q));
        sum = __ldg(p.Ccur + c.x) + __ldg(p.Ccur + c.y) + __ldg(p.Ccur + c.z) + __ldg(p.Ccur + c.w);
      }
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        long long os = __shfl_down_sync(0xffffffffu, sum, o);
        int oo = __shfl_down_sync(0xffffffffu, owner, o);
        if (lane + o < 32 && oo == owner) sum += os;
      }
      int prev = __shfl_up_sync(0xffffffffu, owner, 1);
      if (valid && (lane == 0 || prev != owner))
        atomicAdd(reinterpret_cast<unsigned long long*>(&s_acc[owner]), (unsigned long long)sum);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < nitems; i += SW_THREADS) {
      int nt = s_nt[i];
      if (nt < 0) continue;
      int32_t k = k_lo + i;
      long long total = s_acc[i];
      if (nt > 0) {
        atomicAdd(reinterpret_cast<unsigned long long*>(&p.gacc[k]), (unsigned long long)total);
        __threadfence();
        int ticket = atomicAdd(&p.gcnt[k], 1);
        if (ticket != nt - 1) continue;
        __threadfence();
        total = (long long)atomicExch(reinterpret_cast<unsigned long long*>(&p.gacc[k]), 0ull);
        p.gcnt[k] = 0;
      }
      finalize<MODE>(p, k, s_v[i], total, dmax, edges, verts);
    }
    __syncthreads();
  }
  block_flush_stats(dmax, edges, verts, p.ctl);
}

cudaError_t launch_sweep(int mode, const SweepParams& p, cudaStream_t s) {
  int grid = num_sms() * 4;
  if (mode == SWEEP_FULL) {
    int64_t want = p.ntiles_host > 0 ? p.ntiles_host : 1;
    if (want < grid) grid = (int)want;
  }
  switch (mode) {
    case SWEEP_FULL: note_launch(); k_sweep<SWEEP_FULL><<<grid, SW_THREADS, 0, s>>>(p); break;
    case SWEEP_LIST: note_launch(); k_sweep<SWEEP_LIST><<<grid, SW_THREADS, 0, s>>>(p); break;
    case SWEEP_DF: note_launch(); k_sweep<SWEEP_DF><<<grid, SW_THREADS, 0, s>>>(p); break;
    case SWEEP_DFP: note_launch(); k_sweep<SWEEP_DFP><<<grid, SW_THREADS, 0, s>>>(p); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

// ------------------------------------------------------------------ list scan

constexpr int LS_THREADS = 256;
constexpr int LS_ITEMS = 8;
constexpr int LS_CHUNK = LS_THREADS * LS_ITEMS;

int64_t list_scan_tmp(int32_t n) { return cdiv((int64_t)n + 1, LS_CHUNK) + 2; }

__device__ __forceinline__ int64_t item_quads(const int32_t* deg, int32_t v) { return (deg[v] + 3) >> 2; }

__global__ void __launch_bounds__(LS_THREADS) k_ls_reduce(const int32_t* __restrict__ list, const int32_t* count,
                                                          const int32_t* __restrict__ deg, int64_t* __restrict__ sums) {
  __shared__ int64_t wsum[8];
  int32_t K = *count;
  int64_t nch = cdiv(K, LS_CHUNK);
  for (int64_t c = blockIdx.x; c < nch; c += gridDim.x) {
    int64_t base = c * LS_CHUNK + (int64_t)threadIdx.x * LS_ITEMS;
    int64_t x = 0;
#pragma unroll
    for (int i = 0; i < LS_ITEMS; i++)
      if (base + i < K) x += item_quads(deg, list[base + i]);
    int64_t tot;
    block_incl_scan256<int64_t>(x, &tot, wsum);
    if (threadIdx.x == 0) sums[c] = tot;
  }
}

__global__ void __launch_bounds__(LS_THREADS) k_ls_top(int64_t* sums, const int32_t* count, int64_t* qtot,
                                                       int64_t* ntiles) {
  __shared__ int64_t wsum[8];
  int32_t K = *count;
  int64_t nch = cdiv(K, LS_CHUNK);
  int64_t carry = 0;
  for (int64_t base = 0; base < nch; base += LS_THREADS) {
    int64_t j = base + threadIdx.x;
    int64_t x = j < nch ? sums[j] : 0;
    int64_t tot;
    int64_t inc = block_incl_scan256<int64_t>(x, &tot, wsum);
    if (j < nch) sums[j] = carry + inc - x;
    carry += tot;
  }
  if (threadIdx.x == 0) {
    *qtot = carry;
    *ntiles = cdiv(carry, SW_TILE_Q);
  }
}

__global__ void __launch_bounds__(LS_THREADS) k_ls_down(const int32_t* __restrict__ list, const int32_t* count,
                                                        const int32_t* __restrict__ deg, const int64_t* __restrict__ sums,
                                                        int64_t* __restrict__ qs, int32_t* __restrict__ tfirst,
                                                        const int64_t* qtot, const int64_t* ntiles) {
  __shared__ int64_t wsum[8];
  int32_t K = *count;
  int64_t nch = cdiv(K, LS_CHUNK);
  for (int64_t c = blockIdx.x; c < nch; c += gridDim.x) {
    int64_t base = c * LS_CHUNK + (int64_t)threadIdx.x * LS_ITEMS;
    int64_t len[LS_ITEMS];
    int64_t x = 0;
#pragma unroll
    for (int i = 0; i < LS_ITEMS; i++) {
      len[i] = base + i < K ? item_quads(deg, list[base + i]) : 0;
      x += len[i];
    }
    int64_t tot;
    int64_t run = sums[c] + block_incl_scan256<int64_t>(x, &tot, wsum) - x;
#pragma unroll
    for (int i = 0; i < LS_ITEMS; i++) {
      int64_t k = base + i;
      if (k < K) {
        qs[k] = run;
        for (int64_t t = cdiv(run, SW_TILE_Q); t * SW_TILE_Q < run + len[i]; t++) tfirst[t] = (int32_t)k;
      }
      run += len[i];
    }
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    qs[K] = *qtot;
    tfirst[*ntiles] = K;
  }
}

cudaError_t launch_list_scan(const int32_t* list, const int32_t* count, const int32_t* deg, int32_t n, int64_t* qs,
                             int32_t* tfirst, int64_t* qtot_dev, int64_t* ntiles_dev, int64_t* tmp, cudaStream_t s) {
  int64_t maxch = cdiv((int64_t)n + 1, LS_CHUNK);
  int grid = (int)(maxch < num_sms() * 4 ? maxch : num_sms() * 4);
  if (grid < 1) grid = 1;
  note_launch(); k_ls_reduce<<<grid, LS_THREADS, 0, s>>>(list, count, deg, tmp);
  note_launch(); k_ls_top<<<1, LS_THREADS, 0, s>>>(tmp, count, qtot_dev, ntiles_dev);
  note_launch(); k_ls_down<<<grid, LS_THREADS, 0, s>>>(list, count, deg, tmp, qs, tfirst, qtot_dev, ntiles_dev);
  return cudaGetLastError();
}

// ------------------------------------------------------------------ expand

__device__ __forceinline__ bool has_key(const uint64_t* k, int64_t len, uint64_t x) {
  int64_t lo = 0, hi = len;
  while (lo < hi) {
    int64_t mid = (lo + hi) >> 1;
    if (k[mid] < x) lo = mid + 1;
    else hi = mid;
  }
  return lo < len && k[lo] == x;
}

// mark every out-neighbour of every listed vertex (Alg. 1: "mark v' as affected")
__global__ void __launch_bounds__(SW_THREADS) k_expand(ExpandParams p) {
  __shared__ int32_t s_lstart[SW_MAX_ITEMS + 1];
  __shared__ long long s_adj[SW_MAX_ITEMS];
  __shared__ int32_t s_v[SW_MAX_ITEMS];
  const int64_t ntiles = *p.ntiles_dev;
  const int32_t K = *p.count;
  const int64_t Qtot = p.qs[K];
  const uint64_t sent = (uint64_t)p.n;
  for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const int64_t T0 = t * SW_TILE_Q;
    const int64_t T1 = min(T0 + (int64_t)SW_TILE_Q, Qtot);
    const int32_t k_lo = p.tfirst[t];
    int32_t k_hi = p.tfirst[t + 1];
    if (k_hi > K - 1) k_hi = K - 1;
    int nitems = k_hi - k_lo + 1;
    if (nitems > SW_MAX_ITEMS || nitems < 1) break;
    for (int i = threadIdx.x; i < nitems; i += SW_THREADS) {
      int32_t k = k_lo + i;
      int32_t v = p.list[k];
      int64_t q0 = p.qs[k];
      s_v[i] = v;
      s_lstart[i] = (int32_t)(max(q0, T0) - T0);
      s_adj[i] = p.ooff[v] - 4 * q0 + 4 * T0;
    }
    if (threadIdx.x == 0) s_lstart[nitems] = INT_MAX;
    __syncthreads();
    const int nq = (int)(T1 - T0);
#pragma unroll
    for (int j = 0; j < SW_QPT; j++) {
      const int q = threadIdx.x + j * SW_THREADS;
      const bool valid = q < nq;
      int4 c = make_int4(p.n, p.n, p.n, p.n);
      int32_t v = 0;
      if (valid) {
        int owner = tile_owner(s_lstart, nitems, q);
        v = s_v[owner];
        c = __ldg(reinterpret_cast<const int4*>(p.ocol + s_adj[owner] + 4 * (int64_t)q));
      }
      int ws[4] = {c.x, c.y, c.z, c.w};
#pragma unroll
      for (int e = 0; e < 4; e++) {
        int32_t w = ws[e];
        bool cand = (uint64_t)w != sent;
        if (cand && p.ins_src_bits && bit_get(p.ins_src_bits, v))
          cand = !has_key(p.dplus, p.n_dplus, ((uint64_t)v << p.id_bits) | (uint64_t)w);
        bool add = cand && bit_tas(p.bits, w);
        int slot = warp_append(p.cnt, add);
        if (add) {
          p.wl[slot] = w;
          if (p.ever) atomicOr(p.ever + (w >> 5), 1u << (w & 31));
        }
      }
    }
    __syncthreads();
  }
}

cudaError_t launch_expand(const ExpandParams& p, cudaStream_t s) {
  note_launch(); k_expand<<<num_sms() * 4, SW_THREADS, 0, s>>>(p);
  return cudaGetLastError();
}

// ------------------------------------------------------------------ commit

__global__ void k_commit(const int32_t* __restrict__ list, const int32_t* count, const double* __restrict__ rnew,
                         double* __restrict__ R, long long* __restrict__ C, const int32_t* __restrict__ odeg,
                         const double* __restrict__ tab_sc, uint32_t* bits_clear) {
  int32_t K = *count;
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < K; k += (int64_t)gridDim.x * blockDim.x) {
    int32_t v = list[k];
    double r = rnew[k];
    int32_t d = odeg[v];
    R[v] = r;
    double sc = d < TAB ? tab_sc[d] : FIX_ONE / (double)d;
    C[v] = __double2ll_rn(r * sc);
    if (bits_clear) atomicAnd(bits_clear + (v >> 5), ~(1u << (v & 31)));
  }
}

cudaError_t launch_commit(const int32_t* list, const int32_t* count, const double* rnew, double* R, long long* C,
                          const int32_t* odeg, const double* tab_sc, uint32_t* bits_clear, int32_t n, cudaStream_t s) {
  note_launch(); k_commit<<<grid_for(n, 256), 256, 0, s>>>(list, count, rnew, R, C, odeg, tab_sc, bits_clear);
  return cudaGetLastError();
}

}  // namespace dfpr
