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
#include <algorithm>
#include <vector>
#include <climits>
#include <map>
#include <mutex>
#include <tuple>
#include "sweep.cuh"
#include "pull_step.cuh"
#include "fixconv.cuh"
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

// ------------------------------------------------------------------ tiles

// Shared-memory view of one tile: for every item (list entry) touching the
// tile its vertex, the slot offset of its quads, how many tiles it spans, and
// per local quad the item that owns it.
struct TileSmem {
  int16_t owner[SW_TILE_Q];
  long long adj[SW_MAX_ITEMS];
  long long acc[SW_MAX_ITEMS];
  int32_t v[SW_MAX_ITEMS];
  int32_t nt[SW_MAX_ITEMS];
  int32_t any[SW_MAX_ITEMS];
  int32_t wmax[SW_THREADS / WARP];
};

// Load the items of tile [T0, T1) and build owner[] with a block-wide max-scan
// of the item starts (each item owns at least one quad, so starts are distinct).
// ident: items are vertices k with quads ioff[k]/4 .. ioff[k+1]/4; otherwise
// items are list[k] with quads qs[k] .. qs[k+1].  Returns the item count, or -1
// for a malformed tile table.
__device__ __forceinline__ int tile_setup(TileSmem& sm, bool ident, const int32_t* list, const int64_t* qs,
                                          const int64_t* off, int64_t T0, int64_t T1, int32_t k_lo, int32_t k_hi) {
  const int nq = (int)(T1 - T0);
  const int nitems = k_hi - k_lo + 1;
  if (nitems > SW_MAX_ITEMS || nitems < 1) return -1;
#pragma unroll
  for (int j = 0; j < SW_QPT; j++) sm.owner[threadIdx.x * SW_QPT + j] = -1;
  __syncthreads();
  for (int i = threadIdx.x; i < nitems; i += SW_THREADS) {
    int32_t k = k_lo + i;
    int32_t v = ident ? k : list[k];
    int64_t q0 = ident ? (off[v] >> 2) : qs[k];
    int64_t q1 = ident ? (off[v + 1] >> 2) : qs[k + 1];
    sm.v[i] = v;
    sm.adj[i] = off[v] - 4 * q0 + 4 * T0;
    int nt;
    if (q0 >= T1 || q1 <= T0) nt = -1;
    else if (q0 >= T0 && q1 <= T1) nt = 0;
    else nt = (int)((q1 - 1) / SW_TILE_Q - q0 / SW_TILE_Q + 1);
    sm.nt[i] = nt;
    sm.acc[i] = 0;
    sm.any[i] = 0;
    int64_t ls = q0 > T0 ? q0 - T0 : 0;
    if (ls < nq) sm.owner[ls] = (int16_t)i;
  }
  __syncthreads();
  // inclusive max-scan of owner[] (SW_QPT consecutive entries per thread)
  int run[SW_QPT];
  int m = -1;
#pragma unroll
  for (int j = 0; j < SW_QPT; j++) {
    m = max(m, (int)sm.owner[threadIdx.x * SW_QPT + j]);
    run[j] = m;
  }
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  int inc = m;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    int y = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc = max(inc, y);
  }
  if (lane == 31) sm.wmax[w] = inc;
  int excl = __shfl_up_sync(0xffffffffu, inc, 1);
  if (lane == 0) excl = -1;
  __syncthreads();
  for (int ww = 0; ww < w; ww++) excl = max(excl, sm.wmax[ww]);
#pragma unroll
  for (int j = 0; j < SW_QPT; j++) sm.owner[threadIdx.x * SW_QPT + j] = (int16_t)max(excl, run[j]);
  __syncthreads();
  return nitems;
}

// set bit v in B for every lane that asks, one atomic per 32-bit word per warp
__device__ __forceinline__ void agg_set_bit(uint32_t* B, int32_t v, bool set) {
  unsigned act = __activemask();
  unsigned word = (unsigned)v >> 5;
  unsigned grp = __match_any_sync(act, word);
  unsigned val = __reduce_or_sync(grp, set ? (1u << (v & 31)) : 0u);
  if ((threadIdx.x & 31) == __ffs(grp) - 1 && val) atomicOr(B + word, val);
}

__device__ __forceinline__ void agg_count(int32_t* c, bool yes) {
  unsigned act = __activemask();
  unsigned k = __popc(__ballot_sync(act, yes));
  if ((threadIdx.x & 31) == __ffs(act) - 1 && k) atomicAdd(c, (int)k);
}

// ------------------------------------------------------------------ sweep

template <int MODE>
__device__ __forceinline__ void finalize(const SweepParams& p, int32_t k, int32_t v, long long sum, bool any,
                                         double& dmax, long long& edges, long long& verts) {
  constexpr bool pull = MODE == SWEEP_PULL_DF || MODE == SWEEP_PULL_DFP;
  constexpr bool closed = MODE == SWEEP_DFP || MODE == SWEEP_PULL_DFP;
  bool member = true;
  if (pull) member = any || bit_get(p.S_cur, v);
  double Rv = p.R[v];
  int32_t d = p.odeg[v];
  double r;
  if (closed) {
    // Eq. 2: K = sum over in-neighbours minus the vertex's own self-loop term,
    // r = (C0 + alpha K) / (1 - alpha/d); the self term is removed exactly in
    // fixed point, and the expression is one FMA with the coefficients of
    // closed_coeffs, as in the every-vertex epilogues, so that push and pull
    // forms give bit-identical ranks
    long long K = sum - p.Ccur[v];
    const double2 ab = d < TAB ? p.tab_ab[d] : closed_coeffs(p.alpha, p.n, d);
    r = fma(ab.x, (double)K, ab.y);
  } else {
    // Eq. 1: r = C0 + alpha c
    r = fma(p.alpha * FIX_INV, (double)sum, p.C0);
  }
  double dr = fabs(r - Rv);
  if (member) {
    dmax = fmax(dmax, dr);
    edges += p.ideg[v];
    verts += 1;
  }
  if (MODE == SWEEP_FULL || pull) {
    long long cn;
    if (member) {
      p.R[v] = r;
      double sc = d < TAB ? p.tab_sc[d] : FIX_ONE / (double)d;
      cn = __double2ll_rn(r * sc);
    } else {
      cn = p.Ccur[v];
    }
    p.Cnext[v] = cn;
    if (pull) {
      // Alg. 1: prune when dr / max(r, R[v]) <= tau_p (DF-P), expand when it
      // is > tau_f (or the other measures of Sec. 4.3); both compared
      // without the division, in FP64
      double mr = measure_base(p.metric, fmax(r, Rv), d);
      bool stay = member && (MODE == SWEEP_PULL_DF || !(dr <= p.tau_p * mr));
      bool expand = member && dr > p.tau_f * mr;
      agg_set_bit(p.S_next, v, stay);
      agg_set_bit(p.X_next, v, expand);
      agg_set_bit(p.ever, v, member);
      agg_count(p.cnt_next, stay);
      agg_count(p.cnt_x, expand);
    }
    return;
  }
  p.rnew[k] = r;
  if (MODE == SWEEP_DF || MODE == SWEEP_DFP) {
    double mr = measure_base(p.metric, fmax(r, Rv), d);
    bool stay = (MODE == SWEEP_DF) || !(dr <= p.tau_p * mr);
    bool expand = dr > p.tau_f * mr;
    agg_set_bit(p.ever, v, true);
    bool add = stay && bit_tas(p.bits_next, v);
    int slot = warp_append(p.cnt_next, add);
    if (add) p.wl_next[slot] = v;
    int xs = warp_append(p.cnt_x, expand);
    if (expand) p.xl[xs] = v;
  }
}

template <int MODE>
__global__ void __launch_bounds__(SW_THREADS) k_sweep(SweepParams p) {
  __shared__ TileSmem sm;
  constexpr bool pull = MODE == SWEEP_PULL_DF || MODE == SWEEP_PULL_DFP;
  constexpr bool ident = MODE == SWEEP_FULL || pull;
  const int64_t ntiles = ident ? p.ntiles_host : *p.ntiles_dev;
  const int32_t K = ident ? p.n : *p.count;
  const int64_t Qtot = ident ? (p.ioff[p.n] >> 2) : p.qs[K];
  const uint64_t pol_stream = policy_evict_first();
  const uint64_t pol_keep = policy_evict_last();
  const int32_t sent = p.n;
  const int32_t hot = p.hot;
  double dmax = 0.0;
  long long edges = 0, verts = 0;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;

  for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const int64_t T0 = t * SW_TILE_Q;
    const int64_t T1 = min(T0 + (int64_t)SW_TILE_Q, Qtot);
    const int32_t k_lo = p.tfirst[t];
    int32_t k_hi = p.tfirst[t + 1];
    if (k_hi > K - 1) k_hi = K - 1;
    const int nitems = tile_setup(sm, ident, p.list, p.qs, p.ioff, T0, T1, k_lo, k_hi);
    if (nitems < 0) {   // cannot happen for a well-formed tile table
      if (threadIdx.x == 0) p.ctl->status = 1;
      break;
    }
    const int nq = (int)(T1 - T0);
    // all column loads of this thread first, then all gathers, then the reductions
    int own[SW_QPT];
    int4 c[SW_QPT];
#pragma unroll
    for (int j = 0; j < SW_QPT; j++) {
      const int q = lane + WARP * (w + (SW_THREADS / WARP) * j);
      own[j] = SW_MAX_ITEMS;
      c[j] = make_int4(sent, sent, sent, sent);
      if (q < nq) {
        own[j] = sm.owner[q];
        const long long base = ident ? 4 * T0 : sm.adj[own[j]];
        c[j] = ld_stream4(p.icol + base + 4 * (long long)q, pol_stream);
      }
    }
    long long sum[SW_QPT];
    unsigned xb[SW_QPT];
#pragma unroll
    for (int j = 0; j < SW_QPT; j++) {
      sum[j] = ld_hint(p.Ccur + c[j].x, c[j].x < hot ? pol_keep : pol_stream) +
               ld_hint(p.Ccur + c[j].y, c[j].y < hot ? pol_keep : pol_stream) +
               ld_hint(p.Ccur + c[j].z, c[j].z < hot ? pol_keep : pol_stream) +
               ld_hint(p.Ccur + c[j].w, c[j].w < hot ? pol_keep : pol_stream);
      xb[j] = 0;
      if (pull) {
        xb[j] = ((__ldg(p.X_cur + (c[j].x >> 5)) >> (c[j].x & 31)) | (__ldg(p.X_cur + (c[j].y >> 5)) >> (c[j].y & 31)) |
                 (__ldg(p.X_cur + (c[j].z >> 5)) >> (c[j].z & 31)) | (__ldg(p.X_cur + (c[j].w >> 5)) >> (c[j].w & 31))) &
                1u;
      }
    }
#pragma unroll
    for (int j = 0; j < SW_QPT; j++) {
      const int owner = own[j];
      long long s = sum[j];
      unsigned x = xb[j];
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        long long os = __shfl_down_sync(0xffffffffu, s, o);
        unsigned ox = __shfl_down_sync(0xffffffffu, x, o);
        int oo = __shfl_down_sync(0xffffffffu, owner, o);
        if (lane + o < 32 && oo == owner) {
          s += os;
          x |= ox;
        }
      }
      int prev = __shfl_up_sync(0xffffffffu, owner, 1);
      if (owner != SW_MAX_ITEMS && (lane == 0 || prev != owner)) {
        atomicAdd(reinterpret_cast<unsigned long long*>(&sm.acc[owner]), (unsigned long long)s);
        if (pull && x) sm.any[owner] = 1;
      }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < nitems; i += SW_THREADS) {
      int nt = sm.nt[i];
      if (nt < 0) continue;
      int32_t k = k_lo + i;
      long long total = sm.acc[i];
      int any = sm.any[i];
      if (nt > 0) {
        atomicAdd(reinterpret_cast<unsigned long long*>(&p.gacc[k]), (unsigned long long)total);
        if (pull && any) atomicOr(&p.gany[k], 1);
        __threadfence();
        int ticket = atomicAdd(&p.gcnt[k], 1);
        if (ticket != nt - 1) continue;
        __threadfence();
        total = (long long)atomicExch(reinterpret_cast<unsigned long long*>(&p.gacc[k]), 0ull);
        if (pull) any = atomicExch(&p.gany[k], 0);
        p.gcnt[k] = 0;
      }
      finalize<MODE>(p, k, sm.v[i], total, any != 0, dmax, edges, verts);
    }
    __syncthreads();
  }
  block_flush_stats(dmax, edges, verts, p.ctl);
}

// ------------------------------------------------------------------ full sweeps in two phases
//
// A sweep over every vertex (Static, ND, and the pull form of DF / DF-P) needs
// no vertex list: the in-CSR rows lie in vertex order, quad-aligned, so the
// quad space is walked linearly (pull_step.cuh).
//   k_gather_rows: warps take 32 x SW_QPT quads per step and add each row
//     piece's partial sum to the row's accumulator;
//   k_finish_pull / k_finish_full: read and clear each vertex's accumulator
//     and run the epilogue.
//   With HUB, every block first stages the contributions of the hub vertices
//   [0, hub_k) (and, in pull form, the expanded bits of their words) in
//   shared memory; the grid is then one wave of resident blocks, so the
//   staging is paid once per block and sweep.
// (2 quads per lane: held to 32 registers, two 1024-thread blocks per SM)
template <bool PULL, int QPT, bool HUB>
__global__ void __launch_bounds__(1024, QPT == 2 ? 2 : 1) k_gather_rows(const int32_t* __restrict__ icol, const long long* __restrict__ C,
                                                      const uint32_t* __restrict__ X, const uint32_t* __restrict__ S,
                                                      const uint32_t* __restrict__ rowbits,
                                                      const int32_t* __restrict__ rowbase, int64_t nquads, int32_t sent,
                                                      long long* __restrict__ acc, uint32_t* __restrict__ anyb,
                                                      int32_t hub_k, int32_t hub_kx, const int64_t* __restrict__ ioff,
                                                      int32_t v_lo, int32_t v_hi) {
  extern __shared__ __align__(16) unsigned char hub_smem[];
  const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const uint64_t pol_stream = policy_evict_first();
  const uint64_t pol_keep = policy_evict_last();
  HubView hub;
  if (HUB) {
    long long* hc = reinterpret_cast<long long*>(hub_smem);
    uint32_t* hx = reinterpret_cast<uint32_t*>(hc + hub_k);
    for (int i = threadIdx.x; i < hub_k; i += blockDim.x) hc[i] = ld_hint(C + i, pol_keep);
    if (PULL)
      for (int i = threadIdx.x; i < hub_kx; i += blockDim.x) hx[i] = __ldg(X + i);
    __syncthreads();
    hub.c = hc;
    hub.x = hx;
    hub.k = hub_k;
    hub.kx = PULL ? hub_kx : 0;
  }
  // the rows of vertices [v_lo, v_hi): quads [qlo, qhi), walked in steps
  // aligned to 32 x QPT quads (the row-start index is per 32-quad word)
  const int64_t qlo = v_lo > 0 ? __ldg(ioff + v_lo) >> 2 : 0;
  const int64_t qhi = v_hi < sent ? __ldg(ioff + v_hi) >> 2 : nquads;
  const int64_t q0 = qlo / (32 * QPT) * (32 * QPT);
  for (int64_t base = q0 + warp * 32 * QPT; base < qhi; base += nw * 32 * QPT)
    gather_step<PULL, QPT, HUB>(icol, C, X, S, rowbits, rowbase, qhi, sent, acc, anyb, base, pol_stream, pol_keep,
                                hub, qlo);
}

// (the 32-vertex chunks [ch_lo, ch_hi); ch_lo a multiple of FIN_U)
template <bool CLOSED, bool REL, bool SAME = false>
__global__ void __launch_bounds__(256, 3) k_finish_pull(SweepParams p, long long* __restrict__ acc,
                                                        uint32_t* __restrict__ anyb, int64_t ch_lo, int64_t ch_hi) {
  const int lane = threadIdx.x & 31;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  PullTotals t;
  for (int64_t ch0 = ch_lo + ((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5) * FIN_U; ch0 < ch_hi;
       ch0 += nw * FIN_U)
    finish_pull_step<CLOSED, SweepParams, false, FIN_U, REL, SAME>(p, acc, anyb, ch0, ch_hi, t);
  if (lane == 0) {
    if (t.stays) atomicAdd(p.cnt_next, t.stays);
    if (t.exps) atomicAdd(p.cnt_x, t.exps);
  }
  block_flush_stats(__longlong_as_double((long long)t.dmax), t.edges, t.verts, p.ctl);
}

// Epilogue of a sweep over every vertex with Eq. 1 (Static, ND): all vertices
// are processed; loads of U vertices per lane are issued together.
// (vertices [v_lo, v_hi))
__global__ void __launch_bounds__(256, 4) k_finish_full(SweepParams p, long long* __restrict__ acc, int64_t v_lo,
                                                        int64_t v_hi) {
  constexpr int U = 4;
  const double alpha_fix = p.alpha * FIX_INV;
  unsigned long long dmax = 0ull;
  long long edges = 0, verts = 0;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t v0 = v_lo + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v0 < v_hi; v0 += stride * U) {
    long long sum[U];
    double Rv[U];
    int32_t d[U];
#pragma unroll
    for (int u = 0; u < U; u++) {
      const int64_t v = v0 + u * stride;
      const bool ok = v < v_hi;
      sum[u] = ok ? acc[v] : 0;
      Rv[u] = ok ? p.R[v] : 0.0;
      d[u] = ok ? p.odeg[v] : 1;
    }
#pragma unroll
    for (int u = 0; u < U; u++) {
      const int64_t v = v0 + u * stride;
      if (v >= v_hi) continue;
      acc[v] = 0;
      const double r = fma(alpha_fix, (double)sum[u], p.C0);   // Eq. 1
      const unsigned long long drb = dbits(fabs(r - Rv[u]));
      dmax = drb > dmax ? drb : dmax;
      edges += p.ideg[v];
      verts += 1;
      p.R[v] = r;
      const double sc = d[u] < TAB ? p.tab_sc[d[u]] : FIX_ONE / (double)d[u];
      p.Cnext[v] = fixconv::f64_to_i64_rn(r * sc);   // integer pipes: the FP64 pipe bounds this epilogue
    }
  }
  block_flush_stats(__longlong_as_double((long long)dmax), edges, verts, p.ctl);
}

// ------------------------------------------------------------------ every-vertex sweep in one launch
//
// The gather of the rows and the epilogue of Eq. 1 / Eq. 2 in one kernel.  The
// vertices are cut into chunks of FIN_U x 32; every task (TASK_Q consecutive
// quads, gathered by one warp) that adds to the rows of a chunk counts itself
// in done[chunk] after its writes are visible (fence, then the count).  The
// task that brings the count to the number of tasks over the chunk's rows runs
// the chunk's epilogue itself and resets the count.  Nothing waits on anything: a chunk
// is finished by whichever warp completes it.  The epilogue is bound by the
// FP64 pipe and the gather by memory throughput, so in one launch the two
// overlap across the warps of an SM.

// Eq. 1 for every vertex of chunks [ch0, ch0 + U) (Static, ND): the
// arithmetic of k_finish_full, one lane per vertex
template <int U>
__device__ __forceinline__ void finish_full_step(const SweepParams& p, long long* __restrict__ acc, int64_t ch0,
                                                 PullTotals& t) {
  const int lane = threadIdx.x & 31;
  const double alpha_fix = p.alpha * FIX_INV;
  long long sum[U];
  double Rv[U];
  int32_t d[U];
#pragma unroll
  for (int u = 0; u < U; u++) {
    const int64_t v = (ch0 + u) * 32 + lane;
    const bool ok = v < p.n;
    sum[u] = ok ? __ldcg(acc + v) : 0;
    Rv[u] = ok ? p.R[v] : 0.0;
    d[u] = ok ? p.odeg[v] : 1;
  }
#pragma unroll
  for (int u = 0; u < U; u++) {
    const int64_t v = (ch0 + u) * 32 + lane;
    if (v >= p.n) continue;
    acc[v] = 0;
    const double r = fma(alpha_fix, (double)sum[u], p.C0);   // Eq. 1
    const unsigned long long drb = dbits(fabs(r - Rv[u]));
    t.dmax = drb > t.dmax ? drb : t.dmax;
    t.edges += p.ideg[v];
    t.verts += 1;
    p.R[v] = r;
    const double sc = d[u] < TAB ? p.tab_sc[d[u]] : FIX_ONE / (double)d[u];
    p.Cnext[v] = fixconv::f64_to_i64_rn(r * sc);
  }
}

// block totals of the epilogue (any block size up to 1024)
__device__ __forceinline__ void block_flush_totals(const PullTotals& t, Ctl* ctl, int32_t* cnt_next, int32_t* cnt_x) {
  __shared__ unsigned long long s_d[32];
  __shared__ long long s_e[32], s_v[32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (lane == 0) {
    if (t.stays) atomicAdd(cnt_next, t.stays);
    if (t.exps) atomicAdd(cnt_x, t.exps);
  }
  unsigned long long dm = t.dmax;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long y = __shfl_xor_sync(0xffffffffu, dm, o);
    dm = y > dm ? y : dm;
  }
  const long long e = warp_sum_ll(t.edges), v = warp_sum_ll(t.verts);
  if (lane == 0) {
    s_d[w] = dm;
    s_e[w] = e;
    s_v[w] = v;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long d = 0;
    long long es = 0, vs = 0;
    for (int i = 0; i < (int)(blockDim.x >> 5); i++) {
      d = s_d[i] > d ? s_d[i] : d;
      es += s_e[i];
      vs += s_v[i];
    }
    if (d) atomicMax(&ctl->dR, d);
    if (es) atomicAdd((unsigned long long*)&ctl->edges, (unsigned long long)es);
    if (vs) atomicAdd((unsigned long long*)&ctl->verts, (unsigned long long)vs);
  }
}

constexpr int64_t TASK_Q = 1024;   // quads per task of k_sweep_rows (a multiple of 32 x QPT)

template <int MODE, int QPT, bool HUB>
__global__ void __launch_bounds__(1024) k_sweep_rows(SweepParams p, const uint32_t* __restrict__ rowbits,
                                                     const int32_t* __restrict__ rowbase, uint32_t* __restrict__ anyb,
                                                     int32_t* __restrict__ done, int32_t hub_k, int32_t hub_kx) {
  constexpr bool PULL = MODE != SWEEP_FULL;
  constexpr int64_t UQ = 32 * QPT;          // quads per gather step
  constexpr int CV = FIN_U * 32;            // vertices per epilogue chunk
  extern __shared__ __align__(16) unsigned char hub_smem[];
  const int lane = threadIdx.x & 31;
  const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int64_t nquads = p.ntiles_host;
  const int64_t nunits = cdiv(nquads, UQ);
  const int64_t nch32 = cdiv(p.n, 32);
  const uint64_t pol_stream = policy_evict_first();
  const uint64_t pol_keep = policy_evict_last();
  HubView hub;
  if (HUB) {
    long long* hc = reinterpret_cast<long long*>(hub_smem);
    uint32_t* hx = reinterpret_cast<uint32_t*>(hc + hub_k);
    for (int i = threadIdx.x; i < hub_k; i += blockDim.x) hc[i] = ld_hint(p.Ccur + i, pol_keep);
    if (PULL)
      for (int i = threadIdx.x; i < hub_kx; i += blockDim.x) hx[i] = __ldg(p.X_cur + i);
    __syncthreads();
    hub.c = hc;
    hub.x = hx;
    hub.k = hub_k;
    hub.kx = PULL ? hub_kx : 0;
  }
  PullTotals t;
  // a warp takes TASK_Q consecutive quads (RU gather steps) at a time, so the
  // fence that publishes its sums is paid once per task
  constexpr int RU = (int)(TASK_Q / UQ);
  const int64_t ntasks = cdiv(nunits, RU);
  for (int64_t tk = warp; tk < ntasks; tk += nw) {
    int first = INT_MAX, last = -1;
    bool wrote = false;
    for (int r = 0; r < RU; r++) {
      const int64_t u = tk * RU + r;
      if (u >= nunits) break;
      const GatherSpan sp = gather_step<PULL, QPT, HUB, true>(p.icol, p.Ccur, p.X_cur, p.S_cur, rowbits, rowbase, nquads,
                                                        p.n, p.gacc, anyb, u * UQ, pol_stream, pol_keep, hub);
      first = min(first, sp.first);
      last = max(last, sp.last);
      wrote = wrote || sp.wrote;
    }
    // publish this task's sums, then count it in every chunk it touched; a
    // task spans at most TASK_Q rows, so at most TASK_Q / CV + 2 chunks
    if (wrote) __threadfence();
    __syncwarp();
    const int c0 = first / CV, c1 = last / CV;
    unsigned mine = 0u;
    if (lane <= c1 - c0) {
      const int c = c0 + lane;
      const int64_t v0 = (int64_t)c * CV, v1 = min((int64_t)p.n, v0 + CV);
      const int64_t need = (__ldg(p.ioff + v1) / 4 - 1) / TASK_Q - (__ldg(p.ioff + v0) / 4) / TASK_Q + 1;
      if (atomicAdd(done + c, 1) == (int)need - 1) {
        done[c] = 0;
        mine = 1u;
      }
    }
    unsigned fin = __ballot_sync(0xffffffffu, mine);
    if (fin) __threadfence();   // the chunk's sums, now complete, are read after the count
    while (fin) {
      const int k = __ffs(fin) - 1;
      fin &= fin - 1;
      // one 32-vertex word at a time: other warps hide the latency, and the
      // gather keeps its registers
      for (int w = 0; w < FIN_U; w++) {
        const int64_t ch = (int64_t)(c0 + k) * FIN_U + w;
        if (MODE == SWEEP_FULL)
          finish_full_step<1>(p, p.gacc, ch, t);
        else
          finish_pull_step<MODE == SWEEP_PULL_DFP, SweepParams, true, 1>(p, p.gacc, anyb, ch, nch32, t);
      }
    }
  }
  block_flush_totals(t, p.ctl, p.cnt_next, p.cnt_x);
}

template <int MODE, int QPT, bool HUB>
static cudaError_t sweep_rows_launch(const SweepParams& p, const uint32_t* rowbits, const int32_t* rowbase,
                                     uint32_t* anyb, int32_t* done, int threads, int32_t hub_k, int32_t hub_kx,
                                     cudaStream_t s) {
  const void* fn = (const void*)k_sweep_rows<MODE, QPT, HUB>;
  const size_t smem = HUB ? gather_hub_bytes(hub_k, hub_kx) : 0;
  int bps = 1;
  cudaError_t e = gather_occupancy(fn, threads, smem, &bps);
  if (e != cudaSuccess) return e;
  const int64_t tasks = cdiv(p.ntiles_host, TASK_Q);
  const int64_t cap = (int64_t)num_sms() * bps;
  const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(cdiv(tasks, threads / 32), cap));
  note_launch();
  k_sweep_rows<MODE, QPT, HUB><<<grid, threads, smem, s>>>(p, rowbits, rowbase, anyb, done, hub_k, hub_kx);
  return cudaGetLastError();
}

template <int MODE>
static cudaError_t sweep_rows_dispatch(const SweepParams& p, const GatherCfg& cfg, const uint32_t* rowbits,
                                       const int32_t* rowbase, uint32_t* anyb, int32_t* done, cudaStream_t s) {
  constexpr bool PULL = MODE != SWEEP_FULL;
  const int32_t hub_k = std::min<int32_t>(cfg.hub, p.n + 1);
  const int32_t hub_kx = PULL ? (int32_t)cdiv(std::min<int32_t>(hub_k, p.n), 32) : 0;
  const int t = cfg.threads;
  switch (cfg.qpt * 2 + (hub_k > 0 ? 1 : 0)) {
    case 4: return sweep_rows_launch<MODE, 2, false>(p, rowbits, rowbase, anyb, done, t, 0, 0, s);
    case 5: return sweep_rows_launch<MODE, 2, true>(p, rowbits, rowbase, anyb, done, t, hub_k, hub_kx, s);
    case 8: return sweep_rows_launch<MODE, 4, false>(p, rowbits, rowbase, anyb, done, t, 0, 0, s);
    case 9: return sweep_rows_launch<MODE, 4, true>(p, rowbits, rowbase, anyb, done, t, hub_k, hub_kx, s);
    case 16: return sweep_rows_launch<MODE, 8, false>(p, rowbits, rowbase, anyb, done, t, 0, 0, s);
    case 17: return sweep_rows_launch<MODE, 8, true>(p, rowbits, rowbase, anyb, done, t, hub_k, hub_kx, s);
    default: return cudaErrorInvalidValue;
  }
}

template <bool PULL, int QPT, bool HUB>
static cudaError_t gather_launch(const SweepParams& p, const uint32_t* rowbits, const int32_t* rowbase, uint32_t* anyb,
                                 int64_t nquads, int threads, int32_t hub_k, int32_t hub_kx, int32_t v_lo, int32_t v_hi,
                                 bool one_wave, cudaStream_t s) {
  const void* fn = (const void*)k_gather_rows<PULL, QPT, HUB>;
  const size_t smem = HUB ? gather_hub_bytes(hub_k, hub_kx) : 0;
  int bps = 1;
  cudaError_t e = gather_occupancy(fn, threads, smem, &bps);
  if (e != cudaSuccess) return e;
  // one wave of resident blocks when each block stages a hub cache, else up
  // to 64 blocks of 256 threads per SM (eight waves of 1024-thread blocks at
  // two per SM: the blocks' uneven ends, from hub rows and their atomics,
  // are spread over more, shorter blocks; DF-P pull sweeps at R-MAT 25 took
  // 4.06 ms with two waves, 3.97 with eight, 3.99 with sixteen, 4.04 with
  // thirty-two and 4.28 with sixty-four, and one wave 3.5% more than two);
  // never more warps than work units
  const int64_t units = cdiv(nquads, 32 * QPT);
  const int64_t cap = HUB || one_wave ? (int64_t)num_sms() * bps : (int64_t)num_sms() * 64 * 256 / threads;
  const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(cdiv(units, threads / 32), cap));
  note_launch();
  k_gather_rows<PULL, QPT, HUB><<<grid, threads, smem, s>>>(p.icol, p.Ccur, PULL ? p.X_cur : nullptr,
                                                          PULL ? p.S_cur : nullptr, rowbits, rowbase, nquads, p.n,
                                                          p.gacc, anyb, hub_k, hub_kx, p.ioff, v_lo, v_hi);
  return cudaGetLastError();
}

template <bool PULL>
static cudaError_t gather_dispatch(const SweepParams& p, const GatherCfg& cfg, const uint32_t* rowbits,
                                   const int32_t* rowbase, uint32_t* anyb, int64_t nquads, int32_t v_lo, int32_t v_hi,
                                   cudaStream_t s) {
  const bool ow = cfg.parts > 1;
  const int32_t hub_k = std::min<int32_t>(cfg.hub, p.n + 1);
  const int32_t hub_kx = PULL ? (int32_t)cdiv(std::min<int32_t>(hub_k, p.n), 32) : 0;
  const bool hub = hub_k > 0;
  const int t = cfg.threads;
  switch (cfg.qpt * 2 + (hub ? 1 : 0)) {
    case 4: return gather_launch<PULL, 2, false>(p, rowbits, rowbase, anyb, nquads, t, 0, 0, v_lo, v_hi, ow, s);
    case 5: return gather_launch<PULL, 2, true>(p, rowbits, rowbase, anyb, nquads, t, hub_k, hub_kx, v_lo, v_hi, ow, s);
    case 8: return gather_launch<PULL, 4, false>(p, rowbits, rowbase, anyb, nquads, t, 0, 0, v_lo, v_hi, ow, s);
    case 9: return gather_launch<PULL, 4, true>(p, rowbits, rowbase, anyb, nquads, t, hub_k, hub_kx, v_lo, v_hi, ow, s);
    case 16: return gather_launch<PULL, 8, false>(p, rowbits, rowbase, anyb, nquads, t, 0, 0, v_lo, v_hi, ow, s);
    case 17: return gather_launch<PULL, 8, true>(p, rowbits, rowbase, anyb, nquads, t, hub_k, hub_kx, v_lo, v_hi, ow, s);
    default: return cudaErrorInvalidValue;
  }
}

size_t gather_hub_bytes(int32_t hub_k, int32_t hub_kx) {
  return sizeof(long long) * (size_t)hub_k + sizeof(uint32_t) * (size_t)hub_kx;
}

// resident blocks per SM of a gather kernel with `smem` bytes of dynamic
// shared memory (raising the kernel's dynamic shared memory limit once)
cudaError_t gather_occupancy(const void* fn, int threads, size_t smem, int* bps) {
  static std::mutex mu;
  static std::map<const void*, size_t> limit;
  static std::map<std::tuple<const void*, int, size_t>, int> cache;
  std::lock_guard<std::mutex> lock(mu);
  auto key = std::make_tuple(fn, threads, smem);
  auto it = cache.find(key);
  if (it != cache.end()) {
    *bps = it->second;
    return cudaSuccess;
  }
  size_t& lim = limit[fn];
  if (smem > lim) {
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    lim = smem;
  }
  int b = 0;
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, fn, threads, smem);
  if (e != cudaSuccess) return e;
  if (b < 1) return cudaErrorInvalidConfiguration;
  cache[key] = b;
  *bps = b;
  return cudaSuccess;
}

bool gather_cfg_valid(const GatherCfg& c) {
  if (c.threads != 256 && c.threads != 512 && c.threads != 1024) return false;
  if (c.qpt != 2 && c.qpt != 4 && c.qpt != 8) return false;
  if (c.fused != 0 && c.fused != 1) return false;
  if (c.parts != 1 && c.parts != 2 && c.parts != 4 && c.parts != 8) return false;
  if (c.parts > 1 && c.fused) return false;
  return c.hub >= 0 && gather_hub_bytes(c.hub, (int32_t)cdiv(c.hub, 32)) <= (size_t)GATHER_SMEM_MAX;
}

cudaError_t launch_gather(bool pull, const SweepParams& p, const GatherCfg& cfg, const uint32_t* rowbits,
                          const int32_t* rowbase, uint32_t* anyb, int64_t nquads, cudaStream_t s) {
  if (!gather_cfg_valid(cfg)) return cudaErrorInvalidValue;
  return pull ? gather_dispatch<true>(p, cfg, rowbits, rowbase, anyb, nquads, 0, p.n, s)
              : gather_dispatch<false>(p, cfg, rowbits, rowbase, anyb, nquads, 0, p.n, s);
}

// in-degree sums of the 128-vertex chunks
__global__ void k_chunk_degrees(const int32_t* __restrict__ ideg, int32_t n, int64_t chunks, int64_t* __restrict__ out) {
  for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < chunks; c += (int64_t)gridDim.x * blockDim.x) {
    const int64_t v0 = c * 128, v1 = v0 + 128 < (int64_t)n ? v0 + 128 : (int64_t)n;
    int64_t sum = 0;
    for (int64_t v = v0; v < v1; v++) sum += ideg[v];
    out[c] = sum;
  }
}

// pre[0..chunks]: in-degree prefix before each chunk (pre[chunks] = all);
// first[k - 1] = the first chunk j in [0, chunks] with P pre[j] >= k pre[chunks]
__global__ void k_range_chunks(const int64_t* __restrict__ pre, int64_t chunks, int P, int64_t* __restrict__ first) {
  const int64_t W = pre[chunks];
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j <= chunks; j += (int64_t)gridDim.x * blockDim.x)
    for (int k = 1; k < P; k++)
      if (pre[j] * P >= (int64_t)k * W && (j == 0 || pre[j - 1] * P < (int64_t)k * W)) first[k - 1] = j;
}

int64_t async_range_scratch(int32_t n, int P) {
  const int64_t chunks = cdiv((int64_t)n, 128);
  return chunks + 1 + scan_tmp_elems(chunks) + P;
}

cudaError_t async_range_bounds(const int32_t* ideg, int32_t n, int P, int64_t* scratch, int32_t* bounds,
                               cudaStream_t s) {
  bounds[0] = 0;
  bounds[P > 1 && n >= 128 * P ? P : 1] = n;
  if (P <= 1 || n < 128 * P) return cudaSuccess;
  const int64_t chunks = cdiv((int64_t)n, 128);
  int64_t* pre = scratch;
  int64_t* tmp = pre + chunks + 1;
  int64_t* first = tmp + scan_tmp_elems(chunks);
  note_launch();
  k_chunk_degrees<<<grid_for(chunks, 256), 256, 0, s>>>(ideg, n, chunks, pre);
  cudaError_t e = scan_excl<int64_t>(pre, pre, chunks, tmp, s);
  if (e != cudaSuccess) return e;
  note_launch();
  k_range_chunks<<<grid_for(chunks + 1, 256), 256, 0, s>>>(pre, chunks, P, first);
  std::vector<int64_t> h(P - 1);
  if ((e = cudaMemcpyAsync(h.data(), first, sizeof(int64_t) * (P - 1), cudaMemcpyDeviceToHost, s)) != cudaSuccess ||
      (e = cudaStreamSynchronize(s)) != cudaSuccess)
    return e;
  for (int k = 1; k < P; k++) bounds[k] = (int32_t)std::min<int64_t>(128 * h[k - 1], n);
  return cudaGetLastError();
}

cudaError_t launch_full_sweep(int mode, const SweepParams& p, const GatherCfg& cfg, const uint32_t* rowbits,
                              const int32_t* rowbase, uint32_t* anyb, int32_t* done, const SweepAux* aux,
                              cudaStream_t s, bool ordered, const int32_t* bounds) {
  const int64_t nquads = p.ntiles_host;   // quads of the in-CSR capacity
  const bool pull = mode == SWEEP_PULL_DF || mode == SWEEP_PULL_DFP;
  if (pull) {
    cudaError_t e = cudaMemsetAsync(anyb, 0, sizeof(uint32_t) * (size_t)(cdiv(p.n, 32) + 1), s);
    if (e != cudaSuccess) return e;
  }
  if (cfg.fused && !ordered) {
    if (!gather_cfg_valid(cfg)) return cudaErrorInvalidValue;
    switch (mode) {
      case SWEEP_FULL: return sweep_rows_dispatch<SWEEP_FULL>(p, cfg, rowbits, rowbase, anyb, done, s);
      case SWEEP_PULL_DF: return sweep_rows_dispatch<SWEEP_PULL_DF>(p, cfg, rowbits, rowbase, anyb, done, s);
      case SWEEP_PULL_DFP: return sweep_rows_dispatch<SWEEP_PULL_DFP>(p, cfg, rowbits, rowbase, anyb, done, s);
      default: return cudaErrorInvalidValue;
    }
  }
  if (!ordered && !gather_cfg_valid(cfg)) return cudaErrorInvalidValue;
  // P vertex ranges cut at multiples of 128: the gather of range k + 1 runs on
  // s while the epilogue of range k runs on the auxiliary stream, so the
  // FP64-bound epilogue overlaps the memory-bound gather; the epilogues join s
  // at the end.  P = 1: gather then epilogue on s.  Ordered (asynchronous
  // order): every range's gather and epilogue on s, one range after another.
  const int P = ordered ? (p.n >= 128 * cfg.parts ? cfg.parts : 1)
                        : ((aux && cfg.parts > 1 && p.n >= 128 * cfg.parts) ? cfg.parts : 1);
  if (ordered) aux = nullptr;
  cudaStream_t fs = P > 1 && !ordered ? aux->stream : s;
  for (int k = 0; k < P; k++) {
    // the asynchronous order's ranges hold equal shares of the in-edges;
    // ranges overlapping gather and epilogue are cut by vertex count
    const int32_t v_lo = ordered && bounds ? bounds[k] : (int32_t)((int64_t)p.n * k / P / 128 * 128);
    const int32_t v_hi = ordered && bounds ? bounds[k + 1]
                                           : (k + 1 == P ? p.n : (int32_t)((int64_t)p.n * (k + 1) / P / 128 * 128));
    if (ordered && v_hi <= v_lo) continue;   // an empty range (a hub range holding several shares)
    cudaError_t e = pull ? gather_dispatch<true>(p, cfg, rowbits, rowbase, anyb, nquads, v_lo, v_hi, s)
                         : gather_dispatch<false>(p, cfg, rowbits, rowbase, anyb, nquads, v_lo, v_hi, s);
    if (e != cudaSuccess) return e;
    if (P > 1 && !ordered) {
      if ((e = cudaEventRecord(aux->ev[k], s)) != cudaSuccess) return e;
      if ((e = cudaStreamWaitEvent(fs, aux->ev[k], 0)) != cudaSuccess) return e;
    }
    const int64_t ch_lo = v_lo / 32, ch_hi = cdiv(v_hi, 32);
    // one wave of resident epilogue blocks: every warp strides over the same
    // number of chunks, and no partial last wave leaves most SMs idle
    int bps = 1;
    const bool rel = p.metric == METRIC_RELATIVE;
    const void* fin = mode == SWEEP_FULL       ? (const void*)k_finish_full
                      : mode == SWEEP_PULL_DF  ? (rel ? (const void*)k_finish_pull<false, true>
                                                      : (const void*)k_finish_pull<false, false>)
                      : rel && p.tau_f == p.tau_p ? (const void*)k_finish_pull<true, true, true>
                      : rel                        ? (const void*)k_finish_pull<true, true>
                                                   : (const void*)k_finish_pull<true, false>;
    if ((e = gather_occupancy(fin, 256, 0, &bps)) != cudaSuccess) return e;
    const int rgrid = (int)std::min<int64_t>(grid_for(v_hi - v_lo, 256), (int64_t)num_sms() * bps);
    switch (mode) {
      case SWEEP_FULL: note_launch(); k_finish_full<<<rgrid, 256, 0, fs>>>(p, p.gacc, v_lo, v_hi); break;
      case SWEEP_PULL_DF:
        note_launch();
        if (p.metric == METRIC_RELATIVE) k_finish_pull<false, true><<<rgrid, 256, 0, fs>>>(p, p.gacc, anyb, ch_lo, ch_hi);
        else k_finish_pull<false, false><<<rgrid, 256, 0, fs>>>(p, p.gacc, anyb, ch_lo, ch_hi);
        break;
      case SWEEP_PULL_DFP:
        note_launch();
        if (p.metric == METRIC_RELATIVE && p.tau_f == p.tau_p)
          k_finish_pull<true, true, true><<<rgrid, 256, 0, fs>>>(p, p.gacc, anyb, ch_lo, ch_hi);
        else if (p.metric == METRIC_RELATIVE)
          k_finish_pull<true, true><<<rgrid, 256, 0, fs>>>(p, p.gacc, anyb, ch_lo, ch_hi);
        else k_finish_pull<true, false><<<rgrid, 256, 0, fs>>>(p, p.gacc, anyb, ch_lo, ch_hi);
        break;
      default: return cudaErrorInvalidValue;
    }
  }
  if (P > 1 && !ordered) {
    cudaError_t e = cudaEventRecord(aux->ev[P], fs);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(s, aux->ev[P], 0);
    if (e != cudaSuccess) return e;
  }
  return cudaGetLastError();
}

// bitmap of the quads where an in-CSR row starts, and per 32-quad word the
// number of rows that start before it
__global__ void k_row_start_bits(const int64_t* __restrict__ off, int32_t n, uint32_t* __restrict__ bits) {
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
    int64_t q = off[v] >> 2;
    atomicOr(bits + (q >> 5), 1u << (q & 31));
  }
}
__global__ void k_word_popc(const uint32_t* __restrict__ bits, int64_t words, int32_t* __restrict__ out) {
  for (int64_t w = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; w < words; w += (int64_t)gridDim.x * blockDim.x)
    out[w] = __popc(bits[w]);
}

cudaError_t launch_row_start_index(const int64_t* off, int32_t n, int64_t nquads, uint32_t* rowbits, int32_t* rowbase,
                                   int32_t* tmp, cudaStream_t s) {
  const int64_t words = cdiv(nquads, 32);
  cudaError_t e = cudaMemsetAsync(rowbits, 0, sizeof(uint32_t) * (size_t)(words + 1), s);
  if (e != cudaSuccess) return e;
  note_launch(); k_row_start_bits<<<grid_for(n, 256), 256, 0, s>>>(off, n, rowbits);
  note_launch(); k_word_popc<<<grid_for(words, 256), 256, 0, s>>>(rowbits, words, rowbase);
  e = scan_excl<int32_t>(rowbase, rowbase, words, tmp, s);
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

cudaError_t launch_sweep(int mode, const SweepParams& p, cudaStream_t s) {
  int grid = num_sms() * 4;
  if (mode == SWEEP_FULL || mode == SWEEP_PULL_DF || mode == SWEEP_PULL_DFP) {
    int64_t want = p.ntiles_host > 0 ? p.ntiles_host : 1;
    if (want < grid) grid = (int)want;
  }
  switch (mode) {
    case SWEEP_FULL: note_launch(); k_sweep<SWEEP_FULL><<<grid, SW_THREADS, 0, s>>>(p); break;
    case SWEEP_LIST: note_launch(); k_sweep<SWEEP_LIST><<<grid, SW_THREADS, 0, s>>>(p); break;
    case SWEEP_DF: note_launch(); k_sweep<SWEEP_DF><<<grid, SW_THREADS, 0, s>>>(p); break;
    case SWEEP_DFP: note_launch(); k_sweep<SWEEP_DFP><<<grid, SW_THREADS, 0, s>>>(p); break;
    case SWEEP_PULL_DF: note_launch(); k_sweep<SWEEP_PULL_DF><<<grid, SW_THREADS, 0, s>>>(p); break;
    case SWEEP_PULL_DFP: note_launch(); k_sweep<SWEEP_PULL_DFP><<<grid, SW_THREADS, 0, s>>>(p); break;
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
  __shared__ TileSmem sm;
  const int64_t ntiles = *p.ntiles_dev;
  const int32_t K = *p.count;
  const int64_t Qtot = p.qs[K];
  const uint64_t pol_stream = policy_evict_first();
  const int32_t sent = p.n;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const int64_t T0 = t * SW_TILE_Q;
    const int64_t T1 = min(T0 + (int64_t)SW_TILE_Q, Qtot);
    const int32_t k_lo = p.tfirst[t];
    int32_t k_hi = p.tfirst[t + 1];
    if (k_hi > K - 1) k_hi = K - 1;
    const int nitems = tile_setup(sm, false, p.list, p.qs, p.ooff, T0, T1, k_lo, k_hi);
    if (nitems < 0) break;
    const int nq = (int)(T1 - T0);
    int4 c[SW_QPT];
    int32_t src[SW_QPT];
#pragma unroll
    for (int j = 0; j < SW_QPT; j++) {
      const int q = lane + WARP * (w + (SW_THREADS / WARP) * j);
      c[j] = make_int4(sent, sent, sent, sent);
      src[j] = 0;
      if (q < nq) {
        const int owner = sm.owner[q];
        src[j] = sm.v[owner];
        c[j] = ld_stream4(p.ocol + sm.adj[owner] + 4 * (long long)q, pol_stream);
      }
    }
#pragma unroll
    for (int j = 0; j < SW_QPT; j++) {
      int ws[4] = {c[j].x, c[j].y, c[j].z, c[j].w};
#pragma unroll
      for (int e = 0; e < 4; e++) {
        int32_t wv = ws[e];
        bool cand = wv != sent;
        if (cand && p.ins_src_bits && bit_get(p.ins_src_bits, src[j]))
          cand = !has_key(p.dplus, p.n_dplus, ((uint64_t)src[j] << p.id_bits) | (uint64_t)wv);
        bool add = cand && bit_tas(p.bits, wv);
        int slot = warp_append(p.cnt, add);
        if (add) {
          p.wl[slot] = wv;
          if (p.ever) atomicOr(p.ever + (wv >> 5), 1u << (wv & 31));
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
