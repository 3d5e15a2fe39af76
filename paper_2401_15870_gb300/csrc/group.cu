// group.cu -- one update (Static, ND, DF or DF-P) of many graphs at once.
//
// Every iteration sweeps all graphs of the group that have not converged in
// one launch pair: a gather kernel whose warps walk a work space made of every
// graph's in-CSR quads laid end to end, and an epilogue kernel over every
// graph's 32-vertex chunks laid end to end.  A warp finds the graph of a work
// unit by binary search over a prefix of the per-graph unit counts held in
// shared memory, then runs the same warp step as the single-graph pull sweep
// (pull_step.cuh), so a graph's ranks do not depend on the group it runs in.
// Each graph converges on its own: a one-block control kernel closes the
// iteration of every live graph (L-inf change against tau, iteration count
// against max_iter) and sets the condition of the CUDA graph's WHILE node that
// repeats the iteration, so the whole update runs without a host round trip.
//
// The initial frontier of DF / DF-P (Alg. 1) is expressed in the pull form of
// the frontier, F = S u out(X): X holds the sources of the effective change,
// whose G_t out-neighbours are found by the gather step from the in-rows
// (every source reaches itself through its self-loop), and S holds the
// targets of deleted edges, which completes G_{t-1}.out(u).  Static and ND
// start with every vertex in S and never prune, which makes every iteration a
// full sweep of Eq. 1.
#include <algorithm>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <vector>
#include "dfpr.h"
#include "frontier.cuh"
#include "handle.cuh"
#include "prim.cuh"
#include "pull_step.cuh"
#include "group.cuh"

using namespace dfpr;

namespace {

constexpr int GR_THREADS = 256;
// the unit sizes a group can be set to: quads per lane of a gather warp step
// (32 x QPT quads) and warp steps per gather unit, and 32-vertex chunks of an
// epilogue unit
constexpr int GR_QPT[4] = {2, 4, 8, 2};
constexpr int GR_STEPS[4] = {1, 1, 1, 4};   // warp steps per gather unit (same graph, looked up once)
constexpr int GR_NQ = 4;
constexpr int GR_FU[3] = {1, 2, 4};
// unit sizes of the one-kernel loop (k_g_loop): one gather warp step of 32 x 2
// quads and one epilogue chunk per unit
constexpr int LOOP_QPT = 2;
constexpr int LOOP_FU = 1;

// per graph, fixed during one update
struct GDesc {
  const int32_t* icol;
  const uint32_t* rowbits;
  const int32_t* rowbase;
  int64_t nquads;
  const int32_t* odeg;
  const int32_t* ideg;
  long long* C[2];       // C[0] holds the contributions of the ranks on entry
  double* R;
  long long* acc;
  uint32_t* anyb;
  uint32_t* S[2];
  uint32_t* X[2];
  uint32_t* ever;
  const uint64_t* dmin;
  const uint64_t* dplus;
  int64_t n_dmin, n_dplus;
  int32_t n, id_bits;
  double C0;
  const double2* tab_ab;   // the graph's own Eq. 2 coefficients (its n, the group's alpha)
};

// per graph, written by the loop
struct GState {
  unsigned long long dR;        // this iteration's L-inf change (bits of a non-negative double)
  unsigned long long dR_last;   // of the last finished iteration
  long long edges, verts, ever;
  int32_t cur, iter, done, converged;
  unsigned long long dR_odd;    // the one-kernel loop: odd iterations' change (even ones in dR)
};

// the update: method, tolerances and the work-space prefixes (G + 1 each)
struct GRun {
  double alpha, tau, tau_f, tau_p;
  int32_t max_iter, method, G, loops;
  int32_t metric, pad;
  int32_t live, use_graph;   // loop condition, written to `live` instead of the WHILE node when use_graph is 0
  // the one-kernel loop (k_g_loop): arrivals at its grid barriers (never
  // reset: barrier k completes at k x blocks), the number of the last
  // completed barrier, and 1 when a barrier wait ran out
  uint32_t bar_count, bar_done;
  int32_t err, pad2;
  const int64_t* wpre;   // gather units
  const int64_t* fpre;   // epilogue units (FIN_U chunks)
  const int64_t* bpre;   // bitset words
  const int64_t* dpre;   // changed edges (deletions then insertions)
  const double* tab_sc;
};

// the largest g in [0, G) with pre[g] <= u (pre[0] = 0 <= u < pre[G]); graphs
// with no units of this kind are passed over
__device__ __forceinline__ int find_graph(const int64_t* pre, int G, int64_t u) {
  int lo = 0, hi = G;
  while (hi - lo > 1) {
    int mid = (lo + hi) >> 1;
    if (pre[mid] <= u) lo = mid;
    else hi = mid;
  }
  return lo;
}

__device__ __forceinline__ void load_prefix(int64_t* sm, const int64_t* pre, int G) {
  for (int i = threadIdx.x; i <= G; i += blockDim.x) sm[i] = pre[i];
  __syncthreads();
}

// bitsets of every graph cleared, Static / ND frontiers set to every vertex,
// Static ranks set to 1/n; the loop condition set from max_iter (pre: the
// bitset-word prefix in shared memory)
__device__ __forceinline__ void g_init_phase(const GRun* __restrict__ run, const GDesc* __restrict__ desc,
                                             GState* __restrict__ st, cudaGraphConditionalHandle cond,
                                             const int64_t* pre) {
  const int G = run->G;
  const int method = run->method;
  if (blockIdx.x == 0) {
    for (int g = threadIdx.x; g < G; g += blockDim.x) {
      GState z;
      memset(&z, 0, sizeof(z));
      st[g] = z;
    }
    // the sentinel slot n of both contribution buffers reads as zero
    for (int g = threadIdx.x; g < G; g += blockDim.x) {
      desc[g].C[0][desc[g].n] = 0;
      desc[g].C[1][desc[g].n] = 0;
    }
    if (threadIdx.x == 0 && run->use_graph) cudaGraphSetConditional(cond, run->max_iter > 0 ? 1u : 0u);
  }
  const int lane = threadIdx.x & 31;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int64_t total = pre[G];
  for (int64_t u = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; u < total; u += nw) {
    const int g = find_graph(pre, G, u);
    const GDesc& d = desc[g];
    const int64_t w = u - pre[g];
    const int64_t v = w * 32 + lane;
    const bool valid = v < d.n;
    const unsigned all = __ballot_sync(0xffffffffu, valid);
    if (method == PR_STATIC && valid) {
      const double r = 1.0 / (double)d.n;
      const int32_t dv = d.odeg[v];
      const double sc = dv < TAB ? run->tab_sc[dv] : FIX_ONE / (double)dv;
      d.R[v] = r;
      d.C[0][v] = __double2ll_rn(r * sc);
    }
    if (lane == 0) {
      d.S[0][w] = (method == PR_STATIC || method == PR_NAIVE_DYNAMIC) ? all : 0u;
      d.X[0][w] = 0u;
      d.ever[w] = 0u;
      d.anyb[w] = 0u;
    }
  }
}

__global__ void __launch_bounds__(GR_THREADS) k_g_init(const GRun* __restrict__ run, const GDesc* __restrict__ desc,
                                                       GState* __restrict__ st, cudaGraphConditionalHandle cond) {
  extern __shared__ int64_t pre[];   // G + 1 prefix entries
  load_prefix(pre, run->bpre, run->G);
  g_init_phase(run, desc, st, cond, pre);
}

// DF / DF-P initial frontier: X <- sources of the effective change, S <-
// targets of deleted edges
__device__ __forceinline__ void g_mark_phase(const GRun* __restrict__ run, const GDesc* __restrict__ desc,
                                             const int64_t* pre) {
  const int G = run->G;
  const int64_t total = pre[G];
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    const int g = find_graph(pre, G, i);
    const GDesc& d = desc[g];
    const int64_t k = i - pre[g];
    const bool del = k < d.n_dmin;
    const uint64_t key = del ? d.dmin[k] : d.dplus[k - d.n_dmin];
    const int32_t src = (int32_t)(key >> d.id_bits);
    atomicOr(d.X[0] + (src >> 5), 1u << (src & 31));
    if (del) {
      const int32_t dst = (int32_t)(key & ((1ull << d.id_bits) - 1));
      atomicOr(d.S[0] + (dst >> 5), 1u << (dst & 31));
    }
  }
}

__global__ void __launch_bounds__(GR_THREADS) k_g_mark(const GRun* __restrict__ run, const GDesc* __restrict__ desc) {
  extern __shared__ int64_t pre[];   // G + 1 prefix entries
  if (run->method != PR_DF && run->method != PR_DFP) return;
  load_prefix(pre, run->dpre, run->G);
  g_mark_phase(run, desc, pre);
}

// gather phase of one iteration, every live graph (units of STEPS x 32 x QPT
// quads: STEPS warp steps on one graph per lookup of the graph)
// Where a phase finds a graph's state: whether it is done, the parity of its
// double buffers, and the word its epilogue adds this iteration's change to.
// The kernels of the CUDA graph read the states in device memory, which the
// control kernel writes between launches.
struct StatesInMemory {
  GState* st;
  __device__ __forceinline__ bool done(int g) const { return st[g].done != 0; }
  __device__ __forceinline__ int cur(int g) const { return st[g].cur; }
  __device__ __forceinline__ unsigned long long* dR(int g) const { return &st[g].dR; }
};
// The one-kernel loop: every block keeps each graph's state in shared memory
// (bit 0 done, bit 1 parity, bit 2 converged, iteration count from bit 3) and
// closes each iteration itself from the same changes, so no barrier separates
// the control step from the next gather; the changes of consecutive
// iterations go to two words, so one can be read while the next is cleared.
struct StatesInBlock {
  GState* st;
  const uint32_t* sm;
  int odd;   // parity of the iteration
  __device__ __forceinline__ bool done(int g) const { return sm[g] & 1u; }
  __device__ __forceinline__ int cur(int g) const { return (sm[g] >> 1) & 1u; }
  __device__ __forceinline__ unsigned long long* dR(int g) const { return odd ? &st[g].dR_odd : &st[g].dR; }
};

// COH: inside the one-kernel loop, where contributions and frontier words
// were written earlier in the same launch
template <int QPT, int STEPS, bool COH, class SV>
__device__ __forceinline__ void g_gather_phase(const GRun* __restrict__ run, const GDesc* __restrict__ desc,
                                               const SV& sv, const int64_t* pre) {
  const int G = run->G;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int64_t total = pre[G];
  const uint64_t pol_stream = policy_evict_first();
  const uint64_t pol_keep = policy_evict_last();
  for (int64_t u = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; u < total; u += nw) {
    const int g = find_graph(pre, G, u);
    if (sv.done(g)) continue;
    const GDesc& d = desc[g];
    const int c = sv.cur(g);
    const int64_t ub = (u - pre[g]) * (STEPS * 32 * QPT);
#pragma unroll 1
    for (int k = 0; k < STEPS; k++) {
      const int64_t base = ub + k * (32 * QPT);
      if (base >= d.nquads) break;
      gather_step<true, QPT, false, false, COH>(d.icol, d.C[c], d.X[c], d.S[c], d.rowbits, d.rowbase, d.nquads, d.n,
                                                d.acc, d.anyb, base, pol_stream, pol_keep);
    }
  }
}

template <int QPT, int STEPS>
__global__ void __launch_bounds__(GR_THREADS) k_g_gather(const GRun* __restrict__ run, const GDesc* __restrict__ desc,
                                                         const GState* __restrict__ st) {
  extern __shared__ int64_t pre[];   // G + 1 prefix entries
  load_prefix(pre, run->wpre, run->G);
  g_gather_phase<QPT, STEPS, false>(run, desc, StatesInMemory{const_cast<GState*>(st)}, pre);
}

// the fields finish_pull_step reads, for one graph and one parity
struct GView {
  int32_t n;
  const int32_t* odeg;
  const int32_t* ideg;
  double* R;
  const long long* Ccur;
  long long* Cnext;
  const uint32_t* S_cur;
  uint32_t* S_next;
  uint32_t* X_next;
  uint32_t* ever;
  const double* tab_sc;
  const double2* tab_ab;
  double alpha, C0, tau_f, tau_p;
  int32_t metric;
};

__device__ __forceinline__ void flush_totals(PullTotals& t, GState* s, unsigned long long* dRw) {
  const int lane = threadIdx.x & 31;
  unsigned long long dm = t.dmax;
  long long e = t.edges, v = t.verts;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    unsigned long long odm = __shfl_xor_sync(0xffffffffu, dm, o);
    dm = odm > dm ? odm : dm;
    e += __shfl_xor_sync(0xffffffffu, e, o);
    v += __shfl_xor_sync(0xffffffffu, v, o);
  }
  if (lane == 0) {
    if (dm) atomicMax(dRw, dm);
    if (e) atomicAdd(reinterpret_cast<unsigned long long*>(&s->edges), (unsigned long long)e);
    if (v) atomicAdd(reinterpret_cast<unsigned long long*>(&s->verts), (unsigned long long)v);
    if (t.ever_new) atomicAdd(reinterpret_cast<unsigned long long*>(&s->ever), (unsigned long long)t.ever_new);
  }
  t = PullTotals();
}

// epilogue phase of one iteration, every live graph, units of FU chunks
// (Eq. 2 for DF-P when CLOSED, else Eq. 1)
template <bool CLOSED, int FU, bool REL, bool COH, class SV>
__device__ __forceinline__ void g_finish_phase(const GRun* __restrict__ run, const GDesc* __restrict__ desc,
                                               const SV& sv, const int64_t* pre) {
  const int G = run->G;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int64_t total = pre[G];
  PullTotals t;
  int tg = -1;   // graph the totals belong to
  for (int64_t u = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; u < total; u += nw) {
    const int g = find_graph(pre, G, u);
    if (sv.done(g)) continue;
    if (g != tg) {
      if (tg >= 0) flush_totals(t, sv.st + tg, sv.dR(tg));
      tg = g;
    }
    const GDesc& d = desc[g];
    const int c = sv.cur(g);
    GView p;
    p.n = d.n;
    p.odeg = d.odeg;
    p.ideg = d.ideg;
    p.R = d.R;
    p.Ccur = d.C[c];
    p.Cnext = d.C[c ^ 1];
    p.S_cur = d.S[c];
    p.S_next = d.S[c ^ 1];
    p.X_next = d.X[c ^ 1];
    p.ever = d.ever;
    p.tab_sc = run->tab_sc;
    p.tab_ab = d.tab_ab;
    p.alpha = run->alpha;
    p.C0 = d.C0;
    p.tau_f = run->tau_f;
    p.tau_p = run->tau_p;
    p.metric = run->metric;
    const int64_t nchunks = cdiv(d.n, 32);
    const int64_t ch0 = (u - pre[g]) * FU;
    finish_pull_step<CLOSED, GView, false, FU, REL, false, COH>(p, d.acc, d.anyb, ch0, nchunks, t);
  }
  if (tg >= 0) flush_totals(t, sv.st + tg, sv.dR(tg));
}

template <bool CLOSED, int FU, bool REL>
__global__ void __launch_bounds__(GR_THREADS, 2) k_g_finish(const GRun* __restrict__ run,
                                                            const GDesc* __restrict__ desc, GState* __restrict__ st) {
  extern __shared__ int64_t pre[];   // G + 1 prefix entries
  load_prefix(pre, run->fpre, run->G);
  g_finish_phase<CLOSED, FU, REL, false>(run, desc, StatesInMemory{st}, pre);
}

// close the iteration of every live graph; loop while any is live (one block)
__global__ void k_g_control(GRun* run, GState* st, cudaGraphConditionalHandle cond) {
  __shared__ int live;
  if (threadIdx.x == 0) live = 0;
  __syncthreads();
  const double tau = run->tau;
  for (int g = threadIdx.x; g < run->G; g += blockDim.x) {
    GState& s = st[g];
    if (s.done) continue;
    s.iter += 1;
    s.cur ^= 1;
    s.dR_last = s.dR;
    s.dR = 0ull;
    const double dR = __longlong_as_double((long long)s.dR_last);
    if (dR <= tau) {
      s.converged = 1;
      s.done = 1;
    } else if (s.iter >= run->max_iter) {
      s.done = 1;
    } else {
      live = 1;
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    run->loops += 1;
    // every graph is done after max_iter iterations; the guard bounds the loop
    // even if a state were corrupted
    const unsigned go = (live && run->loops < run->max_iter) ? 1u : 0u;
    run->live = (int32_t)go;
    if (run->use_graph) cudaGraphSetConditional(cond, go);
  }
}


// ------------------------------------------------------------------ the whole loop in one kernel
//
// For groups whose sweeps take a few microseconds, the launches of the CUDA
// graph (three kernels per iteration) cost more than the work.  k_g_loop runs
// init, mark and every iteration's gather, epilogue and control in one
// cooperative launch (every block resident), the phases separated by grid
// barriers.  Same phase code, same arithmetic: the ranks and statistics are
// bit-identical to the CUDA graph's.  Data written in an earlier phase is read
// from L2 (COH), never through the read-only path.

// iterations of a barrier wait before it gives up (after the first 4096 each
// with a short sleep: about a second in all, against microseconds when every
// block runs)
constexpr long long BAR_SPINS = 1ll << 24;
// resident blocks per SM of the one-kernel loop, at most: fewer blocks make
// the barriers cheaper (one arrival each), more make the phases of larger
// graphs faster.  One per SM: R-MAT graphs of 2^8 to 2^14 vertices update
// 4-8% faster than with two, and the loop is the default only below
// PR_ONE_KERNEL_SLOTS, where it beats the CUDA graph (equal at about 2^20)
constexpr int LOOP_BPS = 1;

__device__ __forceinline__ uint32_t ld_acquire_u32(const uint32_t* p) {
  uint32_t v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// barrier number `k` (1, 2, ...) over the grid's blocks.  False when a wait
// ran out, here or in another block (run->err set): the caller returns.
__device__ __forceinline__ bool grid_barrier(GRun* run, uint32_t k) {
  __shared__ int ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    int good = 1;
    __threadfence();   // this block's writes before the arrival
    const uint32_t arrived = atomicAdd(&run->bar_count, 1u) + 1u;
    if (arrived == k * gridDim.x) {
      __threadfence();
      atomicExch(&run->bar_done, k);
    } else {
      long long spins = 0;
      while (ld_acquire_u32(&run->bar_done) < k) {
        if (*(volatile int32_t*)&run->err) {
          good = 0;
          break;
        }
        if (++spins > BAR_SPINS) {
          atomicExch(&run->err, 1);
          good = 0;
          break;
        }
        if (spins > 4096) __nanosleep(64);   // poll at full rate for the first few microseconds
      }
    }
    __threadfence();
    ok = good;
  }
  __syncthreads();
  return ok != 0;
}

// Every block closes iteration `it` of every live graph from the changes in
// the word of its parity, with the same arithmetic as k_g_control, so all
// blocks hold the same states; block 0 also writes them to device memory for
// the host.  Returns whether any graph is still live.
__device__ __forceinline__ bool loop_control(GRun* run, GState* st, uint32_t* sm, int it) {
  __shared__ int live;
  if (threadIdx.x == 0) live = 0;
  __syncthreads();
  const double tau = run->tau;
  for (int g = threadIdx.x; g < run->G; g += blockDim.x) {
    uint32_t w = sm[g];
    if (w & 1u) continue;
    const unsigned long long dRb = __ldcg((it & 1) ? &st[g].dR_odd : &st[g].dR);
    const uint32_t iter = (w >> 3) + 1;
    uint32_t cur = ((w >> 1) & 1u) ^ 1u, done = 0, conv = 0;
    const double dR = __longlong_as_double((long long)dRb);
    if (dR <= tau) {
      conv = 1;
      done = 1;
    } else if ((int32_t)iter >= run->max_iter) {
      done = 1;
    } else {
      live = 1;
    }
    sm[g] = (iter << 3) | (conv << 2) | (cur << 1) | done;
    if (blockIdx.x == 0) {
      GState& s = st[g];
      s.iter = (int32_t)iter;
      s.cur = (int32_t)cur;
      s.done = (int32_t)done;
      s.converged = (int32_t)conv;
      s.dR_last = dRb;
    }
  }
  __syncthreads();
  return live != 0;
}

// shared memory: the four prefixes (gather units, epilogue units, bitset
// words, changed edges; G + 1 entries each), then the G packed states
template <bool CLOSED, bool REL>
__global__ void __launch_bounds__(GR_THREADS, 2) k_g_loop(GRun* run, const GDesc* __restrict__ desc, GState* st) {
  extern __shared__ int64_t pre[];
  const int G = run->G;
  uint32_t* sm = reinterpret_cast<uint32_t*>(pre + 4 * (G + 1));
  for (int i = threadIdx.x; i <= G; i += blockDim.x) {
    pre[i] = run->wpre[i];
    pre[(G + 1) + i] = run->fpre[i];
    pre[2 * (G + 1) + i] = run->bpre[i];
    pre[3 * (G + 1) + i] = run->dpre[i];
    if (i < G) sm[i] = 0u;
  }
  __syncthreads();
  uint32_t k = 0;
  g_init_phase(run, desc, st, 0, pre + 2 * (G + 1));   // zeroes every state, both change words included
  if (!grid_barrier(run, ++k)) return;
  if (run->method == PR_DF || run->method == PR_DFP) {
    g_mark_phase(run, desc, pre + 3 * (G + 1));
    if (!grid_barrier(run, ++k)) return;
  }
  int32_t loops = 0;
  bool live = run->max_iter > 0;
  for (int32_t it = 0; live; it++) {
    const StatesInBlock sv{st, sm, it & 1};
    g_gather_phase<LOOP_QPT, 1, true>(run, desc, sv, pre);
    if (!grid_barrier(run, ++k)) return;
    // the word of the next iteration's changes was last read by every block's
    // control step of the iteration before this one, which the barrier above
    // follows: clear it for the next epilogue
    if (blockIdx.x == 0)
      for (int g = threadIdx.x; g < G; g += blockDim.x) *((it & 1) ? &st[g].dR : &st[g].dR_odd) = 0ull;
    g_finish_phase<CLOSED, LOOP_FU, REL, true>(run, desc, sv, pre + (G + 1));
    if (!grid_barrier(run, ++k)) return;
    live = loop_control(run, st, sm, it);
    loops += 1;
    // every graph is done after max_iter iterations; the guard bounds the
    // loop even if a state were corrupted
    if (loops >= run->max_iter) live = false;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    run->loops = loops;
    run->live = 0;
  }
}

}  // namespace

struct pr_group {
  int32_t G = 0;
  std::vector<pr_graph*> graphs;
  int dev = 0;
  cudaStream_t stream = nullptr;
  // device: run, descriptors, states, prefixes (4 x (G + 1)), tables
  GRun* d_run = nullptr;
  GDesc* d_desc = nullptr;
  GState* d_state = nullptr;
  int64_t* d_pre = nullptr;
  double* tab_sc = nullptr;
  double tab_alpha = -1.0;
  // pinned host staging
  GRun* h_run = nullptr;
  GDesc* h_desc = nullptr;
  GState* h_state = nullptr;
  int64_t* h_pre = nullptr;
  // unit sizes (indices into GR_QPT and GR_STEPS / GR_FU), set by pr_group_set_tuning or
  // pr_group_autotune
  int qi = 1, fi = 2;
  float tune_ms = 0.f;
  int32_t tune_trials = 0;
  // one CUDA graph per epilogue form (index 1: DF-P), built on first use with
  // the unit sizes of exec_q / exec_f
  cudaGraph_t graph[2] = {nullptr, nullptr};
  cudaGraphExec_t exec[2] = {nullptr, nullptr};
  int exec_q[2] = {-1, -1}, exec_f[2] = {-1, -1}, exec_rel[2] = {-1, -1};
  cudaGraphConditionalHandle cond[2] = {0, 0};
  cudaEvent_t ev[3] = {nullptr, nullptr, nullptr};
  // resident blocks per SM of the one-kernel loop [form][relative measure], 0 until asked
  int loop_bps[2][2] = {{0, 0}, {0, 0}};
  // the update in flight: its members (group indices) and method
  std::vector<int32_t> members;
  bool in_flight = false;
  pr_method cur_method = PR_DFP;
};

static void drop_exec(pr_group* q, int k);

static void group_free(pr_group* q) {
  if (!q) return;
  if (q->stream) cudaStreamSynchronize(q->stream);
  for (int k = 0; k < 2; k++) drop_exec(q, k);
  for (void* p : {(void*)q->d_run, (void*)q->d_desc, (void*)q->d_state, (void*)q->d_pre, (void*)q->tab_sc})
    if (p) cudaFree(p);
  for (void* p : {(void*)q->h_run, (void*)q->h_desc, (void*)q->h_state, (void*)q->h_pre})
    if (p) cudaFreeHost(p);
  for (cudaEvent_t e : q->ev)
    if (e) cudaEventDestroy(e);
  delete q;
}

static int blocks_per_sm(const void* fn, int threads, size_t smem) {
  int b = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, fn, threads, smem) != cudaSuccess || b < 1) b = 1;
  return b;
}

// shared memory of the kernels that look a unit's graph up: the prefix of
// per-graph unit counts of at most the group's G graphs
static size_t prefix_bytes(const pr_group* q) { return sizeof(int64_t) * (size_t)(q->G + 1); }

static cudaError_t add_kernel(cudaGraph_t graph, cudaGraphNode_t* node, const cudaGraphNode_t* dep, size_t ndep,
                              const void* fn, int grid, void** args, size_t smem) {
  cudaKernelNodeParams kp;
  memset(&kp, 0, sizeof(kp));
  kp.func = const_cast<void*>(fn);
  kp.gridDim = dim3(grid);
  kp.blockDim = dim3(GR_THREADS);
  kp.sharedMemBytes = (unsigned)smem;
  kp.kernelParams = args;
  return cudaGraphAddKernelNode(node, graph, dep, ndep, &kp);
}

static const void* gather_fn(int qi) {
  switch (qi) {
    case 0: return (const void*)k_g_gather<2, 1>;
    case 1: return (const void*)k_g_gather<4, 1>;
    case 2: return (const void*)k_g_gather<8, 1>;
    default: return (const void*)k_g_gather<2, 4>;
  }
}

// epilogue kernel for form k (1: DF-P), unit-size index fi, and whether the
// measure is the relative change of Alg. 1 (compiled in) or chosen at run time
static const void* finish_fn(int k, int fi, bool rel) {
  if (rel) {
    switch (fi * 2 + k) {
      case 0: return (const void*)k_g_finish<false, 1, true>;
      case 1: return (const void*)k_g_finish<true, 1, true>;
      case 2: return (const void*)k_g_finish<false, 2, true>;
      case 3: return (const void*)k_g_finish<true, 2, true>;
      case 4: return (const void*)k_g_finish<false, 4, true>;
      default: return (const void*)k_g_finish<true, 4, true>;
    }
  }
  switch (fi * 2 + k) {
    case 0: return (const void*)k_g_finish<false, 1, false>;
    case 1: return (const void*)k_g_finish<true, 1, false>;
    case 2: return (const void*)k_g_finish<false, 2, false>;
    case 3: return (const void*)k_g_finish<true, 2, false>;
    case 4: return (const void*)k_g_finish<false, 4, false>;
    default: return (const void*)k_g_finish<true, 4, false>;
  }
}

static void drop_exec(pr_group* q, int k) {
  if (q->exec[k]) cudaGraphExecDestroy(q->exec[k]);
  if (q->graph[k]) cudaGraphDestroy(q->graph[k]);
  q->exec[k] = nullptr;
  q->graph[k] = nullptr;
  q->exec_q[k] = q->exec_f[k] = q->exec_rel[k] = -1;
}

// init -> mark -> WHILE (gather -> finish -> control); k = 1 for the DF-P epilogue
static cudaError_t build_exec(pr_group* q, int k, bool rel) {
  cudaError_t e;
  cudaGraph_t& graph = q->graph[k];
  if ((e = cudaGraphCreate(&graph, 0)) != cudaSuccess) return e;
  if ((e = cudaGraphConditionalHandleCreate(&q->cond[k], graph, 0, 0)) != cudaSuccess) return e;
  const void* fin = finish_fn(k, q->fi, rel);
  const void* gat = gather_fn(q->qi);
  q->exec_q[k] = q->qi;
  q->exec_f[k] = q->fi;
  q->exec_rel[k] = rel ? 1 : 0;
  const int sms = num_sms();
  const size_t sm = prefix_bytes(q);
  const int g_init = sms * blocks_per_sm((const void*)k_g_init, GR_THREADS, sm);
  const int g_gather = sms * blocks_per_sm(gat, GR_THREADS, sm);
  const int g_finish = sms * blocks_per_sm(fin, GR_THREADS, sm);
  cudaGraphNode_t n_init, n_mark, n_loop, n_gather, n_finish, n_ctl;
  void* a_init[] = {&q->d_run, &q->d_desc, &q->d_state, &q->cond[k]};
  void* a_mark[] = {&q->d_run, &q->d_desc};
  void* a_gather[] = {&q->d_run, &q->d_desc, &q->d_state};
  void* a_finish[] = {&q->d_run, &q->d_desc, &q->d_state};
  void* a_ctl[] = {&q->d_run, &q->d_state, &q->cond[k]};
  if ((e = add_kernel(graph, &n_init, nullptr, 0, (const void*)k_g_init, g_init, a_init, sm)) != cudaSuccess) return e;
  if ((e = add_kernel(graph, &n_mark, &n_init, 1, (const void*)k_g_mark, g_init, a_mark, sm)) != cudaSuccess) return e;
  cudaGraphNodeParams cp = {};
  cp.type = cudaGraphNodeTypeConditional;
  cp.conditional.handle = q->cond[k];
  cp.conditional.type = cudaGraphCondTypeWhile;
  cp.conditional.size = 1;
  if ((e = cudaGraphAddNode(&n_loop, graph, &n_mark, nullptr, 1, &cp)) != cudaSuccess) return e;
  cudaGraph_t body = cp.conditional.phGraph_out[0];
  if ((e = add_kernel(body, &n_gather, nullptr, 0, gat, g_gather, a_gather, sm)) != cudaSuccess) return e;
  if ((e = add_kernel(body, &n_finish, &n_gather, 1, fin, g_finish, a_finish, sm)) != cudaSuccess) return e;
  cudaKernelNodeParams kp;
  memset(&kp, 0, sizeof(kp));
  kp.func = (void*)k_g_control;
  kp.gridDim = dim3(1);
  kp.blockDim = dim3(GR_THREADS);
  kp.kernelParams = a_ctl;
  if ((e = cudaGraphAddKernelNode(&n_ctl, body, &n_finish, 1, &kp)) != cudaSuccess) return e;
  return cudaGraphInstantiate(&q->exec[k], graph, 0);
}

extern "C" {

pr_status pr_group_create(int32_t count, pr_graph* const* graphs, void* stream, pr_group** out) {
  if (!out) return PR_EINVAL;
  *out = nullptr;
  if (count < 1 || count > PR_GROUP_MAX || !graphs) return PR_EINVAL;
  int dev = -1;
  for (int32_t i = 0; i < count; i++) {
    if (!graphs[i]) return PR_EINVAL;
    for (int32_t j = 0; j < i; j++)
      if (graphs[j] == graphs[i]) return PR_EINVAL;   // each graph once
    if (i == 0) dev = graphs[i]->g.dev;
    else if (graphs[i]->g.dev != dev) return PR_EINVAL;
  }
  int cur = 0;
  if (cudaGetDevice(&cur) != cudaSuccess || cur != dev) return PR_EINVAL;
  pr_group* q = new (std::nothrow) pr_group();
  if (!q) return PR_ENOMEM;
  q->G = count;
  q->graphs.assign(graphs, graphs + count);
  q->dev = dev;
  q->stream = (cudaStream_t)stream;
  const size_t pre_elems = 4 * (size_t)(count + 1);
  bool ok = dev_malloc((void**)&q->d_run, sizeof(GRun)) == cudaSuccess &&
            dev_malloc((void**)&q->d_desc, sizeof(GDesc) * count) == cudaSuccess &&
            dev_malloc((void**)&q->d_state, sizeof(GState) * count) == cudaSuccess &&
            dev_malloc((void**)&q->d_pre, sizeof(int64_t) * pre_elems) == cudaSuccess &&
            dev_malloc((void**)&q->tab_sc, sizeof(double) * TAB) == cudaSuccess &&
            cudaMallocHost((void**)&q->h_run, sizeof(GRun)) == cudaSuccess &&
            cudaMallocHost((void**)&q->h_desc, sizeof(GDesc) * count) == cudaSuccess &&
            cudaMallocHost((void**)&q->h_state, sizeof(GState) * count) == cudaSuccess &&
            cudaMallocHost((void**)&q->h_pre, sizeof(int64_t) * pre_elems) == cudaSuccess;
  for (int i = 0; ok && i < 3; i++) ok = cudaEventCreate(&q->ev[i]) == cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    group_free(q);
    return PR_ENOMEM;
  }
  *out = q;
  return PR_OK;
}

void pr_group_destroy(pr_group* q) { group_free(q); }

}  // extern "C"

static const void* loop_fn(int k, bool rel) {
  if (rel) return k ? (const void*)k_g_loop<true, true> : (const void*)k_g_loop<false, true>;
  return k ? (const void*)k_g_loop<true, false> : (const void*)k_g_loop<false, false>;
}

// the whole update as one cooperative launch of every resident block.  Two
// such grids launched from different streams at once could each hold part of
// the SMs while waiting at a barrier for blocks that the other keeps out, so
// every launch of the process is ordered after the previous one on the
// device (an event per device; the host does not wait)
static cudaError_t launch_one_kernel(pr_group* q, int k, bool rel) {
  static std::mutex mu;
  static std::map<int, cudaEvent_t> last;
  const void* fn = loop_fn(k, rel);
  const size_t smem = 4 * prefix_bytes(q) + sizeof(uint32_t) * (size_t)q->G;
  int& bps = q->loop_bps[k][rel ? 1 : 0];
  if (bps == 0) {
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, fn, GR_THREADS, smem);
    if (e != cudaSuccess) return e;
    if (bps < 1) return cudaErrorInvalidConfiguration;
    bps = std::min(bps, LOOP_BPS);
  }
  void* args[] = {&q->d_run, &q->d_desc, &q->d_state};
  std::lock_guard<std::mutex> lock(mu);
  cudaEvent_t& ev = last[q->dev];
  cudaError_t e = cudaSuccess;
  if (!ev) e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
  else e = cudaStreamWaitEvent(q->stream, ev, 0);
  if (e != cudaSuccess) return e;
  note_launch();
  e = cudaLaunchCooperativeKernel(fn, dim3(num_sms() * bps), dim3(GR_THREADS), args, smem, q->stream);
  if (e != cudaSuccess) return e;
  return cudaEventRecord(ev, q->stream);
}

// the same kernels launched one by one, the loop condition read back after
// every iteration (PR_OPT_HOST_LOOP): for profilers that cannot see into a
// CUDA graph with conditional nodes, and for drivers without them
static cudaError_t host_loop(pr_group* q, int k, int32_t max_iter, bool rel) {
  cudaStream_t s = q->stream;
  const int sms = num_sms();
  const void* fin = finish_fn(k, q->fi, rel);
  const void* gat = gather_fn(q->qi);
  const size_t sm = prefix_bytes(q);
  const int g_init = sms * blocks_per_sm((const void*)k_g_init, GR_THREADS, sm);
  const int g_gather = sms * blocks_per_sm(gat, GR_THREADS, sm);
  const int g_finish = sms * blocks_per_sm(fin, GR_THREADS, sm);
  const cudaGraphConditionalHandle none = 0;
  void* a3[] = {&q->d_run, &q->d_desc, &q->d_state};
  note_launch();
  k_g_init<<<g_init, GR_THREADS, sm, s>>>(q->d_run, q->d_desc, q->d_state, none);
  note_launch();
  k_g_mark<<<g_init, GR_THREADS, sm, s>>>(q->d_run, q->d_desc);
  for (int32_t it = 0; it < max_iter; it++) {
    note_launch();
    cudaError_t le = cudaLaunchKernel(gat, dim3(g_gather), dim3(GR_THREADS), a3, sm, s);
    if (le != cudaSuccess) return le;
    note_launch();
    le = cudaLaunchKernel(fin, dim3(g_finish), dim3(GR_THREADS), a3, sm, s);
    if (le != cudaSuccess) return le;
    note_launch();
    k_g_control<<<1, GR_THREADS, 0, s>>>(q->d_run, q->d_state, none);
    cudaError_t e = cudaMemcpyAsync(&q->h_run->live, &q->d_run->live, sizeof(int32_t), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return e;
    if (!q->h_run->live) break;
  }
  return cudaGetLastError();
}

// launch an update of the members (indices into the group; NULL: every graph)
// on the group's stream without waiting for it
pr_status group_launch(pr_group* q, pr_method method, double alpha, double tau, const pr_options* opts,
                       const int32_t* members, int32_t nm) {
  if (!q || q->in_flight) return PR_EINVAL;
  if (method != PR_STATIC && method != PR_NAIVE_DYNAMIC && method != PR_DF && method != PR_DFP) return PR_EINVAL;
  if (!(alpha >= 0.0 && alpha < 1.0) || !(tau >= 0.0)) return PR_EINVAL;
  pr_options o = {1e-6, 1e-6, 500, 0};
  if (opts) o = *opts;
  if (!(o.tau_f >= 0.0) || !(o.tau_p >= 0.0) || o.max_iter < 0) return PR_EINVAL;
  if (o.flags &
      ~(PR_OPT_HOST_LOOP | PR_OPT_DEVICE_LOOP | PR_OPT_ONE_KERNEL | PR_OPT_MEASURE_ABSOLUTE | PR_OPT_MEASURE_CONTRIB))
    return PR_EINVAL;
  const int loops_asked = !!(o.flags & PR_OPT_HOST_LOOP) + !!(o.flags & PR_OPT_DEVICE_LOOP) + !!(o.flags & PR_OPT_ONE_KERNEL);
  if (loops_asked > 1) return PR_EINVAL;
  if ((o.flags & PR_OPT_MEASURE_ABSOLUTE) && (o.flags & PR_OPT_MEASURE_CONTRIB)) return PR_EINVAL;
  std::vector<int32_t>& mem = q->members;
  mem.clear();
  if (members) {
    if (nm < 1 || nm > q->G) return PR_EINVAL;
    std::vector<char> seen(q->G, 0);
    for (int32_t i = 0; i < nm; i++) {
      if (members[i] < 0 || members[i] >= q->G || seen[members[i]]) return PR_EINVAL;
      seen[members[i]] = 1;
      mem.push_back(members[i]);
    }
  } else {
    for (int32_t i = 0; i < q->G; i++) mem.push_back(i);
  }
  const int G = (int)mem.size();
  if (method != PR_STATIC)
    for (int i = 0; i < G; i++)
      if (!q->graphs[mem[i]]->g.has_ranks) return PR_ENORANKS;
  cudaStream_t s = q->stream;
  // the loop in one kernel when asked, or by default when the sweeps are short
  int64_t slots = 0;
  for (int i = 0; i < G; i++) slots += q->graphs[mem[i]]->g.in.cap;
  const bool one = (o.flags & PR_OPT_ONE_KERNEL) || (loops_asked == 0 && slots < PR_ONE_KERNEL_SLOTS);
  const int64_t gq = one ? 32 * LOOP_QPT : 32 * GR_QPT[q->qi] * GR_STEPS[q->qi];   // quads per gather unit
  const int64_t fu = one ? LOOP_FU : GR_FU[q->fi];                                 // chunks per epilogue unit
  int64_t* wpre = q->h_pre;
  int64_t* fpre = wpre + (G + 1);
  int64_t* bpre = fpre + (G + 1);
  int64_t* dpre = bpre + (G + 1);
  wpre[0] = fpre[0] = bpre[0] = dpre[0] = 0;
  for (int i = 0; i < G; i++) {
    Graph* g = &q->graphs[mem[i]]->g;
    GDesc& d = q->h_desc[i];
    memset(&d, 0, sizeof(d));
    d.icol = g->in.col;
    d.rowbits = g->rowbits;
    d.rowbase = g->rowbase;
    d.nquads = g->in.cap >> 2;
    d.odeg = g->out.deg;
    d.ideg = g->in.deg;
    d.C[0] = g->C[g->ccur];
    d.C[1] = g->C[g->ccur ^ 1];
    d.R = g->R;
    d.acc = g->gacc;
    d.anyb = g->anyb;
    d.S[0] = g->bits[0];
    d.S[1] = g->bits[1];
    d.X[0] = g->aux;
    d.X[1] = g->aux2;
    d.ever = g->ever;
    d.dmin = g->dmin;
    d.dplus = g->dplus;
    d.n_dmin = g->n_dmin;
    d.n_dplus = g->n_dplus;
    d.n = g->n;
    d.id_bits = g->id_bits;
    d.C0 = (1.0 - alpha) / (double)g->n;
    d.tab_ab = g->tab_ab;
    wpre[i + 1] = wpre[i] + cdiv(d.nquads, gq);
    fpre[i + 1] = fpre[i] + cdiv(cdiv((int64_t)g->n, 32), fu);
    bpre[i + 1] = bpre[i] + cdiv((int64_t)g->n, 32);
    dpre[i + 1] = dpre[i] + ((method == PR_DF || method == PR_DFP) ? g->n_dmin + g->n_dplus : 0);
  }
  GRun& r = *q->h_run;
  memset(&r, 0, sizeof(r));
  r.alpha = alpha;
  r.tau = tau;
  r.tau_f = o.tau_f;
  r.tau_p = o.tau_p;
  r.max_iter = o.max_iter;
  r.method = (int32_t)method;
  r.G = G;
  r.loops = 0;
  r.wpre = q->d_pre;
  r.fpre = q->d_pre + (G + 1);
  r.bpre = q->d_pre + 2 * (G + 1);
  r.dpre = q->d_pre + 3 * (G + 1);
  r.tab_sc = q->tab_sc;
  r.use_graph = (o.flags & PR_OPT_HOST_LOOP) || one ? 0 : 1;
  r.metric = (o.flags & PR_OPT_MEASURE_ABSOLUTE) ? METRIC_ABSOLUTE
             : (o.flags & PR_OPT_MEASURE_CONTRIB) ? METRIC_CONTRIB
                                                  : METRIC_RELATIVE;

  // order after the work already queued on the members' streams
  for (int i = 0; i < G; i++) {
    cudaStream_t gs = q->graphs[mem[i]]->g.stream;
    if (gs == s) continue;
    if (cudaEventRecord(q->ev[2], gs) != cudaSuccess || cudaStreamWaitEvent(s, q->ev[2], 0) != cudaSuccess)
      return PR_ECUDA;
  }
  if (cudaEventRecord(q->ev[0], s) != cudaSuccess) return PR_ECUDA;
  if (q->tab_alpha != alpha) {
    if (launch_tables(q->tab_sc, nullptr, alpha, 1, s) != cudaSuccess) return PR_ECUDA;
    q->tab_alpha = alpha;
  }
  // each member's own Eq. 2 coefficients for this alpha (after the work
  // already queued on its stream, which the waits above order before s)
  for (int i = 0; i < G; i++) {
    Graph* g = &q->graphs[mem[i]]->g;
    if (g->tab_alpha != alpha) {
      if (launch_tables(g->tab_sc, g->tab_ab, alpha, g->n, s) != cudaSuccess) return PR_ECUDA;
      g->tab_alpha = alpha;
    }
  }
  if (cudaMemcpyAsync(q->d_pre, q->h_pre, sizeof(int64_t) * 4 * (size_t)(G + 1), cudaMemcpyHostToDevice, s) !=
          cudaSuccess ||
      cudaMemcpyAsync(q->d_desc, q->h_desc, sizeof(GDesc) * G, cudaMemcpyHostToDevice, s) != cudaSuccess ||
      cudaMemcpyAsync(q->d_run, q->h_run, sizeof(GRun), cudaMemcpyHostToDevice, s) != cudaSuccess)
    return PR_ECUDA;
  const int k = method == PR_DFP ? 1 : 0;
  if (one) {
    if (launch_one_kernel(q, k, r.metric == METRIC_RELATIVE) != cudaSuccess) {
      cudaGetLastError();
      return PR_ECUDA;
    }
  } else if (r.use_graph) {
    const int rel = r.metric == METRIC_RELATIVE ? 1 : 0;
    if (q->exec[k] && (q->exec_q[k] != q->qi || q->exec_f[k] != q->fi || q->exec_rel[k] != rel)) drop_exec(q, k);
    if (!q->exec[k] && build_exec(q, k, rel != 0) != cudaSuccess) {
      cudaGetLastError();
      return PR_ECUDA;
    }
    if (cudaGraphLaunch(q->exec[k], s) != cudaSuccess) return PR_ECUDA;
  } else if (host_loop(q, k, o.max_iter, r.metric == METRIC_RELATIVE) != cudaSuccess) {
    return PR_ECUDA;
  }
  if (cudaMemcpyAsync(q->h_state, q->d_state, sizeof(GState) * G, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaMemcpyAsync(q->h_run, q->d_run, sizeof(GRun), cudaMemcpyDeviceToHost, s) != cudaSuccess)
    return PR_ECUDA;
  if (cudaEventRecord(q->ev[1], s) != cudaSuccess) return PR_ECUDA;
  q->in_flight = true;
  q->cur_method = method;
  return PR_OK;
}

// true when the launched update has finished (does not block)
bool group_done(pr_group* q) { return !q->in_flight || cudaEventQuery(q->ev[1]) != cudaErrorNotReady; }

// wait for the launched update; stats (NULL or one entry per graph of the
// group, by group index) are written for the members
pr_status group_complete(pr_group* q, pr_stats* stats) {
  if (!q || !q->in_flight) return PR_EINVAL;
  q->in_flight = false;
  if (cudaEventSynchronize(q->ev[1]) != cudaSuccess) return PR_ECUDA;
  const pr_method method = q->cur_method;
  if (q->h_run->err) {
    // a grid barrier of the one-kernel loop gave up: the ranks are partial
    for (int32_t gi : q->members) q->graphs[gi]->g.has_ranks = false;
    return PR_ETIMEOUT;
  }
  float ms = 0.f;
  cudaEventElapsedTime(&ms, q->ev[0], q->ev[1]);
  // kernels the CUDA graph ran: init, mark, and three per loop pass (the host
  // loop counted its launches itself)
  if (q->h_run->use_graph) note_launches(2ull + 3ull * (unsigned long long)q->h_run->loops);
  for (size_t i = 0; i < q->members.size(); i++) {
    const int32_t gi = q->members[i];
    pr_graph* h = q->graphs[gi];
    Graph* g = &h->g;
    const GState& st = q->h_state[i];
    if (st.cur) g->ccur ^= 1;
    g->has_ranks = true;
    if (stats) {
      pr_stats& o2 = stats[gi];
      memset(&o2, 0, sizeof(o2));
      double dR;
      memcpy(&dR, &st.dR_last, sizeof(dR));
      o2.iterations = st.iter;
      o2.converged = st.converged;
      o2.delta_R = st.iter ? dR : 0.0;
      o2.vertices_ever_affected =
          (method == PR_DF || method == PR_DFP) ? st.ever : (st.iter > 0 ? (int64_t)g->n : 0);
      o2.edges_processed = st.edges;
      o2.vertices_processed = st.verts;
      o2.eff_deletions = g->n_dmin;
      o2.eff_insertions = g->n_dplus;
      o2.ms_apply = h->ms_apply;
      o2.ms_update = ms;
      o2.ms_sweep = 0.0;
      o2.sweeps = st.iter;
    }
  }
  return PR_OK;
}

extern "C" {

pr_status pr_group_update(pr_group* q, pr_method method, double alpha, double tau, const pr_options* opts,
                          pr_stats* stats) {
  return pr_group_update_members(q, method, alpha, tau, opts, nullptr, 0, stats);
}

pr_status pr_group_update_members(pr_group* q, pr_method method, double alpha, double tau, const pr_options* opts,
                                  const int32_t* members, int32_t count, pr_stats* stats) {
  pr_status st = group_launch(q, method, alpha, tau, opts, members, count);
  if (st != PR_OK) return st;
  return group_complete(q, stats);
}

}  // extern "C"

// ------------------------------------------------------------------ unit sizes

extern "C" {

pr_status pr_group_get_tuning(const pr_group* q, pr_group_tuning* out) {
  if (!q || !out) return PR_EINVAL;
  out->quads_per_lane = GR_QPT[q->qi];
  out->steps_per_unit = GR_STEPS[q->qi];
  out->chunks_per_unit = GR_FU[q->fi];
  out->ms_update = q->tune_ms;
  out->candidates = q->tune_trials;
  return PR_OK;
}

pr_status pr_group_set_tuning(pr_group* q, const pr_group_tuning* in) {
  if (!q || !in || q->in_flight) return PR_EINVAL;
  int qi = -1, fi = -1;
  for (int i = 0; i < GR_NQ; i++)
    if (GR_QPT[i] == in->quads_per_lane && GR_STEPS[i] == in->steps_per_unit) qi = i;
  for (int i = 0; i < 3; i++)
    if (GR_FU[i] == in->chunks_per_unit) fi = i;
  if (qi < 0 || fi < 0) return PR_EINVAL;
  q->qi = qi;
  q->fi = fi;
  q->tune_ms = 0.f;
  q->tune_trials = 0;
  return PR_OK;
}

pr_status pr_group_autotune(pr_group* q, pr_method method, double alpha, double tau, int32_t reps,
                            pr_group_tuning* out) {
  if (!q || q->in_flight || reps < 0 || reps > 100) return PR_EINVAL;
  if (method != PR_STATIC && method != PR_NAIVE_DYNAMIC && method != PR_DF && method != PR_DFP) return PR_EINVAL;
  if (!(alpha >= 0.0 && alpha < 1.0) || !(tau >= 0.0)) return PR_EINVAL;
  if (reps == 0) reps = 1;
  const int G = q->G;
  if (method != PR_STATIC)
    for (int i = 0; i < G; i++)
      if (!q->graphs[i]->g.has_ranks) return PR_ENORANKS;
  // the ranks of every graph on entry, put back before every trial and at the end
  std::vector<int64_t> off(G + 1, 0);
  for (int i = 0; i < G; i++) off[i + 1] = off[i] + (q->graphs[i]->g.has_ranks ? q->graphs[i]->g.n : 0);
  double* saved = nullptr;
  if (off[G] > 0 && dev_malloc((void**)&saved, sizeof(double) * (size_t)off[G]) != cudaSuccess) {
    cudaGetLastError();
    return PR_ENOMEM;
  }
  auto copy_ranks = [&](bool back) -> cudaError_t {
    for (int i = 0; i < G; i++) {
      Graph* g = &q->graphs[i]->g;
      if (off[i + 1] == off[i]) continue;
      double* dst = back ? g->R : saved + off[i];
      const double* src = back ? saved + off[i] : g->R;
      cudaError_t e = cudaMemcpyAsync(dst, src, sizeof(double) * (size_t)g->n, cudaMemcpyDeviceToDevice, g->stream);
      if (e == cudaSuccess && back) e = launch_contrib_all(g->R, g->C[g->ccur], g->out.deg, g->tab_sc, g->n, g->stream);
      if (e == cudaSuccess) e = cudaStreamSynchronize(g->stream);
      if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
  };
  pr_status st = copy_ranks(false) == cudaSuccess ? PR_OK : PR_ECUDA;
  const int qi0 = q->qi, fi0 = q->fi;
  int bq = qi0, bf = fi0, trials = 0;
  float best = -1.f;
  std::vector<pr_stats> stats(G);
  for (int qi = 0; qi < GR_NQ && st == PR_OK; qi++)
    for (int fi = 0; fi < 3 && st == PR_OK; fi++) {
      q->qi = qi;
      q->fi = fi;
      double ms = 0.0;
      for (int r = 0; r < reps && st == PR_OK; r++) {
        if (copy_ranks(true) != cudaSuccess) {
          st = PR_ECUDA;
          break;
        }
        // timed on the CUDA-graph loop: the unit sizes are its (and the host
        // loop's); the one-kernel loop of small groups has fixed ones
        const pr_options graph_loop = {1e-6, 1e-6, 500, PR_OPT_DEVICE_LOOP};
        st = group_launch(q, method, alpha, tau, &graph_loop, nullptr, 0);
        if (st == PR_OK) st = group_complete(q, stats.data());
        ms += stats[0].ms_update;
      }
      if (st != PR_OK) break;
      trials++;
      if (best < 0.f || ms / reps < best) {
        best = (float)(ms / reps);
        bq = qi;
        bf = fi;
      }
    }
  if (st == PR_OK && copy_ranks(true) != cudaSuccess) st = PR_ECUDA;
  if (saved) cudaFree(saved);
  q->qi = st == PR_OK ? bq : qi0;
  q->fi = st == PR_OK ? bf : fi0;
  if (st != PR_OK) return st;
  q->tune_ms = best;
  q->tune_trials = trials;
  return out ? pr_group_get_tuning(q, out) : PR_OK;
}

}  // extern "C"
