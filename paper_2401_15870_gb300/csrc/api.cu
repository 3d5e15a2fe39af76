// api.cu -- the C ABI of include/dfpr.h and the method drivers.
//
// pr_update drives the iterations of Alg. 1 (and of the comparators) from the
// host: every iteration enqueues its kernels on the graph's stream and reads
// back the 100-byte control block, which holds the iteration's L-inf change.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>
#include <vector>
#include <nvtx3/nvToolsExt.h>
#include "dfpr.h"
#include "batch.cuh"
#include "frontier.cuh"
#include "graph.cuh"
#include "handle.cuh"
#include "prim.cuh"
#include "sweep.cuh"

using namespace dfpr;

// DF / DF-P direction choice: a frontier whose in-edges exceed this share of
// all edges is swept in pull form (every vertex, membership test); a pull
// frontier whose estimated size falls below this share of the vertices goes
// back to lists
constexpr double PULL_EDGE_FRACTION = 0.33;
constexpr double PUSH_VERTEX_FRACTION = 0.10;
// share of L2 given to the contributions gathered with an evict-last policy
constexpr double HOT_L2_FRACTION = 0.5;


#define TRY(x)                                          \
  do {                                                  \
    cudaError_t _e = (x);                               \
    if (_e != cudaSuccess) return (pr_status)cuda_fail(g, _e, #x); \
  } while (0)

#define RC(x)                       \
  do {                              \
    int _r = (x);                   \
    if (_r != OK) return (pr_status)_r; \
  } while (0)

// temporary device buffer of an export call, freed on every return path
template <typename T>
struct DevBuf {
  T* p = nullptr;
  cudaError_t alloc(int64_t count) { return dev_malloc((void**)&p, sizeof(T) * (size_t)(count > 0 ? count : 1)); }
  ~DevBuf() {
    if (p) cudaFree(p);
  }
};

static int bits_for(int32_t n) {
  int b = 1;
  while ((1ll << b) < (int64_t)n) b++;
  return b;
}

// ------------------------------------------------------------------ construction helpers

__global__ void k_edge_keys(const int32_t* __restrict__ src, const int32_t* __restrict__ dst, int64_t m, int32_t n,
                            int bits, uint64_t* __restrict__ keys) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m + n; i += (int64_t)gridDim.x * blockDim.x) {
    if (i < m) keys[i] = ((uint64_t)src[i] << bits) | (uint64_t)dst[i];
    else keys[i] = ((uint64_t)(i - m) << bits) | (uint64_t)(i - m);
  }
}

__global__ void k_csr_keys(const int64_t* __restrict__ off, const int32_t* __restrict__ col, int64_t m, int32_t n,
                           int bits, uint64_t* __restrict__ keys) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m + n; i += (int64_t)gridDim.x * blockDim.x) {
    if (i < m) {
      int32_t lo = 0, hi = n - 1;   // row u with off[u] <= i < off[u+1]
      while (lo < hi) {
        int32_t mid = (lo + hi + 1) >> 1;
        if (off[mid] <= i) lo = mid;
        else hi = mid - 1;
      }
      keys[i] = ((uint64_t)lo << bits) | (uint64_t)col[i];
    } else {
      keys[i] = ((uint64_t)(i - m) << bits) | (uint64_t)(i - m);
    }
  }
}

__global__ void k_validate_ids(const int32_t* __restrict__ a, int64_t m, int32_t n, unsigned long long* bad) {
  unsigned long long c = 0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x)
    c += (a[i] < 0 || a[i] >= n) ? 1 : 0;
  if (c) atomicAdd(bad, c);
}

// pr_get_rows: degree and row start of each requested vertex (caller's ids)
__global__ void k_row_meta(const int32_t* __restrict__ v, int64_t count, const int32_t* __restrict__ perm,
                           const int64_t* __restrict__ off, const int32_t* __restrict__ deg, int32_t* __restrict__ d_out,
                           int64_t* __restrict__ base_out) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < count; k += (int64_t)gridDim.x * blockDim.x) {
    int32_t r = perm[v[k]];
    d_out[k] = deg[r];
    base_out[k] = off[r];
  }
}

// pr_get_rows: one warp per requested row, neighbours mapped back to caller's ids
__global__ void k_row_copy_out(int64_t count, const int64_t* __restrict__ base, const int64_t* __restrict__ off,
                               const int32_t* __restrict__ col, const int32_t* __restrict__ iperm,
                               int32_t* __restrict__ adj) {
  int lane = threadIdx.x & 31;
  int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t k = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; k < count; k += nw) {
    int64_t d = off[k + 1] - off[k];
    for (int64_t x = lane; x < d; x += 32) adj[off[k] + x] = iperm[col[base[k] + x]];
  }
}

__global__ void k_check_ranks(const double* __restrict__ r, int32_t n, unsigned long long* bad, double* sum) {
  double s = 0.0;
  unsigned long long b = 0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    double x = r[i];
    if (!(x >= 0.0) || !isfinite(x)) b++;
    else s += x;
  }
  if (b) atomicAdd(bad, b);
  atomicAdd(sum, s);
}

__global__ void k_bits_to_bytes(const uint32_t* __restrict__ a, const uint32_t* __restrict__ b,
                                const int32_t* __restrict__ perm, int32_t n, uint8_t* __restrict__ out) {
  for (int64_t u = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; u < n; u += (int64_t)gridDim.x * blockDim.x) {
    int32_t v = perm[u];
    uint32_t w = a[v >> 5] | (b ? b[v >> 5] : 0u);
    out[u] = (w >> (v & 31)) & 1u;
  }
}

static pr_status alloc_state(pr_graph* h) {
  Graph* g = &h->g;
  int32_t n = g->n;
  int64_t words = cdiv(n, 32) + 1;
  TRY(dalloc(g, (void**)&g->R, sizeof(double) * n));
  for (int i = 0; i < 2; i++) {
    TRY(dalloc(g, (void**)&g->C[i], sizeof(long long) * (n + 1)));
    TRY(cudaMemsetAsync(g->C[i], 0, sizeof(long long) * (n + 1), g->stream));
    TRY(dalloc(g, (void**)&g->bits[i], sizeof(uint32_t) * words));
    TRY(dalloc(g, (void**)&g->wl[i], sizeof(int32_t) * n));
  }
  TRY(dalloc(g, (void**)&g->ever, sizeof(uint32_t) * words));
  TRY(dalloc(g, (void**)&g->aux, sizeof(uint32_t) * words));
  TRY(dalloc(g, (void**)&g->aux2, sizeof(uint32_t) * words));
  TRY(dalloc(g, (void**)&g->anyb, sizeof(uint32_t) * words));
  TRY(dalloc(g, (void**)&g->xl, sizeof(int32_t) * n));
  TRY(dalloc(g, (void**)&g->rnew, sizeof(double) * n));
  TRY(dalloc(g, (void**)&g->qs, sizeof(int64_t) * (n + 1)));
  TRY(dalloc(g, (void**)&g->xqs, sizeof(int64_t) * (n + 1)));
  TRY(dalloc(g, (void**)&g->gacc, sizeof(long long) * n));
  TRY(cudaMemsetAsync(g->gacc, 0, sizeof(long long) * n, g->stream));
  TRY(dalloc(g, (void**)&g->gcnt, sizeof(int32_t) * n));
  TRY(cudaMemsetAsync(g->gcnt, 0, sizeof(int32_t) * n, g->stream));
  TRY(dalloc(g, (void**)&g->gany, sizeof(int32_t) * n));
  TRY(cudaMemsetAsync(g->gany, 0, sizeof(int32_t) * n, g->stream));
  TRY(dalloc(g, (void**)&g->done, sizeof(int32_t) * (cdiv(n, 128) + 1)));
  TRY(cudaMemsetAsync(g->done, 0, sizeof(int32_t) * (cdiv(n, 128) + 1), g->stream));
  TRY(dalloc(g, (void**)&g->tab_sc, sizeof(double) * TAB));
  TRY(dalloc(g, (void**)&g->tab_ab, sizeof(double2) * TAB));
  TRY(dalloc(g, (void**)&g->ctl, sizeof(Ctl)));
  TRY(cudaMemsetAsync(g->ctl, 0, sizeof(Ctl), g->stream));
  TRY(cudaMallocHost((void**)&g->ctl_h, sizeof(Ctl)));
  TRY(dalloc(g, (void**)&h->lbits_tmp, sizeof(int32_t) * bits_to_list_tmp(n)));
  TRY(dalloc(g, (void**)&h->ls_tmp, sizeof(int64_t) * list_scan_tmp(n)));
  TRY(dalloc(g, (void**)&h->vec_tmp, sizeof(double) * (n > 4 ? n : 4)));
  TRY(launch_tables(g->tab_sc, g->tab_ab, 0.85, g->n, g->stream));
  g->tab_alpha = 0.85;
  for (int i = 0; i < 6; i++) TRY(cudaEventCreate(&h->ev[i]));
  return PR_OK;
}

// grow the tile tables to cover any list of the current graph
static pr_status ensure_tiles(pr_graph* h) {
  Graph* g = &h->g;
  int64_t need = cdiv(g->m / 4 + g->n + 1, SW_TILE_Q) + 2;
  if (need <= h->tiles_cap) return PR_OK;
  int64_t cap = need + need / 4 + 16;
  for (auto& p : g->allocs)
    if (p == g->tfirst || p == g->xtfirst) {
      cudaFree(p);
      p = nullptr;
    }
  TRY(dalloc(g, (void**)&g->tfirst, sizeof(int32_t) * cap));
  TRY(dalloc(g, (void**)&g->xtfirst, sizeof(int32_t) * cap));
  h->tiles_cap = cap;
  return PR_OK;
}

static pr_status finish_create(pr_graph* h, uint64_t* keys, int64_t nkeys, pr_graph** out) {
  Graph* g = &h->g;
  RC(build_graph_from_user_keys(g, keys, nkeys));
  pr_status st = alloc_state(h);
  if (st != PR_OK) return st;
  st = ensure_tiles(h);
  if (st != PR_OK) return st;
  TRY(cudaStreamSynchronize(g->stream));
  *out = h;
  return PR_OK;
}

static void destroy_handle(pr_graph* h) {
  if (!h) return;
  if (h->solo) pr_group_destroy(h->solo);
  Graph* g = &h->g;
  if (g->stream) cudaStreamSynchronize(g->stream);
  dfree_all(g);
  if (g->dmin) cudaFree(g->dmin);
  if (g->dplus) cudaFree(g->dplus);
  if (g->ctl_h) cudaFreeHost(g->ctl_h);
  if (g->small_h) cudaFreeHost(g->small_h);
  for (int i = 0; i < 6; i++)
    if (h->ev[i]) cudaEventDestroy(h->ev[i]);
  for (cudaEvent_t e : h->saux.ev)
    if (e) cudaEventDestroy(e);
  if (h->saux.stream) cudaStreamDestroy(h->saux.stream);
  delete h;
}

// a non-blocking stream at the highest priority, so that the epilogue blocks
// of one range are scheduled as soon as the gather of the next leaves room
cudaError_t dfpr::sweep_aux(pr_graph* h, const GatherCfg& c, const SweepAux** out) {
  *out = nullptr;
  if (c.parts <= 1) return cudaSuccess;
  SweepAux& a = h->saux;
  if (!a.stream) {
    int least = 0, greatest = 0;
    cudaError_t e = cudaDeviceGetStreamPriorityRange(&least, &greatest);
    if (e == cudaSuccess) e = cudaStreamCreateWithPriority(&a.stream, cudaStreamNonBlocking, greatest);
    for (int i = 0; e == cudaSuccess && i < 9; i++) e = cudaEventCreateWithFlags(&a.ev[i], cudaEventDisableTiming);
    if (e != cudaSuccess) return e;
  }
  *out = &a;
  return cudaSuccess;
}

// ------------------------------------------------------------------ drivers

static pr_status read_ctl(Graph* g) {
  TRY(cudaMemcpyAsync(g->ctl_h, g->ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, g->stream));
  TRY(cudaStreamSynchronize(g->stream));
  if (g->ctl_h->status) return (pr_status)set_error(g, ECUDA_, "device reported an inconsistent tile table");
  return PR_OK;
}

static double ctl_dR(const Ctl* c) {
  double d;
  unsigned long long b = c->dR_last;
  memcpy(&d, &b, sizeof(d));
  return d;
}

// vertices whose contributions fit in a share of L2 (the most-gathered ones)
static int32_t hot_vertices(Graph* g) {
  int l2 = 0;
  if (cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, g->dev) != cudaSuccess || l2 <= 0) l2 = 64 << 20;
  int64_t hot = (int64_t)(HOT_L2_FRACTION * (double)l2) / (int64_t)sizeof(long long);
  return (int32_t)(hot < g->n ? hot : g->n);
}

SweepParams dfpr::base_params(Graph* g, double alpha, double tau_f, double tau_p) {
  SweepParams p;
  memset(&p, 0, sizeof(p));
  p.n = g->n;
  p.ioff = g->in.off;
  p.ideg = g->in.deg;
  p.icol = g->in.col;
  p.odeg = g->out.deg;
  p.R = g->R;
  p.rnew = g->rnew;
  p.tab_sc = g->tab_sc;
  p.tab_ab = g->tab_ab;
  p.alpha = alpha;
  p.C0 = (1.0 - alpha) / (double)g->n;
  p.tau_f = tau_f;
  p.tau_p = tau_p;
  p.gacc = g->gacc;
  p.gcnt = g->gcnt;
  p.ctl = g->ctl;
  p.hot = hot_vertices(g);
  return p;
}

static ExpandParams expand_params(Graph* g, const int32_t* list, const int32_t* count, uint32_t* bits, uint32_t* ever,
                                  int32_t* wl, int32_t* cnt) {
  ExpandParams e;
  memset(&e, 0, sizeof(e));
  e.n = g->n;
  e.ooff = g->out.off;
  e.ocol = g->out.col;
  e.list = list;
  e.count = count;
  e.qs = g->xqs;
  e.tfirst = g->xtfirst;
  e.ntiles_dev = &g->ctl->xntiles;
  e.bits = bits;
  e.ever = ever;
  e.wl = wl;
  e.cnt = cnt;
  e.id_bits = g->id_bits;
  return e;
}

// expand the listed vertices' out-rows (expander tables)
static pr_status run_expand(pr_graph* h, const int32_t* list, const int32_t* count, uint32_t* bits, uint32_t* ever,
                            int32_t* wl, int32_t* cnt, const uint32_t* ins_src_bits) {
  Graph* g = &h->g;
  TRY(launch_list_scan(list, count, g->out.deg, g->n, g->xqs, g->xtfirst, &g->ctl->xqtot, &g->ctl->xntiles, h->ls_tmp,
                       g->stream));
  ExpandParams e = expand_params(g, list, count, bits, ever, wl, cnt);
  e.ins_src_bits = ins_src_bits;
  e.dplus = g->dplus;
  e.n_dplus = g->n_dplus;
  TRY(launch_expand(e, g->stream));
  return PR_OK;
}

// DF / DF-P initial marking (Alg. 1) into bits[0] / wl[0] / ever
static pr_status initial_marking(pr_graph* h) {
  Graph* g = &h->g;
  cudaStream_t s = g->stream;
  int64_t words = cdiv(g->n, 32) + 1;
  for (uint32_t* b : {g->bits[0], g->bits[1], g->ever, g->aux, g->aux2})
    TRY(cudaMemsetAsync(b, 0, sizeof(uint32_t) * words, s));
  TRY(cudaMemsetAsync(g->ctl, 0, sizeof(Ctl), s));
  // sources of the effective change, each once
  TRY(launch_mark_sources(g->dmin, g->n_dmin, g->dplus, g->n_dplus, g->id_bits, g->aux, g->xl, &g->ctl->nexp, s));
  // G_t.out(u) for every source u ...
  pr_status st = run_expand(h, g->xl, &g->ctl->nexp, g->bits[0], nullptr, g->wl[0], &g->ctl->count[0], nullptr);
  if (st != PR_OK) return st;
  // ... and the targets of deleted edges, which complete G_{t-1}.out(u)
  TRY(launch_mark_targets(g->dmin, g->n_dmin, g->id_bits, g->bits[0], nullptr, g->wl[0], &g->ctl->count[0], s));
  TRY(cudaMemsetAsync(&g->ctl->nexp, 0, sizeof(int32_t), s));
  return PR_OK;
}

// Dynamic Traversal affected set: reach(G_t) in aux, reach(G_{t-1}) in aux2;
// the union as an ascending list in wl[0] / count[0]
static pr_status dt_affected(pr_graph* h) {
  Graph* g = &h->g;
  cudaStream_t s = g->stream;
  int64_t words = cdiv(g->n, 32) + 1;
  for (uint32_t* b : {g->aux, g->aux2, g->bits[1]}) TRY(cudaMemsetAsync(b, 0, sizeof(uint32_t) * words, s));
  TRY(launch_source_bits(g->dplus, g->n_dplus, g->id_bits, g->bits[1], s));
  for (int which = 0; which < 2; which++) {
    uint32_t* vis = which == 0 ? g->aux : g->aux2;
    TRY(cudaMemsetAsync(g->ctl, 0, sizeof(Ctl), s));
    TRY(launch_mark_sources(g->dmin, g->n_dmin, g->dplus, g->n_dplus, g->id_bits, vis, g->wl[0], &g->ctl->count[0], s));
    int c = 0;
    for (;;) {
      pr_status st = run_expand(h, g->wl[c], &g->ctl->count[c], vis, nullptr, g->wl[1 - c], &g->ctl->count[1 - c],
                                which == 1 ? g->bits[1] : nullptr);
      if (st != PR_OK) return st;
      if (which == 1)
        TRY(launch_follow_edges(g->dmin, g->n_dmin, g->id_bits, vis, g->wl[1 - c], &g->ctl->count[1 - c], s));
      TRY(cudaMemsetAsync(&g->ctl->count[c], 0, sizeof(int32_t), s));
      c ^= 1;
      st = read_ctl(g);
      if (st != PR_OK) return st;
      if (g->ctl_h->count[c] == 0) break;
    }
  }
  TRY(cudaMemsetAsync(g->ctl, 0, sizeof(Ctl), s));
  TRY(launch_bits_to_list(g->aux, g->aux2, g->n, g->wl[0], &g->ctl->count[0], h->lbits_tmp, s));
  return PR_OK;
}

// one sweep launch, bracketed by events when timing is on (the host reads the
// control block right after, so the pair is read back at once)
struct SweepTimer {
  pr_graph* h;
  bool on;
  double ms = 0.0;
  int32_t launches = 0;
  int last_mode = 0;
  long long edges0 = 0, verts0 = 0;   // the control block's totals at the previous record
  // asynchronous order: every-vertex sweeps over ASYNC_RANGES vertex ranges in
  // order (bounds: equal shares of the in-edges), the contributions updated in
  // place after each range
  bool async = false;
  int32_t bounds[ASYNC_RANGES + 1] = {};
  cudaError_t launch(int mode, const SweepParams& p, cudaStream_t s) {
    last_mode = mode;
    if (on) cudaEventRecord(h->ev[4], s);
    cudaError_t e;
    if (mode == SWEEP_FULL || mode == SWEEP_PULL_DF || mode == SWEEP_PULL_DFP) {
      Graph* g = &h->g;
      SweepParams q = p;
      q.ntiles_host = g->in.cap >> 2;
      GatherCfg cfg = h->gcfg;
      const SweepAux* aux = nullptr;
      if (async) {
        cfg.fused = 0;
        cfg.parts = ASYNC_RANGES;
        e = cudaSuccess;
      } else {
        e = sweep_aux(h, cfg, &aux);
      }
      if (e == cudaSuccess)
        e = launch_full_sweep(mode, q, cfg, g->rowbits, g->rowbase, g->anyb, g->done, aux, s, async,
                              async ? bounds : nullptr);
    } else {
      e = launch_sweep(mode, p, s);
    }
    if (on) cudaEventRecord(h->ev[5], s);
    launches++;
    return e;
  }
  // after read_ctl: the sweep's time and, from the control block's running
  // totals, the edges and vertices it processed, as one trace record
  void collect() {
    if (!on) return;
    float t = 0.f;
    if (cudaEventElapsedTime(&t, h->ev[4], h->ev[5]) == cudaSuccess) ms += t;
    const Ctl* c = h->g.ctl_h;
    pr_sweep_record r;
    r.iteration = (int32_t)h->sweep_log.size();
    r.form = last_mode == SWEEP_FULL || last_mode == SWEEP_PULL_DF || last_mode == SWEEP_PULL_DFP
                 ? PR_SWEEP_EVERY_VERTEX : PR_SWEEP_LIST;
    r.ms = t;
    r.edges = c->edges - edges0;
    r.vertices = c->verts - verts0;
    edges0 = c->edges;
    verts0 = c->verts;
    h->sweep_log.push_back(r);
  }
};

pr_status dfpr::run_update(pr_graph* h, int method, double alpha, double tau, double tau_f, double tau_p,
                           int32_t max_iter, int32_t flags, pr_stats* out) {
  SweepTimer timer{h, (flags & PR_OPT_TIME_SWEEPS) != 0};
  const bool async = (flags & PR_OPT_ASYNC) != 0;
  timer.async = async;
  if (async) flags |= PR_OPT_FORCE_PULL;
  h->sweep_log.clear();
  Graph* g = &h->g;
  cudaStream_t s = g->stream;
  int32_t n = g->n;
  TRY(cudaEventRecord(h->ev[2], s));
  if (g->tab_alpha != alpha) {
    TRY(launch_tables(g->tab_sc, g->tab_ab, alpha, n, s));
    g->tab_alpha = alpha;
  }
  // the ranges of the asynchronous order from this graph's in-degrees (the
  // rank-export buffer is free during an update and far larger than needed)
  if (async) TRY(async_range_bounds(g->in.deg, n, ASYNC_RANGES, (int64_t*)h->vec_tmp, timer.bounds, s));
  SweepParams p = base_params(g, alpha, tau_f, tau_p);
  p.metric = (flags & PR_OPT_MEASURE_ABSOLUTE) ? METRIC_ABSOLUTE
             : (flags & PR_OPT_MEASURE_CONTRIB) ? METRIC_CONTRIB
                                                : METRIC_RELATIVE;
  int64_t ever = 0;
  int32_t iters = 0;
  double dR = 0.0;
  bool conv = false;
  if (method == PR_STATIC || method == PR_NAIVE_DYNAMIC) {
    TRY(cudaMemsetAsync(g->ctl, 0, sizeof(Ctl), s));
    if (method == PR_STATIC) TRY(launch_init_uniform(g->R, g->C[g->ccur], g->out.deg, g->tab_sc, n, s));
    p.tfirst = g->full_tfirst;
    p.ntiles_host = g->full_ntiles;
    for (int32_t it = 0; it < max_iter; it++) {
      p.Ccur = g->C[g->ccur];
      p.Cnext = g->C[async ? g->ccur : 1 - g->ccur];   // one vector, updated in place, when asynchronous
      TRY(timer.launch(SWEEP_FULL, p, s));
      TRY(launch_control(g->ctl, 0, s));
      if (!async) g->ccur ^= 1;
      pr_status st = read_ctl(g);
      if (st != PR_OK) return st;
      timer.collect();
      iters = it + 1;
      dR = ctl_dR(g->ctl_h);
      if (dR <= tau) {
        conv = true;
        break;
      }
    }
    ever = iters > 0 ? n : 0;
  } else if (method == PR_DYNAMIC_TRAVERSAL) {
    pr_status st = dt_affected(h);
    if (st != PR_OK) return st;
    TRY(launch_list_scan(g->wl[0], &g->ctl->count[0], g->in.deg, n, g->qs, g->tfirst, &g->ctl->qtot, &g->ctl->ntiles,
                         h->ls_tmp, s));
    st = read_ctl(g);
    if (st != PR_OK) return st;
    const int64_t n_aff = g->ctl_h->count[0];
    const bool pull = (flags & PR_OPT_FORCE_PULL) ||
                      (!(flags & PR_OPT_FORCE_PUSH) && (double)(4 * g->ctl_h->qtot) > PULL_EDGE_FRACTION * (double)g->m);
    if (pull) {
      // the affected set holds most in-edges: sweep every row and update the
      // members of A = aux | aux2 only.  This is the pull form of DF with no
      // expansion (tau_f = +inf): the frontier stays A, every member is
      // recomputed with Eq. 1 from the same sums as the list sweep, the other
      // rows keep their ranks and contributions
      const int64_t words = cdiv(n, 32) + 1;
      const size_t wbytes = sizeof(uint32_t) * (size_t)words;
      uint32_t* xb[2] = {g->aux, g->aux2};
      TRY(launch_bits_or(g->aux, g->aux2, g->bits[0], words, s));
      for (uint32_t* b : {g->bits[1], g->aux, g->aux2, g->ever}) TRY(cudaMemsetAsync(b, 0, wbytes, s));
      p.tau_f = HUGE_VAL;
      p.tau_p = HUGE_VAL;
      int cur = 0;
      for (int32_t it = 0; it < max_iter; it++) {
        p.list = nullptr;
        p.tfirst = g->full_tfirst;
        p.ntiles_host = g->full_ntiles;
        p.Ccur = g->C[g->ccur];
        p.Cnext = g->C[1 - g->ccur];
        p.S_cur = g->bits[cur];
        p.X_cur = xb[cur];
        p.S_next = g->bits[1 - cur];
        p.X_next = xb[1 - cur];
        p.gany = g->gany;
        p.ever = g->ever;
        p.cnt_next = &g->ctl->count[1 - cur];
        p.cnt_x = &g->ctl->nexp;
        TRY(timer.launch(SWEEP_PULL_DF, p, s));
        TRY(launch_control(g->ctl, 1, s));
        g->ccur ^= 1;
        cur ^= 1;
        st = read_ctl(g);
        if (st != PR_OK) return st;
        timer.collect();
        iters = it + 1;
        dR = ctl_dR(g->ctl_h);
        if (dR <= tau) {
          conv = true;
          break;
        }
      }
      ever = iters > 0 ? n_aff : 0;
    } else {
      p.list = g->wl[0];
      p.count = &g->ctl->count[0];
      p.qs = g->qs;
      p.tfirst = g->tfirst;
      p.ntiles_dev = &g->ctl->ntiles;
      p.Ccur = g->C[g->ccur];
      for (int32_t it = 0; it < max_iter; it++) {
        TRY(timer.launch(SWEEP_LIST, p, s));
        TRY(launch_commit(g->wl[0], &g->ctl->count[0], g->rnew, g->R, g->C[g->ccur], g->out.deg, g->tab_sc, nullptr, n,
                          s));
        TRY(launch_control(g->ctl, 0, s));
        st = read_ctl(g);
        if (st != PR_OK) return st;
        timer.collect();
        iters = it + 1;
        dR = ctl_dR(g->ctl_h);
        if (dR <= tau) {
          conv = true;
          break;
        }
      }
      if (max_iter == 0) {
        st = read_ctl(g);
        if (st != PR_OK) return st;
      }
      ever = iters > 0 ? g->ctl_h->count[0] : 0;
    }
  } else {
    pr_status st = initial_marking(h);
    if (st != PR_OK) return st;
    const bool prune = method == PR_DFP;
    const int push_mode = prune ? SWEEP_DFP : SWEEP_DF;
    const int pull_mode = prune ? SWEEP_PULL_DFP : SWEEP_PULL_DF;
    uint32_t* xb[2] = {g->aux, g->aux2};
    const size_t wbytes = sizeof(uint32_t) * (size_t)(cdiv(n, 32) + 1);
    const double dbar = (double)g->m / (double)n;
    int cur = 0;
    bool pull = false;
    // quad prefix of F_0: its edge volume picks push or pull for the first sweep
    TRY(launch_list_scan(g->wl[0], &g->ctl->count[0], g->in.deg, n, g->qs, g->tfirst, &g->ctl->qtot,
                         &g->ctl->ntiles, h->ls_tmp, s));
    st = read_ctl(g);
    if (st != PR_OK) return st;
    for (int32_t it = 0; it < max_iter; it++) {
      const bool want_pull = (flags & PR_OPT_FORCE_PULL) ||
                             (!(flags & PR_OPT_FORCE_PUSH) && (double)(4 * g->ctl_h->qtot) > PULL_EDGE_FRACTION * (double)g->m);
      if (!pull && want_pull) {
        // large frontier: sweep every vertex and test membership (F_i = S u out(X),
        // S = bits[cur] holds F_i, X empty)
        pull = true;
        TRY(cudaMemsetAsync(xb[cur], 0, wbytes, s));
      }
      if (pull) {
        // the pull epilogue writes every word of S_next and X_next
        p.list = nullptr;
        p.tfirst = g->full_tfirst;
        p.ntiles_host = g->full_ntiles;
        // with the gather and the epilogue in separate launches over one
        // range, the epilogue updates the contributions in place (the gather
        // that reads them has finished); otherwise into the other buffer.
        // Asynchronous order: in place after every range, on purpose
        const bool inplace = async || (!h->gcfg.fused && h->gcfg.parts == 1);
        p.Ccur = g->C[g->ccur];
        p.Cnext = g->C[inplace ? g->ccur : 1 - g->ccur];
        p.S_cur = g->bits[cur];
        p.X_cur = xb[cur];
        p.S_next = g->bits[1 - cur];
        p.X_next = xb[1 - cur];
        p.gany = g->gany;
        p.ever = g->ever;
        p.cnt_next = &g->ctl->count[1 - cur];
        p.cnt_x = &g->ctl->nexp;
        TRY(timer.launch(pull_mode, p, s));
        TRY(launch_control(g->ctl, 1, s));
        if (!inplace) g->ccur ^= 1;
        cur ^= 1;
        st = read_ctl(g);
        if (st != PR_OK) return st;
        timer.collect();
        iters = it + 1;
        dR = ctl_dR(g->ctl_h);
        if (dR <= tau) {
          conv = true;
          break;
        }
        double est = (double)g->ctl_h->count[cur] + dbar * (double)g->ctl_h->nexp_last;
        if (!(flags & PR_OPT_FORCE_PULL) && est < PUSH_VERTEX_FRACTION * (double)n) {
          // the frontier shrank: materialise F_{i+1} = S u out(X) as a list
          pull = false;
          TRY(launch_bits_to_list(g->bits[cur], nullptr, n, g->wl[cur], &g->ctl->count[cur], h->lbits_tmp, s));
          TRY(launch_bits_to_list(xb[cur], nullptr, n, g->xl, &g->ctl->nexp, h->lbits_tmp, s));
          st = run_expand(h, g->xl, &g->ctl->nexp, g->bits[cur], nullptr, g->wl[cur], &g->ctl->count[cur], nullptr);
          if (st != PR_OK) return st;
          TRY(cudaMemsetAsync(&g->ctl->nexp, 0, sizeof(int32_t), s));
          TRY(cudaMemsetAsync(g->bits[1 - cur], 0, wbytes, s));
          TRY(launch_list_scan(g->wl[cur], &g->ctl->count[cur], g->in.deg, n, g->qs, g->tfirst, &g->ctl->qtot,
                               &g->ctl->ntiles, h->ls_tmp, s));
          st = read_ctl(g);
          if (st != PR_OK) return st;
        }
        continue;
      }
      p.list = g->wl[cur];
      p.count = &g->ctl->count[cur];
      p.qs = g->qs;
      p.tfirst = g->tfirst;
      p.ntiles_dev = &g->ctl->ntiles;
      p.Ccur = g->C[g->ccur];
      p.bits_next = g->bits[1 - cur];
      p.ever = g->ever;
      p.wl_next = g->wl[1 - cur];
      p.cnt_next = &g->ctl->count[1 - cur];
      p.xl = g->xl;
      p.cnt_x = &g->ctl->nexp;
      TRY(timer.launch(push_mode, p, s));
      st = run_expand(h, g->xl, &g->ctl->nexp, g->bits[1 - cur], nullptr, g->wl[1 - cur], &g->ctl->count[1 - cur],
                      nullptr);
      if (st != PR_OK) return st;
      TRY(launch_commit(g->wl[cur], &g->ctl->count[cur], g->rnew, g->R, g->C[g->ccur], g->out.deg, g->tab_sc,
                        g->bits[cur], n, s));
      TRY(launch_control(g->ctl, 1, s));
      cur ^= 1;
      TRY(launch_list_scan(g->wl[cur], &g->ctl->count[cur], g->in.deg, n, g->qs, g->tfirst, &g->ctl->qtot,
                           &g->ctl->ntiles, h->ls_tmp, s));
      st = read_ctl(g);
      if (st != PR_OK) return st;
      timer.collect();
      iters = it + 1;
      dR = ctl_dR(g->ctl_h);
      if (dR <= tau) {
        conv = true;
        break;
      }
    }
    long long* cnt = (long long*)h->vec_tmp;
    TRY(launch_popcount(g->ever, cdiv(n, 32), cnt, s));
    long long ev = 0;
    TRY(cudaMemcpyAsync(&ev, cnt, sizeof(ev), cudaMemcpyDeviceToHost, s));
    TRY(cudaStreamSynchronize(s));
    ever = ev;
    if (max_iter == 0) {
      st = read_ctl(g);
      if (st != PR_OK) return st;
    }
  }
  TRY(cudaEventRecord(h->ev[3], s));
  TRY(cudaEventSynchronize(h->ev[3]));
  float ms = 0.f;
  TRY(cudaEventElapsedTime(&ms, h->ev[2], h->ev[3]));
  g->has_ranks = true;
  if (out) {
    out->iterations = iters;
    out->converged = conv ? 1 : 0;
    out->delta_R = iters ? dR : 0.0;
    out->vertices_ever_affected = ever;
    out->edges_processed = g->ctl_h->edges;
    out->vertices_processed = g->ctl_h->verts;
    out->eff_deletions = g->n_dmin;
    out->eff_insertions = g->n_dplus;
    out->ms_apply = h->ms_apply;
    out->ms_update = ms;
    out->ms_sweep = timer.ms;
    out->sweeps = timer.launches;
    out->reserved = 0;
  }
  return PR_OK;
}

// ------------------------------------------------------------------ C ABI

extern "C" {

static pr_status create_from_keys_host_edges(int32_t n, int64_t m, const int32_t* src, const int32_t* dst,
                                             bool dev_ptrs, int32_t flags, void* stream, pr_graph** out) {
  pr_graph* h = new (std::nothrow) pr_graph();
  if (!h) return PR_ENOMEM;
  Graph* g = &h->g;
  g->n = n;
  g->id_bits = bits_for(n);
  g->stream = (cudaStream_t)stream;
  g->relabel = (flags & 1) == 0;
  cudaGetDevice(&g->dev);
  uint64_t* keys = nullptr;
  int32_t *ds = nullptr, *dd = nullptr;
  pr_status st = PR_OK;
  do {
    cudaError_t e = dev_malloc(&keys, sizeof(uint64_t) * (size_t)(m + n));
    if (e != cudaSuccess) { st = (pr_status)cuda_fail(g, e, "cudaMalloc(keys)"); break; }
    const int32_t *s_dev = src, *d_dev = dst;
    if (!dev_ptrs && m > 0) {
      if ((e = dev_malloc(&ds, sizeof(int32_t) * m)) != cudaSuccess ||
          (e = dev_malloc(&dd, sizeof(int32_t) * m)) != cudaSuccess ||
          (e = cudaMemcpyAsync(ds, src, sizeof(int32_t) * m, cudaMemcpyHostToDevice, g->stream)) != cudaSuccess ||
          (e = cudaMemcpyAsync(dd, dst, sizeof(int32_t) * m, cudaMemcpyHostToDevice, g->stream)) != cudaSuccess) {
        st = (pr_status)cuda_fail(g, e, "copy edge list");
        break;
      }
      s_dev = ds;
      d_dev = dd;
    }
    if (dev_ptrs && m > 0) {
      unsigned long long* bad;
      if ((e = dev_malloc(&bad, sizeof(*bad))) != cudaSuccess) { st = (pr_status)cuda_fail(g, e, "cudaMalloc"); break; }
      cudaMemsetAsync(bad, 0, sizeof(*bad), g->stream);
      note_launch(); k_validate_ids<<<grid_for(m, 256), 256, 0, g->stream>>>(src, m, n, bad);
      note_launch(); k_validate_ids<<<grid_for(m, 256), 256, 0, g->stream>>>(dst, m, n, bad);
      unsigned long long hb = 0;
      cudaMemcpyAsync(&hb, bad, sizeof(hb), cudaMemcpyDeviceToHost, g->stream);
      e = cudaStreamSynchronize(g->stream);
      cudaFree(bad);
      if (e != cudaSuccess) { st = (pr_status)cuda_fail(g, e, "validate"); break; }
      if (hb) { st = PR_ERANGE; break; }
    }
    note_launch(); k_edge_keys<<<grid_for(m + n, 256), 256, 0, g->stream>>>(s_dev, d_dev, m, n, g->id_bits, keys);
    if ((e = cudaGetLastError()) != cudaSuccess) { st = (pr_status)cuda_fail(g, e, "k_edge_keys"); break; }
    if (ds) { cudaStreamSynchronize(g->stream); cudaFree(ds); ds = nullptr; }
    if (dd) { cudaFree(dd); dd = nullptr; }
    st = finish_create(h, keys, m + n, out);
  } while (0);
  if (ds) cudaFree(ds);
  if (dd) cudaFree(dd);
  if (keys) cudaFree(keys);
  if (st != PR_OK) destroy_handle(h);
  return st;
}

pr_status pr_graph_create_edges(int32_t n, int64_t m, const int32_t* src, const int32_t* dst, int32_t device_ptrs,
                                int32_t flags, void* stream, pr_graph** out) {
  if (!out) return PR_EINVAL;
  *out = nullptr;
  if (n < 1 || m < 0 || (m > 0 && (!src || !dst)) || (flags & ~1)) return PR_EINVAL;
  if ((int64_t)n + m >= (int64_t(1) << 31)) return PR_EINVAL;
  if (!device_ptrs)
    for (int64_t i = 0; i < m; i++)
      if (src[i] < 0 || src[i] >= n || dst[i] < 0 || dst[i] >= n) return PR_ERANGE;
  return create_from_keys_host_edges(n, m, src, dst, device_ptrs != 0, flags, stream, out);
}

pr_status pr_graph_create(int32_t n, int64_t m, const int64_t* row_off, const int32_t* col, void* stream,
                          pr_graph** out) {
  if (!out) return PR_EINVAL;
  *out = nullptr;
  if (n < 1 || m < 0 || !row_off || (m > 0 && !col)) return PR_EINVAL;
  if ((int64_t)n + m >= (int64_t(1) << 31)) return PR_EINVAL;
  if (row_off[0] != 0 || row_off[n] != m) return PR_EINVAL;
  for (int32_t u = 0; u < n; u++)
    if (row_off[u + 1] < row_off[u]) return PR_EINVAL;
  for (int64_t i = 0; i < m; i++)
    if (col[i] < 0 || col[i] >= n) return PR_ERANGE;
  pr_graph* h = new (std::nothrow) pr_graph();
  if (!h) return PR_ENOMEM;
  Graph* g = &h->g;
  g->n = n;
  g->id_bits = bits_for(n);
  g->stream = (cudaStream_t)stream;
  cudaGetDevice(&g->dev);
  uint64_t* keys = nullptr;
  int64_t* doff = nullptr;
  int32_t* dcol = nullptr;
  pr_status st = PR_OK;
  cudaError_t e;
  if ((e = dev_malloc(&keys, sizeof(uint64_t) * (size_t)(m + n))) != cudaSuccess ||
      (e = dev_malloc(&doff, sizeof(int64_t) * (size_t)(n + 1))) != cudaSuccess ||
      (e = dev_malloc(&dcol, sizeof(int32_t) * (size_t)(m > 0 ? m : 1))) != cudaSuccess ||
      (e = cudaMemcpyAsync(doff, row_off, sizeof(int64_t) * (n + 1), cudaMemcpyHostToDevice, g->stream)) != cudaSuccess ||
      (m > 0 && (e = cudaMemcpyAsync(dcol, col, sizeof(int32_t) * m, cudaMemcpyHostToDevice, g->stream)) != cudaSuccess)) {
    st = (pr_status)cuda_fail(g, e, "pr_graph_create copy");
  } else {
    note_launch(); k_csr_keys<<<grid_for(m + n, 256), 256, 0, g->stream>>>(doff, dcol, m, n, g->id_bits, keys);
    e = cudaStreamSynchronize(g->stream);
    cudaFree(doff);
    cudaFree(dcol);
    doff = nullptr;
    dcol = nullptr;
    if (e != cudaSuccess) st = (pr_status)cuda_fail(g, e, "k_csr_keys");
    else st = finish_create(h, keys, m + n, out);
  }
  if (doff) cudaFree(doff);
  if (dcol) cudaFree(dcol);
  if (keys) cudaFree(keys);
  if (st != PR_OK) destroy_handle(h);
  return st;
}

void pr_graph_destroy(pr_graph* g) { destroy_handle(g); }

pr_status pr_set_stream(pr_graph* h, void* stream) {
  if (!h) return PR_EINVAL;
  Graph* g = &h->g;
  TRY(cudaStreamSynchronize(g->stream));
  g->stream = (cudaStream_t)stream;
  if (h->solo) {   // rebuilt on the new stream when next used
    pr_group_destroy(h->solo);
    h->solo = nullptr;
  }
  return PR_OK;
}

static pr_status apply_finish(pr_graph* h, bool wait);

static pr_status apply_common(pr_graph* h, const int32_t* ds, const int32_t* dd, int64_t nd, const int32_t* is,
                              const int32_t* id, int64_t ni, bool device) {
  if (!h || nd < 0 || ni < 0 || (nd > 0 && (!ds || !dd)) || (ni > 0 && (!is || !id))) return PR_EINVAL;
  Graph* g = &h->g;
  g->err.clear();
  cudaStream_t s = g->stream;
  int32_t n = g->n;
  TRY(cudaEventRecord(h->ev[0], s));
  int rc;
  if (device) {
    rc = apply_batch_device(g, ds, dd, nd, is, id, ni, false);
  } else {
    for (int64_t i = 0; i < nd; i++)
      if (ds[i] < 0 || ds[i] >= n || dd[i] < 0 || dd[i] >= n)
        return (pr_status)set_error(g, ERANGE_, "pr_apply_batch: vertex id out of range");
    for (int64_t i = 0; i < ni; i++)
      if (is[i] < 0 || is[i] >= n || id[i] < 0 || id[i] >= n)
        return (pr_status)set_error(g, ERANGE_, "pr_apply_batch: vertex id out of range");
    int64_t nk = nd + ni;
    void* stage;
    TRY(scratch_get(g, 0, sizeof(int32_t) * (size_t)(2 * nk + 4) + 1024, &stage));
    int32_t* b = (int32_t*)stage;
    if (nd) {
      TRY(cudaMemcpyAsync(b, ds, sizeof(int32_t) * nd, cudaMemcpyHostToDevice, s));
      TRY(cudaMemcpyAsync(b + nd, dd, sizeof(int32_t) * nd, cudaMemcpyHostToDevice, s));
    }
    if (ni) {
      TRY(cudaMemcpyAsync(b + 2 * nd, is, sizeof(int32_t) * ni, cudaMemcpyHostToDevice, s));
      TRY(cudaMemcpyAsync(b + 2 * nd + ni, id, sizeof(int32_t) * ni, cudaMemcpyHostToDevice, s));
    }
    rc = apply_batch_device(g, b, b + nd, nd, b + 2 * nd, b + 2 * nd + ni, ni, true);
  }
  if (rc != OK) return (pr_status)rc;
  return apply_finish(h, true);
}

// after a batch: the edge count, the tile tables, the end event and (when
// `wait`) the apply time
static pr_status apply_finish(pr_graph* h, bool wait) {
  Graph* g = &h->g;
  g->m += g->n_dplus - g->n_dmin;
  pr_status st = ensure_tiles(h);
  if (st != PR_OK) return st;
  TRY(cudaEventRecord(h->ev[1], g->stream));
  if (!wait) return PR_OK;
  TRY(cudaEventSynchronize(h->ev[1]));
  float ms = 0.f;
  TRY(cudaEventElapsedTime(&ms, h->ev[0], h->ev[1]));
  h->ms_apply = ms;
  return PR_OK;
}

// NVTX ranges name the library's phases for profilers (no cost without one)
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
};

pr_status pr_apply_batch(pr_graph* h, const int32_t* del_src, const int32_t* del_dst, int64_t n_del,
                         const int32_t* ins_src, const int32_t* ins_dst, int64_t n_ins) {
  NvtxRange r("pr_apply_batch");
  return apply_common(h, del_src, del_dst, n_del, ins_src, ins_dst, n_ins, false);
}

pr_status pr_apply_batch_device(pr_graph* h, const int32_t* del_src, const int32_t* del_dst, int64_t n_del,
                                const int32_t* ins_src, const int32_t* ins_dst, int64_t n_ins) {
  NvtxRange r("pr_apply_batch_device");
  return apply_common(h, del_src, del_dst, n_del, ins_src, ins_dst, n_ins, true);
}

// streams on which pr_apply_batches_device runs the graphs' batches side by
// side: a small batch is a chain of short kernels, one of them a single block,
// so one graph's chain leaves the GPU nearly idle (made on first use, one set
// per device, kept for the life of the process)
constexpr int APPLY_STREAMS = 16;

static cudaError_t apply_streams(int dev, cudaStream_t** out) {
  static std::mutex mu;
  static cudaStream_t pool[64][APPLY_STREAMS];
  static bool made[64] = {false};
  *out = nullptr;
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(mu);
  if (!made[dev]) {
    for (int i = 0; i < APPLY_STREAMS; i++) {
      cudaError_t e = cudaStreamCreateWithFlags(&pool[dev][i], cudaStreamNonBlocking);
      if (e != cudaSuccess) {
        for (int j = 0; j < i; j++) cudaStreamDestroy(pool[dev][j]);
        return e;
      }
    }
    made[dev] = true;
  }
  *out = pool[dev];
  return cudaSuccess;
}

// the batches of many graphs (host or device endpoint arrays), side by side on
// the pool's streams
static pr_status apply_many(int32_t count, pr_graph* const* graphs, const int32_t* const* del_src,
                            const int32_t* const* del_dst, const int64_t* n_del, const int32_t* const* ins_src,
                            const int32_t* const* ins_dst, const int64_t* n_ins, bool device) {
  if (count < 0 || (count > 0 && (!graphs || !n_del || !n_ins || !del_src || !del_dst || !ins_src || !ins_dst)))
    return PR_EINVAL;
  for (int32_t i = 0; i < count; i++) {
    if (!graphs[i] || n_del[i] < 0 || n_ins[i] < 0 || (n_del[i] > 0 && (!del_src[i] || !del_dst[i])) ||
        (n_ins[i] > 0 && (!ins_src[i] || !ins_dst[i])))
      return PR_EINVAL;
    for (int32_t j = 0; j < i; j++)
      if (graphs[j] == graphs[i]) return PR_EINVAL;
  }
  if (count == 0) return PR_OK;
  // each graph's batch runs on a stream of the pool that first waits for the
  // graph's own stream (h->ev[0]); the graph's stream waits for the batch's
  // end (h->ev[1]) before the call returns.  Graphs on another device than the
  // current one stay on their own stream.
  int cur = -1;
  cudaStream_t* pool = nullptr;
  if (cudaGetDevice(&cur) != cudaSuccess || apply_streams(cur, &pool) != cudaSuccess) pool = nullptr;
  std::vector<cudaStream_t> home((size_t)count);
  std::vector<SmallApply> pend((size_t)count);
  std::vector<char> queued((size_t)count, 0), done((size_t)count, 0);
  pr_status first = PR_OK;
  auto fail = [&](pr_status st) {
    if (first == PR_OK) first = st;
  };
  // every graph's work queued first, then each finished: the host waits for
  // the device once per graph, when its work is already under way
  for (int32_t i = 0; i < count; i++) {
    pr_graph* h = graphs[i];
    Graph* g = &h->g;
    g->err.clear();
    const int32_t *ds = del_src[i], *dd = del_dst[i], *is = ins_src[i], *id = ins_dst[i];
    const int64_t nd = n_del[i], ni = n_ins[i];
    if (!device) {   // host arrays: ids checked here, before anything is queued
      const int32_t n = g->n;
      bool bad = false;
      for (int64_t k = 0; k < nd && !bad; k++) bad = ds[k] < 0 || ds[k] >= n || dd[k] < 0 || dd[k] >= n;
      for (int64_t k = 0; k < ni && !bad; k++) bad = is[k] < 0 || is[k] >= n || id[k] < 0 || id[k] >= n;
      if (bad) {
        fail((pr_status)set_error(g, ERANGE_, "pr_apply_batches: vertex id out of range"));
        continue;
      }
    }
    home[i] = g->stream;
    if (cudaEventRecord(h->ev[0], g->stream) != cudaSuccess) {
      fail((pr_status)cuda_fail(g, cudaGetLastError(), "pr_apply_batches"));
      continue;
    }
    if (pool && g->dev == cur) {
      cudaStream_t aux = pool[i % APPLY_STREAMS];
      if (cudaStreamWaitEvent(aux, h->ev[0], 0) != cudaSuccess) {
        fail((pr_status)cuda_fail(g, cudaGetLastError(), "pr_apply_batches"));
        continue;
      }
      g->stream = aux;
    }
    queued[i] = 1;
    if (!device && nd + ni > 0) {   // staged in the graph's scratch (slot 0), as pr_apply_batch does
      void* stage;
      cudaError_t e = scratch_get(g, 0, sizeof(int32_t) * (size_t)(2 * (nd + ni) + 4) + 1024, &stage);
      int32_t* b = (int32_t*)stage;
      if (e == cudaSuccess && nd) e = cudaMemcpyAsync(b, ds, sizeof(int32_t) * nd, cudaMemcpyHostToDevice, g->stream);
      if (e == cudaSuccess && nd)
        e = cudaMemcpyAsync(b + nd, dd, sizeof(int32_t) * nd, cudaMemcpyHostToDevice, g->stream);
      if (e == cudaSuccess && ni)
        e = cudaMemcpyAsync(b + 2 * nd, is, sizeof(int32_t) * ni, cudaMemcpyHostToDevice, g->stream);
      if (e == cudaSuccess && ni)
        e = cudaMemcpyAsync(b + 2 * nd + ni, id, sizeof(int32_t) * ni, cudaMemcpyHostToDevice, g->stream);
      if (e != cudaSuccess) {
        fail((pr_status)cuda_fail(g, e, "pr_apply_batches"));
        continue;
      }
      ds = b;
      dd = b + nd;
      is = b + 2 * nd;
      id = b + 2 * nd + ni;
    }
    int rc = apply_batch_launch(g, ds, dd, nd, is, id, ni, !device, &pend[i]);
    if (rc != OK) {
      fail((pr_status)rc);
      continue;
    }
    done[i] = 1;
  }
  for (int32_t i = 0; i < count; i++) {
    if (!done[i]) continue;
    pr_graph* h = graphs[i];
    int rc = apply_batch_complete(&h->g, &pend[i]);
    pr_status st = rc == OK ? apply_finish(h, false) : (pr_status)rc;
    if (st != PR_OK) {
      done[i] = 0;
      fail(st);
    }
  }
  // back to each graph's own stream: it waits for everything the batch queued
  for (int32_t i = 0; i < count; i++) {
    if (!queued[i]) continue;
    pr_graph* h = graphs[i];
    Graph* g = &h->g;
    if (g->stream != home[i]) {
      cudaError_t e = done[i] ? cudaSuccess : cudaEventRecord(h->ev[1], g->stream);
      if (e == cudaSuccess) e = cudaStreamWaitEvent(home[i], h->ev[1], 0);
      if (e != cudaSuccess) {
        cudaStreamSynchronize(g->stream);   // the ordering the event could not give
        fail((pr_status)cuda_fail(g, e, "pr_apply_batches"));
      }
      g->stream = home[i];
    }
  }
  for (int32_t i = 0; i < count; i++) {
    if (!done[i]) continue;
    pr_graph* h = graphs[i];
    float ms = 0.f;
    if (cudaEventSynchronize(h->ev[1]) == cudaSuccess && cudaEventElapsedTime(&ms, h->ev[0], h->ev[1]) == cudaSuccess)
      h->ms_apply = ms;
  }
  return first;
}

pr_status pr_apply_batches(int32_t count, pr_graph* const* graphs, const int32_t* const* del_src,
                           const int32_t* const* del_dst, const int64_t* n_del, const int32_t* const* ins_src,
                           const int32_t* const* ins_dst, const int64_t* n_ins) {
  NvtxRange r("pr_apply_batches");
  return apply_many(count, graphs, del_src, del_dst, n_del, ins_src, ins_dst, n_ins, false);
}

pr_status pr_apply_batches_device(int32_t count, pr_graph* const* graphs, const int32_t* const* del_src,
                                  const int32_t* const* del_dst, const int64_t* n_del, const int32_t* const* ins_src,
                                  const int32_t* const* ins_dst, const int64_t* n_ins) {
  NvtxRange r("pr_apply_batches_device");
  return apply_many(count, graphs, del_src, del_dst, n_del, ins_src, ins_dst, n_ins, true);
}

pr_status pr_update(pr_graph* h, pr_method method, double alpha, double tau, const pr_options* opts,
                    pr_stats* stats) {
  NvtxRange r("pr_update");
  if (!h) return PR_EINVAL;
  Graph* g = &h->g;
  g->err.clear();
  double tau_f = 1e-6, tau_p = 1e-6;
  int32_t max_iter = 500, flags = 0;
  if (opts) {
    tau_f = opts->tau_f;
    tau_p = opts->tau_p;
    max_iter = opts->max_iter;
    flags = opts->flags;
    if (flags & ~(PR_OPT_TIME_SWEEPS | PR_OPT_FORCE_PULL | PR_OPT_FORCE_PUSH | PR_OPT_DEVICE_LOOP | PR_OPT_HOST_LOOP |
                  PR_OPT_MEASURE_ABSOLUTE | PR_OPT_MEASURE_CONTRIB | PR_OPT_ASYNC | PR_OPT_ONE_KERNEL))
      return PR_EINVAL;
    if ((flags & PR_OPT_ONE_KERNEL) &&
        ((flags & (PR_OPT_DEVICE_LOOP | PR_OPT_HOST_LOOP | PR_OPT_TIME_SWEEPS | PR_OPT_FORCE_PULL | PR_OPT_FORCE_PUSH |
                   PR_OPT_ASYNC)) ||
         method == PR_DYNAMIC_TRAVERSAL))
      return PR_EINVAL;
    if ((flags & PR_OPT_ASYNC) &&
        ((flags & (PR_OPT_DEVICE_LOOP | PR_OPT_FORCE_PUSH)) || method == PR_DYNAMIC_TRAVERSAL))
      return PR_EINVAL;
    if ((flags & PR_OPT_MEASURE_ABSOLUTE) && (flags & PR_OPT_MEASURE_CONTRIB)) return PR_EINVAL;
    if ((flags & PR_OPT_FORCE_PULL) && (flags & PR_OPT_FORCE_PUSH)) return PR_EINVAL;
    if ((flags & PR_OPT_DEVICE_LOOP) &&
        (flags & (PR_OPT_HOST_LOOP | PR_OPT_TIME_SWEEPS | PR_OPT_FORCE_PULL | PR_OPT_FORCE_PUSH)))
      return PR_EINVAL;
  }
  if ((int)method < PR_STATIC || (int)method > PR_DFP) return PR_EINVAL;
  if (!(alpha >= 0.0 && alpha < 1.0) || !(tau >= 0.0) || !(tau_f >= 0.0) || !(tau_p >= 0.0) || max_iter < 0)
    return PR_EINVAL;
  if (method != PR_STATIC && !g->has_ranks)
    return (pr_status)set_error(g, ENORANKS_, "pr_update: a dynamic method needs ranks (pr_set_ranks or a previous update)");
  const bool host_flags =
      flags & (PR_OPT_HOST_LOOP | PR_OPT_TIME_SWEEPS | PR_OPT_FORCE_PULL | PR_OPT_FORCE_PUSH | PR_OPT_ASYNC);
  const bool loopable = method != PR_DYNAMIC_TRAVERSAL;
  if (loopable &&
      ((flags & (PR_OPT_DEVICE_LOOP | PR_OPT_ONE_KERNEL)) || (!host_flags && g->in.cap < PR_DEVICE_LOOP_SLOTS))) {
    // the iteration loop on the device: a group of this one graph, on its stream
    if (!h->solo) {
      pr_graph* one[1] = {h};
      pr_status st = pr_group_create(1, one, g->stream, &h->solo);
      if (st != PR_OK) return st;
    }
    // PR_OPT_DEVICE_LOOP keeps the CUDA graph, PR_OPT_ONE_KERNEL asks for one
    // kernel, neither lets the group choose by size
    pr_options o = {tau_f, tau_p, max_iter,
                    flags & (PR_OPT_MEASURE_ABSOLUTE | PR_OPT_MEASURE_CONTRIB | PR_OPT_DEVICE_LOOP | PR_OPT_ONE_KERNEL)};
    return pr_group_update(h->solo, method, alpha, tau, &o, stats);
  }
  return run_update(h, (int)method, alpha, tau, tau_f, tau_p, max_iter, flags, stats);
}

pr_status pr_ranks_device(const pr_graph* hc, double* out) {
  pr_graph* h = const_cast<pr_graph*>(hc);
  if (!h || !out) return PR_EINVAL;
  Graph* g = &h->g;
  if (!g->has_ranks) return PR_ENORANKS;
  TRY(launch_gather_f64(g->R, g->perm, out, g->n, g->stream));
  TRY(cudaStreamSynchronize(g->stream));
  return PR_OK;
}

pr_status pr_ranks(const pr_graph* hc, double* out) {
  pr_graph* h = const_cast<pr_graph*>(hc);
  if (!h || !out) return PR_EINVAL;
  Graph* g = &h->g;
  if (!g->has_ranks) return PR_ENORANKS;
  TRY(launch_gather_f64(g->R, g->perm, h->vec_tmp, g->n, g->stream));
  TRY(cudaMemcpyAsync(out, h->vec_tmp, sizeof(double) * g->n, cudaMemcpyDeviceToHost, g->stream));
  TRY(cudaStreamSynchronize(g->stream));
  return PR_OK;
}

static pr_status set_ranks_from_device(pr_graph* h, const double* dev) {
  Graph* g = &h->g;
  cudaStream_t s = g->stream;
  TRY(launch_scatter_f64(dev, g->perm, g->R, g->n, s));
  TRY(launch_contrib_all(g->R, g->C[g->ccur], g->out.deg, g->tab_sc, g->n, s));
  TRY(cudaStreamSynchronize(s));
  g->has_ranks = true;
  return PR_OK;
}

pr_status pr_set_ranks(pr_graph* h, const double* r) {
  if (!h || !r) return PR_EINVAL;
  Graph* g = &h->g;
  double sum = 0.0;
  for (int32_t i = 0; i < g->n; i++) {
    if (!(r[i] >= 0.0) || !std::isfinite(r[i])) return (pr_status)set_error(g, EINVAL_, "pr_set_ranks: bad rank");
    sum += r[i];
  }
  if (sum > 2.0) return (pr_status)set_error(g, EINVAL_, "pr_set_ranks: ranks sum above 2");
  TRY(cudaMemcpyAsync(h->vec_tmp, r, sizeof(double) * g->n, cudaMemcpyHostToDevice, g->stream));
  return set_ranks_from_device(h, h->vec_tmp);
}

pr_status pr_set_ranks_device(pr_graph* h, const double* r) {
  if (!h || !r) return PR_EINVAL;
  Graph* g = &h->g;
  cudaStream_t s = g->stream;
  struct {
    unsigned long long bad;
    double sum;
  } hv, *dv = (decltype(dv))h->vec_tmp;
  TRY(cudaMemsetAsync(dv, 0, sizeof(hv), s));
  note_launch(); k_check_ranks<<<grid_for(g->n, 256), 256, 0, s>>>(r, g->n, &dv->bad, &dv->sum);
  TRY(cudaMemcpyAsync(&hv, dv, sizeof(hv), cudaMemcpyDeviceToHost, s));
  TRY(cudaStreamSynchronize(s));
  if (hv.bad || hv.sum > 2.0) return (pr_status)set_error(g, EINVAL_, "pr_set_ranks_device: bad ranks");
  return set_ranks_from_device(h, r);
}

// Vertex insertion / deletion (pr_graph_resize): the edge set in user ids,
// rebuilt with the new vertex count.
}  // extern "C"

// any user id at or above n_new that has an edge besides its self-loop
__global__ void k_removed_isolated(const int32_t* __restrict__ iperm, const int32_t* __restrict__ odeg,
                                   const int32_t* __restrict__ ideg, int32_t n, int32_t n_new, int32_t* bad) {
  for (int64_t u = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; u < n; u += (int64_t)gridDim.x * blockDim.x)
    if (iperm[u] >= n_new && (odeg[u] != 1 || ideg[u] != 1)) *bad = 1;
}

__global__ void k_degrees_i64(const int32_t* __restrict__ deg, int32_t n, int64_t* __restrict__ out) {
  for (int64_t u = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; u < n; u += (int64_t)gridDim.x * blockDim.x)
    out[u] = deg[u];
}

// one warp per internal out-row: its edges as user-id keys packed with `bits`
// (the new graph's id width) at pos[u]..; an edge with an end at or above
// n_new (the self-loop of a removed vertex) becomes the key of vertex 0's
// self-loop, which the build collapses.  Then one self-loop key per vertex of
// the new graph.
__global__ void k_export_keys(const int64_t* __restrict__ off, const int32_t* __restrict__ deg,
                              const int32_t* __restrict__ col, const int32_t* __restrict__ iperm,
                              const int64_t* __restrict__ pos, int32_t n, int32_t n_new, int bits,
                              uint64_t* __restrict__ keys) {
  const int lane = threadIdx.x & 31;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t u = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; u < n; u += nw) {
    const int32_t su = iperm[u];
    for (int64_t x = lane; x < deg[u]; x += 32) {
      const int32_t sv = iperm[col[off[u] + x]];
      keys[pos[u] + x] = su < n_new && sv < n_new ? ((uint64_t)su << bits) | (uint64_t)sv : 0ull;
    }
  }
}

__global__ void k_self_loop_keys(int32_t n_new, int bits, uint64_t* __restrict__ keys) {
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n_new; v += (int64_t)gridDim.x * blockDim.x)
    keys[v] = ((uint64_t)v << bits) | (uint64_t)v;
}

// r'[v] = r[v] * ratio for the vertices kept, 1/n_new for the new ones (user ids)
__global__ void k_resize_ranks(const double* __restrict__ r, int32_t n, int32_t n_new, double ratio,
                               double* __restrict__ out) {
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n_new; v += (int64_t)gridDim.x * blockDim.x)
    out[v] = v < n ? r[v] * ratio : 1.0 / (double)n_new;
}

extern "C" {

pr_status pr_graph_resize(pr_graph* h, int32_t n_new) {
  if (!h) return PR_EINVAL;
  Graph* g = &h->g;
  const int32_t n = g->n;
  if (n_new < 1) return (pr_status)set_error(g, EINVAL_, "pr_graph_resize: n_new < 1");
  if ((int64_t)n_new + g->m >= (int64_t(1) << 31))
    return (pr_status)set_error(g, EINVAL_, "pr_graph_resize: too many vertices and edges");
  if (n_new == n) return PR_OK;
  cudaStream_t s = g->stream;
  if (n_new < n) {
    DevBuf<int32_t> bad;
    TRY(bad.alloc(1));
    TRY(cudaMemsetAsync(bad.p, 0, sizeof(int32_t), s));
    note_launch();
    k_removed_isolated<<<grid_for(n, 256), 256, 0, s>>>(g->iperm, g->out.deg, g->in.deg, n, n_new, bad.p);
    int32_t hb = 0;
    TRY(cudaMemcpyAsync(&hb, bad.p, sizeof(hb), cudaMemcpyDeviceToHost, s));
    TRY(cudaStreamSynchronize(s));
    if (hb) return (pr_status)set_error(g, EINVAL_, "pr_graph_resize: a removed vertex still has edges");
  }
  // the edges in user ids, then the self-loops of the new vertex set
  const int64_t m = g->m;
  const int nb = bits_for(n_new);
  DevBuf<int64_t> pos, stmp;
  uint64_t* keys = nullptr;
  TRY(pos.alloc(n + 1));
  TRY(stmp.alloc(scan_tmp_elems(n)));
  note_launch();
  k_degrees_i64<<<grid_for(n, 256), 256, 0, s>>>(g->out.deg, n, pos.p);
  TRY(scan_excl<int64_t>(pos.p, pos.p, n, stmp.p, s));
  TRY(dev_malloc(&keys, sizeof(uint64_t) * (size_t)(m + n_new)));
  note_launch();
  k_export_keys<<<grid_for((int64_t)n * 32, 256), 256, 0, s>>>(g->out.off, g->out.deg, g->out.col, g->iperm, pos.p,
                                                                n, n_new, nb, keys);
  note_launch();
  k_self_loop_keys<<<grid_for(n_new, 256), 256, 0, s>>>(n_new, nb, keys + m);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    cudaFree(keys);
    return (pr_status)cuda_fail(g, e, "pr_graph_resize: keys");
  }
  pr_graph* h2 = new (std::nothrow) pr_graph();
  if (!h2) {
    cudaFree(keys);
    return PR_ENOMEM;
  }
  Graph* g2 = &h2->g;
  g2->n = n_new;
  g2->id_bits = nb;
  g2->stream = s;
  g2->relabel = g->relabel;
  g2->dev = g->dev;
  pr_graph* made = nullptr;
  pr_status st = finish_create(h2, keys, m + n_new, &made);
  cudaFree(keys);
  if (st == PR_OK && g->has_ranks) {
    // ranks in user order, carried over to the new vertex set
    e = launch_gather_f64(g->R, g->perm, h->vec_tmp, n, s);
    if (e == cudaSuccess) {
      note_launch();
      k_resize_ranks<<<grid_for(n_new, 256), 256, 0, s>>>(h->vec_tmp, n, n_new, (double)n / (double)n_new,
                                                           h2->vec_tmp);
      e = cudaGetLastError();
    }
    st = e == cudaSuccess ? set_ranks_from_device(h2, h2->vec_tmp) : (pr_status)cuda_fail(g, e, "pr_graph_resize");
  }
  if (st != PR_OK) {
    if (st != PR_ENOMEM && st != PR_ECUDA) g->err = g2->err;
    destroy_handle(h2);
    return st;
  }
  // the new state moves into the caller's handle; the old one is freed with h2
  if (h->solo) {
    pr_group_destroy(h->solo);
    h->solo = nullptr;
  }
  std::swap(h->g, h2->g);
  std::swap(h->lbits_tmp, h2->lbits_tmp);
  std::swap(h->ls_tmp, h2->ls_tmp);
  std::swap(h->vec_tmp, h2->vec_tmp);
  std::swap(h->tiles_cap, h2->tiles_cap);
  destroy_handle(h2);
  return PR_OK;
}

pr_status pr_sweep_log(const pr_graph* h, pr_sweep_record* out, int32_t cap, int32_t* count) {
  if (!h || !count || cap < 0 || (cap > 0 && !out)) return PR_EINVAL;
  const int32_t k = (int32_t)h->sweep_log.size();
  for (int32_t i = 0; i < k && i < cap; i++) out[i] = h->sweep_log[i];
  *count = k;
  return PR_OK;
}

pr_status pr_graph_info(const pr_graph* h, int32_t* n, int64_t* m) {
  if (!h) return PR_EINVAL;
  if (n) *n = h->g.n;
  if (m) *m = h->g.m;
  return PR_OK;
}

pr_status pr_get_csr(const pr_graph* hc, int32_t which, int64_t* off, int32_t* adj) {
  pr_graph* h = const_cast<pr_graph*>(hc);
  if (!h || !off || !adj || (which != 0 && which != 1)) return PR_EINVAL;
  Graph* g = &h->g;
  const Csr& c = which == 0 ? g->out : g->in;
  int32_t n = g->n;
  std::vector<int64_t> o(n + 1);
  std::vector<int32_t> d(n), col(c.cap), perm(n), iperm(n);
  cudaStream_t s = g->stream;
  TRY(cudaMemcpyAsync(o.data(), c.off, sizeof(int64_t) * (n + 1), cudaMemcpyDeviceToHost, s));
  TRY(cudaMemcpyAsync(d.data(), c.deg, sizeof(int32_t) * n, cudaMemcpyDeviceToHost, s));
  TRY(cudaMemcpyAsync(col.data(), c.col, sizeof(int32_t) * c.cap, cudaMemcpyDeviceToHost, s));
  TRY(cudaMemcpyAsync(perm.data(), g->perm, sizeof(int32_t) * n, cudaMemcpyDeviceToHost, s));
  TRY(cudaMemcpyAsync(iperm.data(), g->iperm, sizeof(int32_t) * n, cudaMemcpyDeviceToHost, s));
  TRY(cudaStreamSynchronize(s));
  int64_t w = 0;
  for (int32_t u = 0; u < n; u++) {
    off[u] = w;
    int32_t r = perm[u];
    int64_t start = w;
    for (int32_t x = 0; x < d[r]; x++) adj[w++] = iperm[col[o[r] + x]];
    std::sort(adj + start, adj + w);
  }
  off[n] = w;
  return PR_OK;
}

pr_status pr_get_rows(const pr_graph* hc, int32_t which, int64_t count, const int32_t* vertices, int64_t* off,
                      int32_t* adj) {
  pr_graph* h = const_cast<pr_graph*>(hc);
  if (!h || count < 0 || (count > 0 && !vertices) || !off || (which != 0 && which != 1)) return PR_EINVAL;
  Graph* g = &h->g;
  const Csr& c = which == 0 ? g->out : g->in;
  int32_t n = g->n;
  for (int64_t k = 0; k < count; k++)
    if (vertices[k] < 0 || vertices[k] >= n) return (pr_status)set_error(g, ERANGE_, "pr_get_rows: vertex id out of range");
  off[0] = 0;
  if (count == 0) return PR_OK;
  cudaStream_t s = g->stream;
  // device side: map the ids, gather degree and row start of every vertex
  DevBuf<int32_t> dv, ddeg;
  DevBuf<int64_t> dbase;
  TRY(dv.alloc(count));
  TRY(ddeg.alloc(count));
  TRY(dbase.alloc(count));
  TRY(cudaMemcpyAsync(dv.p, vertices, sizeof(int32_t) * count, cudaMemcpyHostToDevice, s));
  int grid = grid_for(count, 256);
  note_launch();
  k_row_meta<<<grid, 256, 0, s>>>(dv.p, count, g->perm, c.off, c.deg, ddeg.p, dbase.p);
  TRY(cudaGetLastError());
  std::vector<int32_t> deg(count);
  TRY(cudaMemcpyAsync(deg.data(), ddeg.p, sizeof(int32_t) * count, cudaMemcpyDeviceToHost, s));
  TRY(cudaStreamSynchronize(s));
  for (int64_t k = 0; k < count; k++) off[k + 1] = off[k] + deg[k];
  if (!adj || off[count] == 0) return PR_OK;
  DevBuf<int64_t> doff;
  DevBuf<int32_t> dadj;
  TRY(doff.alloc(count + 1));
  TRY(dadj.alloc(off[count]));
  TRY(cudaMemcpyAsync(doff.p, off, sizeof(int64_t) * (count + 1), cudaMemcpyHostToDevice, s));
  note_launch();
  k_row_copy_out<<<grid_for(count * 32, 256), 256, 0, s>>>(count, dbase.p, doff.p, c.col, g->iperm, dadj.p);
  TRY(cudaGetLastError());
  TRY(cudaMemcpyAsync(adj, dadj.p, sizeof(int32_t) * off[count], cudaMemcpyDeviceToHost, s));
  TRY(cudaStreamSynchronize(s));
  for (int64_t k = 0; k < count; k++) std::sort(adj + off[k], adj + off[k + 1]);
  return PR_OK;
}

pr_status pr_last_delta(const pr_graph* hc, int64_t* n_del, int64_t* n_ins, int32_t* del_src, int32_t* del_dst,
                        int32_t* ins_src, int32_t* ins_dst) {
  pr_graph* h = const_cast<pr_graph*>(hc);
  if (!h) return PR_EINVAL;
  Graph* g = &h->g;
  if (n_del) *n_del = g->n_dmin;
  if (n_ins) *n_ins = g->n_dplus;
  int32_t n = g->n;
  std::vector<int32_t> iperm(n);
  TRY(cudaMemcpy(iperm.data(), g->iperm, sizeof(int32_t) * n, cudaMemcpyDeviceToHost));
  uint64_t mask = (1ull << g->id_bits) - 1;
  for (int side = 0; side < 2; side++) {
    int64_t k = side ? g->n_dplus : g->n_dmin;
    int32_t* os = side ? ins_src : del_src;
    int32_t* od = side ? ins_dst : del_dst;
    if (!k || !os || !od) continue;
    std::vector<uint64_t> keys(k);
    TRY(cudaMemcpy(keys.data(), side ? g->dplus : g->dmin, sizeof(uint64_t) * k, cudaMemcpyDeviceToHost));
    std::vector<std::pair<int32_t, int32_t>> e(k);
    for (int64_t i = 0; i < k; i++) e[i] = {iperm[keys[i] >> g->id_bits], iperm[keys[i] & mask]};
    std::sort(e.begin(), e.end());
    for (int64_t i = 0; i < k; i++) {
      os[i] = e[i].first;
      od[i] = e[i].second;
    }
  }
  return PR_OK;
}

pr_status pr_affected(pr_graph* h, int32_t which, uint8_t* flags) {
  if (!h || !flags || (which != 0 && which != 1)) return PR_EINVAL;
  Graph* g = &h->g;
  cudaStream_t s = g->stream;
  pr_status st = which == 0 ? initial_marking(h) : dt_affected(h);
  if (st != PR_OK) return st;
  uint8_t* tmp = (uint8_t*)h->vec_tmp;
  if (which == 0) { note_launch(); k_bits_to_bytes<<<grid_for(g->n, 256), 256, 0, s>>>(g->bits[0], nullptr, g->perm, g->n, tmp); }
  else { note_launch(); k_bits_to_bytes<<<grid_for(g->n, 256), 256, 0, s>>>(g->aux, g->aux2, g->perm, g->n, tmp); }
  TRY(cudaMemcpyAsync(flags, tmp, g->n, cudaMemcpyDeviceToHost, s));
  TRY(cudaStreamSynchronize(s));
  return PR_OK;
}

unsigned long long pr_kernel_launches(void) { return launches_so_far(); }

const char* pr_last_error(const pr_graph* h) { return h ? h->g.err.c_str() : ""; }

void pr_debug_fail_alloc(int64_t k) { arm_alloc_failure(k); }

const char* pr_status_string(pr_status s) {
  switch (s) {
    case PR_OK: return "PR_OK";
    case PR_EINVAL: return "PR_EINVAL";
    case PR_ERANGE: return "PR_ERANGE";
    case PR_ENOMEM: return "PR_ENOMEM";
    case PR_ENORANKS: return "PR_ENORANKS";
    case PR_ECUDA: return "PR_ECUDA";
    case PR_ETIMEOUT: return "PR_ETIMEOUT";
  }
  return "unknown";
}

}  // extern "C"
