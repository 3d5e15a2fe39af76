/*
 * dfpr_oracle.c -- plain, slow, single-threaded FP64 reference for the
 * Dynamic Frontier (DF) and Dynamic Frontier with Pruning (DF-P) PageRank
 * update of arXiv 2401.15870 and for its comparators (Static, Naive-dynamic,
 * Dynamic Traversal).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the oracle that the CUDA library is
 * checked against.  It shares no code, header, table or helper with the CUDA
 * path, and nothing in the product path may link, load or call it: only the
 * tests, the package smoke check and the benchmark's CPU-baseline leg do.
 *
 * Everything is written for readability against the paper, not for speed:
 *   - a graph is the sorted set of its edge keys (src << 32 | dst), with
 *     exactly one self-loop on every vertex (Sec. 5.1.3, Sec. 5.1.4: self-loops
 *     are added to all vertices, so there are no dead ends);
 *   - out- and in-adjacency lists are rebuilt from that set after every batch;
 *   - every method runs in the synchronous (Jacobi) order: all vertices
 *     processed in iteration i read the ranks R_i of the start of the iteration
 *     (Sec. 4.4 runs Alg. 1 asynchronously with one rank vector, which leaves
 *     the schedule undefined; the synchronous order is one legal interleaving
 *     of its parallel loop and is reproducible).
 *
 * Readings of points where the paper is silent (each is also listed in the
 * design notes):
 *   - set semantics for batches: E_t = (E_{t-1} \ D) u I, deletions first,
 *     duplicate and ineffective entries have no effect (Sec. 3.2 defines the
 *     deletions and insertions as set differences);
 *   - a deletion of a self-loop is ignored: self-loops are re-added with every
 *     batch (Sec. 5.1.4, Sec. 5.2.2);
 *   - the initial marking of Alg. 1 marks (G_{t-1} u G_t).out(u) for every
 *     updated edge (u, v); that set contains u itself through its self-loop;
 *   - Delta r / max(r, R[v]) uses the larger of the new and the old rank
 *     (Sec. 4.2);
 *   - prune when the relative change is <= tau_p, expand when it is > tau_f,
 *     stop when the L-infinity change is <= tau (Alg. 1);
 *   - when a vertex is pruned and also re-marked by an expansion in the same
 *     iteration, the mark wins: F_{i+1} = M_i u (F_i \ P_i);
 *   - Dynamic Traversal marks the union of the vertices reachable from the
 *     updated sources in G_{t-1} and those reachable in G_t (Sec. 3.3.2);
 *   - the other expansion measures of Sec. 4.3 (dr, dr / d) are compared with
 *     tau_p for pruning too, and the asynchronous order (or_update_ex) visits
 *     vertices in ascending id with the flags of Alg. 1 taking effect at once.
 *
 * Build: gcc -O2 -std=c11 -shared -fPIC dfpr_oracle.c -o liboracle.so
 * (no -ffast-math: IEEE round-to-nearest FP64 throughout).
 *
 * The same source built with -fopenmp (liboracle_omp.so) spreads the
 * synchronous sweeps, the sorts and the adjacency rebuild over the host's
 * cores, so that the oracle can also run the large workloads.  Each vertex of
 * a synchronous sweep is still computed alone, by the same instructions on the
 * same inputs (the ranks of the start of the iteration), and flags are only
 * ever set to one value in an iteration; maxima, minima and counts do not
 * depend on the order they are combined in.  The threaded build therefore
 * returns bit for bit what the single-threaded build returns.  The
 * asynchronous order stays sequential in both.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>
#ifdef _OPENMP
#include <omp.h>
#endif

enum { OR_STATIC = 0, OR_NAIVE_DYNAMIC = 1, OR_DYNAMIC_TRAVERSAL = 2, OR_DF = 3, OR_DFP = 4 };
enum { OR_OK = 0, OR_EINVAL = 1, OR_ERANGE = 2, OR_ENOMEM = 3, OR_ENORANKS = 4 };

typedef struct {
  int32_t n;
  int64_t m;             /* |E_t|, self-loops included */
  uint64_t *keys;        /* sorted unique edge keys of E_t */
  int64_t *out_off;      /* n+1: out-rows of E_t, each sorted by target */
  int32_t *out_adj;
  int64_t *in_off;       /* n+1: in-rows of E_t, each sorted by source */
  int32_t *in_adj;
  int64_t m_prev;        /* E_{t-1} of the last batch */
  uint64_t *keys_prev;
  int64_t n_del, n_ins;  /* effective Delta- = E_{t-1} \ E_t, Delta+ = E_t \ E_{t-1} */
  uint64_t *del, *ins;
} or_graph;

typedef struct {
  int32_t iterations, converged;
  double delta_R;
  int64_t vertices_ever_affected;
  int64_t edges_processed;
  int64_t vertices_processed;
  /* the smallest relative distance |x / t - 1| between a compared quantity x
   * and its threshold t over every decision of the run: the frontier measure
   * against tau_f (expand) and tau_p (prune), and Delta R against tau (stop).
   * A second implementation whose ranks differ slightly from these can take a
   * decision the other way only where this is small; the tests use it to tell
   * a genuine near-tie from a different frontier.  Thresholds of 0 or
   * infinity take no part; INFINITY when nothing was compared. */
  double tie_rel;
} or_stats;

static uint64_t key_of(int32_t u, int32_t v) { return ((uint64_t)(uint32_t)u << 32) | (uint32_t)v; }
static int32_t key_src(uint64_t k) { return (int32_t)(k >> 32); }
static int32_t key_dst(uint64_t k) { return (int32_t)(k & 0xffffffffu); }

static int cmp_u64(const void *a, const void *b) {
  uint64_t x = *(const uint64_t *)a, y = *(const uint64_t *)b;
  return (x > y) - (x < y);
}

static int cmp_i32(const void *a, const void *b) {
  int32_t x = *(const int32_t *)a, y = *(const int32_t *)b;
  return (x > y) - (x < y);
}

/* threads of the OpenMP build (1 in the plain build) */
static int n_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}
int or_threads(void) { return n_threads(); }
void or_set_threads(int t) {
#ifdef _OPENMP
  if (t > 0) omp_set_num_threads(t);
#else
  (void)t;
#endif
}

/* merge the sorted runs a[0..la) and b[0..lb) into out */
static void merge_u64(const uint64_t *a, int64_t la, const uint64_t *b, int64_t lb, uint64_t *out) {
  int64_t i = 0, j = 0, w = 0;
  while (i < la && j < lb) out[w++] = (b[j] < a[i]) ? b[j++] : a[i++];
  while (i < la) out[w++] = a[i++];
  while (j < lb) out[w++] = b[j++];
}

/* ascending sort of k[0..len): one qsort, or with several threads one qsort
 * per thread over equal runs followed by rounds of pairwise merges */
static void sort_u64(uint64_t *k, int64_t len) {
  int T = n_threads();
  if (T <= 1 || len < ((int64_t)1 << 22)) {
    qsort(k, (size_t)len, sizeof(uint64_t), cmp_u64);
    return;
  }
  int64_t *bnd = (int64_t *)malloc(sizeof(int64_t) * (size_t)(T + 1));
  uint64_t *tmp = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)len);
  if (!bnd || !tmp) {
    free(bnd); free(tmp);
    qsort(k, (size_t)len, sizeof(uint64_t), cmp_u64);
    return;
  }
  for (int i = 0; i <= T; i++) bnd[i] = len / T * i + (len % T) * i / T;
  bnd[T] = len;
#pragma omp parallel for schedule(static, 1)
  for (int i = 0; i < T; i++) qsort(k + bnd[i], (size_t)(bnd[i + 1] - bnd[i]), sizeof(uint64_t), cmp_u64);
  uint64_t *from = k, *to = tmp;
  for (int w = 1; w < T; w *= 2) {
#pragma omp parallel for schedule(dynamic, 1)
    for (int i = 0; i < T; i += 2 * w) {
      int mid = i + w < T ? i + w : T, hi = i + 2 * w < T ? i + 2 * w : T;
      merge_u64(from + bnd[i], bnd[mid] - bnd[i], from + bnd[mid], bnd[hi] - bnd[mid], to + bnd[i]);
    }
    uint64_t *x = from; from = to; to = x;
  }
  if (from != k) memcpy(k, from, sizeof(uint64_t) * (size_t)len);
  free(tmp); free(bnd);
}

/* sort and drop repeated keys in place; returns the new length */
static int64_t sort_unique(uint64_t *k, int64_t len) {
  if (len == 0) return 0;
  sort_u64(k, len);
  int64_t w = 1;
  for (int64_t i = 1; i < len; i++)
    if (k[i] != k[w - 1]) k[w++] = k[i];
  return w;
}

static int contains(const uint64_t *k, int64_t len, uint64_t x) {
  int64_t lo = 0, hi = len;
  while (lo < hi) {
    int64_t mid = lo + (hi - lo) / 2;
    if (k[mid] < x) lo = mid + 1; else hi = mid;
  }
  return lo < len && k[lo] == x;
}

/* first index with k[i] >= x */
static int64_t lower_bound(const uint64_t *k, int64_t len, uint64_t x) {
  int64_t lo = 0, hi = len;
  while (lo < hi) {
    int64_t mid = lo + (hi - lo) / 2;
    if (k[mid] < x) lo = mid + 1; else hi = mid;
  }
  return lo;
}

/* a \ b for sorted unique arrays; out has room for len_a */
static int64_t set_minus(const uint64_t *a, int64_t la, const uint64_t *b, int64_t lb, uint64_t *out) {
  int64_t i = 0, j = 0, w = 0;
  while (i < la) {
    while (j < lb && b[j] < a[i]) j++;
    if (j < lb && b[j] == a[i]) { i++; continue; }
    out[w++] = a[i++];
  }
  return w;
}

/* a u b for sorted unique arrays; out has room for la + lb */
static int64_t set_union(const uint64_t *a, int64_t la, const uint64_t *b, int64_t lb, uint64_t *out) {
  int64_t i = 0, j = 0, w = 0;
  while (i < la || j < lb) {
    if (j >= lb || (i < la && a[i] < b[j])) out[w++] = a[i++];
    else if (i >= la || b[j] < a[i]) out[w++] = b[j++];
    else { out[w++] = a[i++]; j++; }
  }
  return w;
}

/* rebuild out- and in-adjacency (CSR) from the sorted key set */
static int rebuild_adjacency(or_graph *g) {
  int32_t n = g->n;
  int64_t m = g->m;
  free(g->out_off); free(g->out_adj); free(g->in_off); free(g->in_adj);
  g->out_off = (int64_t *)calloc((size_t)n + 1, sizeof(int64_t));
  g->in_off = (int64_t *)calloc((size_t)n + 1, sizeof(int64_t));
  g->out_adj = (int32_t *)malloc(sizeof(int32_t) * (size_t)(m > 0 ? m : 1));
  g->in_adj = (int32_t *)malloc(sizeof(int32_t) * (size_t)(m > 0 ? m : 1));
  if (!g->out_off || !g->in_off || !g->out_adj || !g->in_adj) return OR_ENOMEM;
  /* keys are sorted by (src, dst): out-row u is the key range of source u,
   * already sorted by dst */
#pragma omp parallel for schedule(static)
  for (int64_t v = 0; v <= (int64_t)n; v++)
    g->out_off[v] = v == n ? m : lower_bound(g->keys, m, key_of((int32_t)v, 0));
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < m; i++) {
    g->out_adj[i] = key_dst(g->keys[i]);
    int32_t d = key_dst(g->keys[i]);
#pragma omp atomic
    g->in_off[d + 1]++;
  }
  for (int32_t v = 0; v < n; v++) g->in_off[v + 1] += g->in_off[v];
  /* bucket by dst: in key order this gives in-rows sorted by src; threads
   * fill the buckets in any order, and each in-row is sorted afterwards */
  int64_t *fill = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
  if (!fill) return OR_ENOMEM;
  for (int32_t v = 0; v < n; v++) fill[v] = g->in_off[v];
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < m; i++) {
    int32_t d = key_dst(g->keys[i]);
    int64_t at;
#pragma omp atomic capture
    at = fill[d]++;
    g->in_adj[at] = key_src(g->keys[i]);
  }
  free(fill);
  if (n_threads() > 1) {
#pragma omp parallel for schedule(dynamic, 4096)
    for (int32_t v = 0; v < n; v++)
      qsort(g->in_adj + g->in_off[v], (size_t)(g->in_off[v + 1] - g->in_off[v]), sizeof(int32_t), cmp_i32);
  }
  return OR_OK;
}

void or_graph_destroy(or_graph *g) {
  if (!g) return;
  free(g->keys); free(g->out_off); free(g->out_adj); free(g->in_off); free(g->in_adj);
  free(g->keys_prev); free(g->del); free(g->ins);
  free(g);
}

/* Graph from a raw edge list (repeats and self-loops allowed): the edge set
 * with exactly one self-loop per vertex (Sec. 5.1.3). */
int or_graph_create(int32_t n, int64_t m, const int32_t *src, const int32_t *dst, or_graph **out) {
  *out = NULL;
  if (n <= 0 || m < 0) return OR_EINVAL;
  for (int64_t i = 0; i < m; i++)
    if (src[i] < 0 || src[i] >= n || dst[i] < 0 || dst[i] >= n) return OR_ERANGE;
  or_graph *g = (or_graph *)calloc(1, sizeof(or_graph));
  if (!g) return OR_ENOMEM;
  g->n = n;
  g->keys = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)(m + n));
  if (!g->keys) { free(g); return OR_ENOMEM; }
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < m; i++) g->keys[i] = key_of(src[i], dst[i]);
  for (int32_t v = 0; v < n; v++) g->keys[m + v] = key_of(v, v);
  g->m = sort_unique(g->keys, m + n);
  int rc = rebuild_adjacency(g);
  if (rc != OR_OK) { or_graph_destroy(g); return rc; }
  *out = g;
  return OR_OK;
}

/* Batch update (Sec. 3.2): E_t = (E_{t-1} \ D) u I with self-loop deletions
 * ignored; records the effective Delta- = E_{t-1} \ E_t and Delta+ = E_t \ E_{t-1}.
 * Ids are validated before anything changes. */
int or_apply_batch(or_graph *g, const int32_t *del_src, const int32_t *del_dst, int64_t n_del,
                   const int32_t *ins_src, const int32_t *ins_dst, int64_t n_ins) {
  int32_t n = g->n;
  if (n_del < 0 || n_ins < 0) return OR_EINVAL;
  for (int64_t i = 0; i < n_del; i++)
    if (del_src[i] < 0 || del_src[i] >= n || del_dst[i] < 0 || del_dst[i] >= n) return OR_ERANGE;
  for (int64_t i = 0; i < n_ins; i++)
    if (ins_src[i] < 0 || ins_src[i] >= n || ins_dst[i] < 0 || ins_dst[i] >= n) return OR_ERANGE;

  uint64_t *D = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)(n_del > 0 ? n_del : 1));
  uint64_t *I = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)(n_ins > 0 ? n_ins : 1));
  if (!D || !I) { free(D); free(I); return OR_ENOMEM; }
  int64_t nd = 0, ni = 0;
  for (int64_t i = 0; i < n_del; i++)
    if (del_src[i] != del_dst[i]) D[nd++] = key_of(del_src[i], del_dst[i]);
  for (int64_t i = 0; i < n_ins; i++) I[ni++] = key_of(ins_src[i], ins_dst[i]);
  nd = sort_unique(D, nd);
  ni = sort_unique(I, ni);

  uint64_t *kept = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)(g->m > 0 ? g->m : 1));
  uint64_t *next = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)(g->m + ni + 1));
  if (!kept || !next) { free(D); free(I); free(kept); free(next); return OR_ENOMEM; }
  int64_t nk = set_minus(g->keys, g->m, D, nd, kept);
  int64_t nn = set_union(kept, nk, I, ni, next);
  free(kept); free(D); free(I);

  uint64_t *dm = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)(g->m + 1));
  uint64_t *dp = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)(nn + 1));
  if (!dm || !dp) { free(dm); free(dp); free(next); return OR_ENOMEM; }
  int64_t ndm = set_minus(g->keys, g->m, next, nn, dm);
  int64_t ndp = set_minus(next, nn, g->keys, g->m, dp);

  free(g->keys_prev); free(g->del); free(g->ins);
  g->keys_prev = g->keys; g->m_prev = g->m;
  g->keys = next; g->m = nn;
  g->del = dm; g->n_del = ndm;
  g->ins = dp; g->n_ins = ndp;
  return rebuild_adjacency(g);
}

/* Vertex insertion and deletion at the end of the id range (|V| fixed in the
 * paper's experiments, Sec. 5.2.2; its temporal graphs gain vertices over
 * time, Sec. 5.1.4): |V| becomes n_new.  Added vertices get their self-loop
 * only (Sec. 5.1.3); removed vertices must have no edge but their self-loop.
 * The last batch's effective change is cleared. */
int or_graph_resize(or_graph *g, int32_t n_new) {
  if (n_new < 1) return OR_EINVAL;
  int32_t n = g->n;
  for (int32_t v = n_new; v < n; v++)
    if (g->out_off[v + 1] - g->out_off[v] != 1 || g->in_off[v + 1] - g->in_off[v] != 1) return OR_EINVAL;
  /* keys are sorted by source: the edges of the removed vertices (their
   * self-loops) are the tail, and self-loops of added vertices sort after
   * every existing key */
  int64_t keep = n_new < n ? lower_bound(g->keys, g->m, key_of(n_new, 0)) : g->m;
  int64_t m_new = keep + (n_new > n ? (int64_t)(n_new - n) : 0);
  uint64_t *k = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)m_new);
  uint64_t *kp = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)m_new);
  if (!k || !kp) { free(k); free(kp); return OR_ENOMEM; }
  memcpy(k, g->keys, sizeof(uint64_t) * (size_t)keep);
  for (int32_t v = n; v < n_new; v++) k[keep + (v - n)] = key_of(v, v);
  memcpy(kp, k, sizeof(uint64_t) * (size_t)m_new);
  free(g->keys); free(g->keys_prev);
  g->keys = k; g->m = m_new;
  g->keys_prev = kp; g->m_prev = m_new;   /* no batch since: Delta- = Delta+ = {} */
  g->n_del = g->n_ins = 0;
  g->n = n_new;
  return rebuild_adjacency(g);
}

/* The previous snapshot's ranks carried over a resize.  Eq. 1 on n vertices
 * is r = (1 - alpha)/n + alpha P^T r; multiplying a solution by n / n_new
 * gives (1 - alpha)/n_new + alpha P^T r', the same equation on n_new vertices
 * (adding or removing isolated vertices leaves P of the others unchanged), and
 * a vertex with only its self-loop solves r = (1 - alpha)/n_new + alpha r,
 * r = 1/n_new.  So r'[v] = r[v] n / n_new for the kept vertices and 1/n_new for
 * the added ones. */
void or_resize_ranks(int32_t n_old, const double *r_old, int32_t n_new, double *r_new) {
  double ratio = (double)n_old / (double)n_new;
  for (int32_t v = 0; v < n_new; v++) r_new[v] = v < n_old ? r_old[v] * ratio : 1.0 / (double)n_new;
}

/* ---- read-only accessors (tests) ---- */
int32_t or_num_vertices(const or_graph *g) { return g->n; }
int64_t or_num_edges(const or_graph *g) { return g->m; }
int64_t or_num_eff_del(const or_graph *g) { return g->n_del; }
int64_t or_num_eff_ins(const or_graph *g) { return g->n_ins; }
void or_get_out_csr(const or_graph *g, int64_t *off, int32_t *adj) {
  memcpy(off, g->out_off, sizeof(int64_t) * ((size_t)g->n + 1));
  memcpy(adj, g->out_adj, sizeof(int32_t) * (size_t)g->m);
}
void or_get_in_csr(const or_graph *g, int64_t *off, int32_t *adj) {
  memcpy(off, g->in_off, sizeof(int64_t) * ((size_t)g->n + 1));
  memcpy(adj, g->in_adj, sizeof(int32_t) * (size_t)g->m);
}
void or_get_eff_delta(const or_graph *g, uint64_t *del, uint64_t *ins) {
  if (g->n_del) memcpy(del, g->del, sizeof(uint64_t) * (size_t)g->n_del);
  if (g->n_ins) memcpy(ins, g->ins, sizeof(uint64_t) * (size_t)g->n_ins);
}

/* ---- affected sets ---- */

/* Initial marking of DF / DF-P (Alg. 1, initial marking loop): for every
 * (u, v) in Delta- u Delta+, mark every v' in (G_{t-1} u G_t).out(u). */
void or_initial_affected(const or_graph *g, uint8_t *flag) {
  memset(flag, 0, (size_t)g->n);
  for (int side = 0; side < 2; side++) {
    const uint64_t *d = side ? g->ins : g->del;
    int64_t nd = side ? g->n_ins : g->n_del;
    for (int64_t e = 0; e < nd; e++) {
      int32_t u = key_src(d[e]);
      /* G_t.out(u) */
      for (int64_t j = g->out_off[u]; j < g->out_off[u + 1]; j++) flag[g->out_adj[j]] = 1;
      /* G_{t-1}.out(u): the key range of source u in the previous edge set */
      int64_t j = lower_bound(g->keys_prev, g->m_prev, key_of(u, 0));
      for (; j < g->m_prev && key_src(g->keys_prev[j]) == u; j++) flag[key_dst(g->keys_prev[j])] = 1;
    }
  }
}

/* Vertices reachable from the sources of the updated edges, in G_{t-1} and
 * in G_t separately, united (Dynamic Traversal, Sec. 3.3.2).  A source reaches
 * itself. */
int or_dt_affected(const or_graph *g, uint8_t *flag) {
  int32_t n = g->n;
  memset(flag, 0, (size_t)n);
  int32_t *queue = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
  uint8_t *seen = (uint8_t *)malloc((size_t)n);
  if (!queue || !seen) { free(queue); free(seen); return OR_ENOMEM; }
  for (int which = 0; which < 2; which++) {   /* 0: G_{t-1}, 1: G_t */
    memset(seen, 0, (size_t)n);
    int64_t head = 0, tail = 0;
    for (int side = 0; side < 2; side++) {
      const uint64_t *d = side ? g->ins : g->del;
      int64_t nd = side ? g->n_ins : g->n_del;
      for (int64_t e = 0; e < nd; e++) {
        int32_t u = key_src(d[e]);
        if (!seen[u]) { seen[u] = 1; queue[tail++] = u; }
      }
    }
    while (head < tail) {
      int32_t x = queue[head++];
      if (which == 1) {
        for (int64_t j = g->out_off[x]; j < g->out_off[x + 1]; j++) {
          int32_t w = g->out_adj[j];
          if (!seen[w]) { seen[w] = 1; queue[tail++] = w; }
        }
      } else {
        int64_t j = lower_bound(g->keys_prev, g->m_prev, key_of(x, 0));
        for (; j < g->m_prev && key_src(g->keys_prev[j]) == x; j++) {
          int32_t w = key_dst(g->keys_prev[j]);
          if (!seen[w]) { seen[w] = 1; queue[tail++] = w; }
        }
      }
    }
    for (int32_t v = 0; v < n; v++) flag[v] |= seen[v];
  }
  free(queue); free(seen);
  return OR_OK;
}

/* ---- rank update ---- */

/* |G_t.out(u)| */
static int64_t out_degree(const or_graph *g, int32_t u) { return g->out_off[u + 1] - g->out_off[u]; }

/* c = sum over u in G_t.in(v) of R[u] / |G_t.out(u)|, in ascending u (Eq. 1);
 * K[u] holds R[u] / |G_t.out(u)|, the quotient taken once per vertex */
static double in_sum(const or_graph *g, const double *K, int32_t v) {
  double c = 0.0;
  for (int64_t j = g->in_off[v]; j < g->in_off[v + 1]; j++) c += K[g->in_adj[j]];
  return c;
}

/* Eq. 1: r = C0 + alpha * c */
double or_rank_plain(double alpha, int32_t n, double c) {
  double C0 = (1.0 - alpha) / (double)n;
  return C0 + alpha * c;
}

/* Eq. 2 (closed-loop form used by DF-P, derived in the appendix):
 * r = 1 / (1 - alpha/d) * (C0 + alpha * (c - R[v]/d)), d = |G_t.out(v)| */
double or_rank_closed_loop(double alpha, int32_t n, double c, double Rv, int64_t d) {
  double C0 = (1.0 - alpha) / (double)n;
  double dd = (double)d;
  return 1.0 / (1.0 - alpha / dd) * (C0 + alpha * (c - Rv / dd));
}

/*
 * The measure a DF / DF-P vertex compares with tau_f (expand) and tau_p
 * (prune).  Sec. 4.3 tries three: the rank change dr, the change of the
 * contribution factor dr / d, and the relative change dr / max(r, R[v]); Alg. 1
 * and every later experiment use the relative change.
 */
enum { OR_METRIC_RELATIVE = 0, OR_METRIC_ABSOLUTE = 1, OR_METRIC_CONTRIB = 2 };
/* Order of the sweeps: synchronous (every vertex of an iteration reads the
 * ranks of the start of the iteration), or asynchronous as Alg. 1 reads with
 * one rank vector and one flag vector, visited in ascending vertex id: a rank
 * written earlier in the iteration is read by later vertices, a vertex marked
 * affected later in the id order is processed in the same iteration, and a
 * vertex marked behind the current id waits for the next one (Sec. 4.4 runs
 * the loop in parallel; ascending id is one of its schedules). */
enum { OR_ORDER_SYNC = 0, OR_ORDER_ASYNC = 1, OR_ORDER_RANGES = 2 };
/* The ranges order is another schedule of Alg. 1's one rank vector: the
 * vertex ids are cut into OR_RANGES consecutive ranges at multiples of 128
 * that hold about equal shares of the in-edges (self-loops included): range k
 * starts at the first multiple of 128, v, whose in-degree prefix (the in-edges
 * of vertices below v) times OR_RANGES reaches k times all in-edges, or at n;
 * one range when n < 128 OR_RANGES.  The ranges are swept one after another,
 * and a vertex reads the ranks of the ranges before its own as updated in this
 * sweep and all others as of the start of the sweep.  Flags take effect in
 * the next iteration, as in the synchronous order. */
enum { OR_RANGES = 8 };

/* bound[0..P]: the ranges of the ranges order on the current in-rows */
static void range_bounds(const or_graph *g, int P, int32_t *bound) {
  const int32_t n = g->n;
  const int64_t W = g->in_off[n];
  const int64_t chunks = ((int64_t)n + 127) / 128;
  bound[0] = 0;
  for (int k = 1; k < P; k++) {
    int64_t j = 0;
    while (j < chunks && g->in_off[128 * j] * P < (int64_t)k * W) j++;
    bound[k] = (int32_t)(128 * j < n ? 128 * j : n);
  }
  bound[P] = n;
}

static double frontier_measure(int metric, double dr, double r, double Rv, int64_t d) {
  if (metric == OR_METRIC_ABSOLUTE) return dr;
  if (metric == OR_METRIC_CONTRIB) return dr / (double)d;
  return dr / fmax(r, Rv);
}

/* relative distance of x from the threshold t (see tie_rel) */
static double tie_to(double x, double t) {
  if (!(t > 0.0) || !isfinite(t)) return INFINITY;
  return fabs(x / t - 1.0);
}

/* What one sweep over the processed vertices gathers for the statistics. */
typedef struct {
  double dR, tie;
  int64_t vertices, edges;
} sweep_sum;

/* The fixed arguments of one method run. */
typedef struct {
  double alpha, tau_f, tau_p;
  int metric, frontier, prune, async;
} run_args;

/*
 * Process vertex v in one iteration of Alg. 1 (Eq. 1, or Eq. 2 for DF-P),
 * reading the ranks R and their quotients K.  Writes the new rank to Rw[v] and
 * the flags of the next frontier to Fw.  Synchronous order: R, K are the
 * ranks of the start of the iteration and Fw is F_{i+1} (v stays unless
 * pruned; expansion marks G_t.out(v)).  Asynchronous order: Rw == R,
 * Fw is the one flag vector (pruning clears v, expansion sets G_t.out(v)),
 * and K[v] follows the new rank at once.
 */
static void visit(const or_graph *g, const run_args *a, int32_t v, const double *R, double *K, double *Rw,
                  uint8_t *Fw, uint8_t *ever, sweep_sum *acc) {
  int32_t n = g->n;
  ever[v] = 1;                                              /* processed in some sweep */
  double c = in_sum(g, K, v);
  int64_t d = out_degree(g, v);
  double Rv = R[v];
  double r = a->prune ? or_rank_closed_loop(a->alpha, n, c, Rv, d) : or_rank_plain(a->alpha, n, c);
  double dr = fabs(r - Rv);
  if (dr > acc->dR) acc->dR = dr;
  acc->vertices++;
  acc->edges += g->in_off[v + 1] - g->in_off[v];
  if (a->frontier) {
    double mv = frontier_measure(a->metric, dr, r, Rv, d);
    acc->tie = fmin(acc->tie, tie_to(mv, a->tau_f));
    if (a->prune) acc->tie = fmin(acc->tie, tie_to(mv, a->tau_p));
    if (a->async) {
      if (a->prune && mv <= a->tau_p) Fw[v] = 0;            /* mark v as not affected */
    } else if (!(a->prune && mv <= a->tau_p)) {
#pragma omp atomic write
      Fw[v] = 1;                                            /* v stays unless pruned */
    }
    if (mv > a->tau_f)                                      /* expand: mark G_t.out(v) */
      for (int64_t j = g->out_off[v]; j < g->out_off[v + 1]; j++) {
#pragma omp atomic write
        Fw[g->out_adj[j]] = 1;
      }
  }
  Rw[v] = r;
  if (a->async) K[v] = r / (double)d;
}

/*
 * One method run (Sec. 3.1, Sec. 3.3, Alg. 1).
 * r_prev: ranks of the previous snapshot (ignored by Static, required by the
 * others).  r_out: the updated ranks.  metric: the DF / DF-P measure above.
 * order: OR_ORDER_SYNC or OR_ORDER_ASYNC.  Returns OR_ENORANKS when a dynamic
 * method has no r_prev.
 */
int or_update_ex(const or_graph *g, int method, double alpha, double tau, double tau_f, double tau_p,
                 int32_t max_iter, int metric, int order, const double *r_prev, double *r_out, or_stats *st) {
  int32_t n = g->n;
  if (method < OR_STATIC || method > OR_DFP || max_iter < 0 || !(alpha >= 0.0 && alpha < 1.0)) return OR_EINVAL;
  if (metric < OR_METRIC_RELATIVE || metric > OR_METRIC_CONTRIB || order < OR_ORDER_SYNC || order > OR_ORDER_RANGES)
    return OR_EINVAL;
  if (method != OR_STATIC && !r_prev) return OR_ENORANKS;
  double *R = (double *)malloc(sizeof(double) * (size_t)n);
  double *Rn = (double *)malloc(sizeof(double) * (size_t)n);
  double *K = (double *)malloc(sizeof(double) * (size_t)n);  /* R[u] / |G_t.out(u)| */
  uint8_t *F = (uint8_t *)calloc((size_t)n, 1);      /* vertices processed in this iteration */
  uint8_t *Fn = (uint8_t *)calloc((size_t)n, 1);     /* F_{i+1} */
  uint8_t *ever = (uint8_t *)calloc((size_t)n, 1);
  if (!R || !Rn || !K || !F || !Fn || !ever) {
    free(R); free(Rn); free(K); free(F); free(Fn); free(ever);
    return OR_ENOMEM;
  }

  if (method == OR_STATIC) for (int32_t v = 0; v < n; v++) R[v] = 1.0 / (double)n;
  else memcpy(R, r_prev, sizeof(double) * (size_t)n);

  if (method == OR_STATIC || method == OR_NAIVE_DYNAMIC) memset(F, 1, (size_t)n);
  else if (method == OR_DYNAMIC_TRAVERSAL) {
    if (or_dt_affected(g, F) != OR_OK) {
      free(R); free(Rn); free(K); free(F); free(Fn); free(ever);
      return OR_ENOMEM;
    }
  } else or_initial_affected(g, F);

  run_args a = {alpha, tau_f, tau_p, metric, method == OR_DF || method == OR_DFP, method == OR_DFP,
                order == OR_ORDER_ASYNC};
  /* range bounds: one range for the synchronous order */
  int P = order == OR_ORDER_RANGES && n >= 128 * OR_RANGES ? OR_RANGES : 1;
  int32_t bound[OR_RANGES + 1];
  range_bounds(g, P, bound);
  or_stats s;
  memset(&s, 0, sizeof(s));
  s.tie_rel = INFINITY;
  for (int32_t i = 0; i < max_iter; i++) {
#pragma omp parallel for schedule(static)
    for (int32_t u = 0; u < n; u++) K[u] = R[u] / (double)out_degree(g, u);
    sweep_sum tot = {0.0, INFINITY, 0, 0};
    if (a.async) {
      /* one rank vector and one flag vector, ascending vertex id */
      for (int32_t v = 0; v < n; v++)
        if (F[v]) visit(g, &a, v, R, K, R, F, ever, &tot);
    } else {
      /* new ranks and flags go to Rn / Fn and are committed after the sweep;
       * in the ranges order the quotients of a range follow its new ranks
       * before the next range is swept */
      memcpy(Rn, R, sizeof(double) * (size_t)n);
      if (a.frontier) memset(Fn, 0, (size_t)n);
      for (int k = 0; k < P; k++) {
#pragma omp parallel
        {
          sweep_sum part = {0.0, INFINITY, 0, 0};
#pragma omp for schedule(dynamic, 1024)
          for (int32_t v = bound[k]; v < bound[k + 1]; v++)
            if (F[v]) visit(g, &a, v, R, K, Rn, Fn, ever, &part);
#pragma omp critical
          {
            if (part.dR > tot.dR) tot.dR = part.dR;
            tot.tie = fmin(tot.tie, part.tie);
            tot.vertices += part.vertices;
            tot.edges += part.edges;
          }
        }
        if (P > 1) {
#pragma omp parallel for schedule(static)
          for (int32_t v = bound[k]; v < bound[k + 1]; v++)
            if (F[v]) K[v] = Rn[v] / (double)out_degree(g, v);
        }
      }
      memcpy(R, Rn, sizeof(double) * (size_t)n);
      if (a.frontier) memcpy(F, Fn, (size_t)n);
    }
    s.vertices_processed += tot.vertices;
    s.edges_processed += tot.edges;
    s.tie_rel = fmin(s.tie_rel, tot.tie);
    s.iterations = i + 1;
    s.delta_R = tot.dR;
    s.tie_rel = fmin(s.tie_rel, tie_to(tot.dR, tau));
    if (tot.dR <= tau) { s.converged = 1; break; }
  }
  for (int32_t v = 0; v < n; v++) s.vertices_ever_affected += ever[v];
  memcpy(r_out, R, sizeof(double) * (size_t)n);
  if (st) *st = s;
  free(R); free(Rn); free(K); free(F); free(Fn); free(ever);
  return OR_OK;
}

/* The synchronous run with the relative measure of Alg. 1. */
int or_update(const or_graph *g, int method, double alpha, double tau, double tau_f, double tau_p,
              int32_t max_iter, const double *r_prev, double *r_out, or_stats *st) {
  return or_update_ex(g, method, alpha, tau, tau_f, tau_p, max_iter, OR_METRIC_RELATIVE, OR_ORDER_SYNC, r_prev,
                      r_out, st);
}
