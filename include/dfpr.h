/*
 * dfpr.h -- C ABI of the GB300 library for the Dynamic Frontier (DF) and
 * Dynamic Frontier with Pruning (DF-P) PageRank update of arXiv 2401.15870
 * ("DF* PageRank: Improved Incrementally Expanding Approaches for Updating
 * PageRank on Dynamic Graphs"), with Static, Naive-dynamic and Dynamic
 * Traversal PageRank as comparators.
 *
 * Conventions for every call:
 *   - Vertex ids are int32 in [0, n); n is fixed when the graph is created
 *     (Sec. 5.2.2: batches add or remove no vertices).
 *   - "host" pointers are ordinary CPU memory; "device" pointers are CUDA
 *     global memory on the graph's device (for example torch CUDA tensors).
 *     Input arrays stay owned by the caller and are only read during the call.
 *     Output arrays are owned by the caller and must hold the stated number of
 *     elements.
 *   - The graph owns all of its device memory and enqueues all work on the
 *     CUDA stream given at creation (pr_set_stream changes it).  Calls return
 *     after their results are available to the caller (host outputs written,
 *     device outputs complete on the graph's stream).
 *   - Inputs are validated before anything is changed: a call that returns an
 *     error leaves the graph as it was, except PR_ECUDA / PR_ENOMEM raised by
 *     the device in the middle of an edit, after which the graph must be
 *     destroyed.  No C++ exception crosses this interface.
 *   - Ranks are FP64.  Contribution sums inside the rank sweep are exact sums
 *     of 2^-61 fixed-point terms (every term R[u]/|out(u)| rounded to the
 *     nearest multiple of 2^-61), so results do not depend on the order of
 *     additions; the caller's ranks must be finite, non-negative and sum to at
 *     most 2.
 *   - One caller at a time per graph (Sec. 3.2: one writer on the graph at
 *     any given time).  Different graphs may be used from different threads.
 */
#ifndef DFPR_H
#define DFPR_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct pr_graph pr_graph;

/* Update methods (Sec. 3.1, Sec. 3.3, Sec. 4.1). */
typedef enum {
  PR_STATIC = 0,            /* power iteration from 1/|V| over all vertices (Sec. 3.1)          */
  PR_NAIVE_DYNAMIC = 1,     /* all vertices, starting from the current ranks (Sec. 3.3.1)        */
  PR_DYNAMIC_TRAVERSAL = 2, /* vertices reachable from updated sources in G_{t-1} or G_t (2.3.2) */
  PR_DF = 3,                /* Dynamic Frontier (Sec. 4.1.1, Alg. 1)                            */
  PR_DFP = 4                /* Dynamic Frontier with Pruning (Sec. 4.1.2, Alg. 1, Eq. 2)         */
} pr_method;

typedef enum {
  PR_OK = 0,
  PR_EINVAL = 1,    /* bad argument (null pointer, negative size, method, alpha, tolerances) */
  PR_ERANGE = 2,    /* a vertex id outside [0, n)                                            */
  PR_ENOMEM = 3,    /* device or host allocation failed                                      */
  PR_ENORANKS = 4,  /* a dynamic method was asked for before any ranks exist                 */
  PR_ECUDA = 5,     /* a CUDA call failed; pr_last_error has the text                        */
  PR_ETIMEOUT = 6   /* a bounded device-side wait gave up                                    */
} pr_status;

/* Tolerances of Alg. 1; NULL options mean tau_f = tau_p = 1e-6 and 500
 * iterations (Sec. 5.1.2, Sec. 4.2, Sec. 4.3). */
typedef struct {
  double tau_f;       /* frontier tolerance: expand when dr / max(r, R[v]) > tau_f  */
  double tau_p;       /* prune tolerance (DF-P): drop v when dr / max(r, R[v]) <= tau_p */
  int32_t max_iter;   /* MAX_ITERATIONS                                              */
  int32_t flags;      /* PR_OPT_* bits; other bits must be 0                          */
} pr_options;

/* pr_options.flags: time every rank-sweep kernel with CUDA events on the
 * graph's stream and report the sum in pr_stats.ms_sweep. */
#define PR_OPT_TIME_SWEEPS 1
/* pr_options.flags for DF / DF-P and DT: sweep the frontier only in pull form
 * (every vertex with a membership test) or only in push form (frontier lists
 * with explicit expansion; DT: its affected set as a list).  By default the
 * form is chosen per iteration (DT: once) from the frontier's size; the result
 * is the same in every form. */
#define PR_OPT_FORCE_PULL 2
#define PR_OPT_FORCE_PUSH 4
/* pr_options.flags for Static, ND, DF and DF-P: where the iteration loop runs.
 * The host loop reads the iteration's change back after every sweep and picks
 * the sweep form; the device loop runs the iterations as a CUDA graph whose
 * WHILE node is driven by a control kernel (the pull form only, no host round
 * trip).  By default graphs below PR_DEVICE_LOOP_SLOTS in-CSR slots use the
 * device loop unless another flag asks for the host loop (any of the flags
 * above); the smallest run it in one kernel (PR_OPT_ONE_KERNEL below).  The
 * result is the same either way. */
#define PR_OPT_DEVICE_LOOP 8
#define PR_OPT_HOST_LOOP 16
/* pr_options.flags for DF / DF-P: the measure a processed vertex compares
 * with tau_f (expand its out-neighbours when above) and tau_p (DF-P: prune it
 * when at or below).  Sec. 4.3 tries three: the relative rank change
 * dr / max(r, R[v]) (the default; Alg. 1 and every later experiment), the rank
 * change dr (PR_OPT_MEASURE_ABSOLUTE) and the change of the contribution
 * factor dr / |out(v)| (PR_OPT_MEASURE_CONTRIB).  At most one of the two may
 * be set; they work with either iteration loop and with groups.  The
 * comparisons are made without a division: dr > tau * max(r, R[v]), dr > tau,
 * dr > tau * |out(v)|. */
#define PR_OPT_MEASURE_ABSOLUTE 32
#define PR_OPT_MEASURE_CONTRIB 64
/* pr_options.flags for Static, ND, DF and DF-P: an asynchronous order of
 * Alg. 1 (Sec. 4.4 runs it with one rank vector updated in place).  The
 * library's vertex order is cut into 8 consecutive ranges at multiples of 128
 * that hold about equal shares of the in-edges (range k starts at the first
 * multiple of 128, v, where 8 times the in-edges of the vertices below v,
 * self-loops included, reaches k times all in-edges, or at n; one range below
 * 1024 vertices), every sweep visits the ranges one after another, and a vertex
 * reads the ranks of the ranges before its own as updated in this sweep and
 * the others as of the start of the sweep.  Frontier flags take effect in the
 * next iteration, as in the synchronous order.  The schedule is fixed, so the
 * result is reproducible; it converges to the same fixed point of Eq. 1,
 * usually in fewer iterations.  The library's vertex order is the caller's
 * when the graph was created keeping it (pr_graph_create_edges flags bit 0),
 * else the internal order by out-degree.  Runs on the host loop; not with
 * PR_OPT_DEVICE_LOOP, PR_OPT_FORCE_PUSH, Dynamic Traversal or groups
 * (PR_EINVAL). */
#define PR_OPT_ASYNC 128
#define PR_DEVICE_LOOP_SLOTS (1ll << 24)
/* pr_options.flags for Static, ND, DF and DF-P, and for groups: the device
 * loop in one cooperative kernel.  Initialisation, marking and every
 * iteration's gather, epilogue and control run as phases of one launch whose
 * blocks are all resident, separated by grid barriers, instead of three kernel
 * launches per iteration in a CUDA graph: on graphs whose sweeps take
 * microseconds the launches cost more than the work.  Without this flag,
 * PR_OPT_DEVICE_LOOP or a host-loop flag, the device loop runs in one kernel
 * when the graphs of the update hold fewer than PR_ONE_KERNEL_SLOTS in-CSR
 * slots in all; PR_OPT_DEVICE_LOOP alone asks for the CUDA graph.  At most one
 * of PR_OPT_HOST_LOOP, PR_OPT_DEVICE_LOOP and PR_OPT_ONE_KERNEL may be set.
 * The result is the same bit for bit.  A barrier wait gives up after about a
 * second (a block that never arrives); the update then returns PR_ETIMEOUT
 * and its graphs are left without ranks. */
#define PR_OPT_ONE_KERNEL 256
#define PR_ONE_KERNEL_SLOTS (1ll << 20)

/* Outcome of one pr_update (Sec. 5.1.5 measures time and affected vertices). */
typedef struct {
  int32_t iterations;              /* sweeps run                                            */
  int32_t converged;               /* 1 if the last L-inf change was <= tau                 */
  double delta_R;                  /* L-inf change of the last sweep                        */
  int64_t vertices_ever_affected;  /* vertices processed by at least one sweep (Sec. 5.2.3) */
  int64_t edges_processed;         /* in-edges summed over all sweeps                       */
  int64_t vertices_processed;      /* vertex updates over all sweeps                        */
  int64_t eff_deletions;           /* |Delta-| of the last batch                            */
  int64_t eff_insertions;          /* |Delta+| of the last batch                            */
  double ms_apply;                 /* device time of the last pr_apply_batch*               */
  double ms_update;                /* device time of this pr_update                         */
  double ms_sweep;                 /* rank-sweep kernel time (PR_OPT_TIME_SWEEPS), else 0   */
  int32_t sweeps;                  /* rank-sweep kernel launches                            */
  int32_t reserved;
} pr_stats;

/*
 * Create a graph from an out-edge CSR in host memory (Sec. 3.1 notation:
 * G.out(u) = col[row_off[u] .. row_off[u+1])).  row_off has n+1 entries with
 * row_off[0] = 0 and row_off[n] = m; col has m entries in [0, n).  Repeated
 * edges are collapsed and every vertex gets exactly one self-loop (Sec. 5.1.3:
 * self-loops on all vertices remove dead ends).  stream is a cudaStream_t
 * (NULL = the default stream) on the current device.  On success *out owns a
 * new graph without ranks.  Errors: PR_EINVAL (n < 1, m < 0, null pointers,
 * row_off not non-decreasing from 0 to m), PR_ERANGE (a column outside
 * [0, n)), PR_ENOMEM, PR_ECUDA.
 */
pr_status pr_graph_create(int32_t n, int64_t m, const int64_t* row_off, const int32_t* col, void* stream,
                          pr_graph** out);

/*
 * Create a graph from an edge list src[i] -> dst[i], i < m, in host memory
 * (device_ptrs = 0) or device memory (device_ptrs = 1).  Same semantics and
 * errors as pr_graph_create.  flags: bit 0 set keeps the caller's vertex order
 * inside the library (by default vertices are renumbered internally by
 * decreasing out-degree for locality; ranks and batches always use the
 * caller's ids).
 */
pr_status pr_graph_create_edges(int32_t n, int64_t m, const int32_t* src, const int32_t* dst, int32_t device_ptrs,
                                int32_t flags, void* stream, pr_graph** out);

/* Free the graph and all its device memory (NULL is ignored). */
void pr_graph_destroy(pr_graph* g);

/* Rebind the graph to another CUDA stream of the same device. */
pr_status pr_set_stream(pr_graph* g, void* stream);

/*
 * Vertex insertion and deletion: change |V| to n_new.  The paper keeps |V|
 * fixed in its experiments (Sec. 5.2.2) while its temporal graphs gain
 * vertices over time (Sec. 5.1.4); this call adds or removes vertices at the
 * end of the id range.
 *   n_new > n: vertices n .. n_new-1 are added with their self-loop only
 *     (Sec. 5.1.3), and no other edge.
 *   n_new < n: vertices n_new .. n-1 are removed; each must have no edge but
 *     its self-loop (delete its edges with pr_apply_batch first), else
 *     PR_EINVAL and nothing changes.
 * Ranks (if the graph has them) are carried over by a closed form.  With
 * C0 = (1 - alpha)/|V| in Eq. 1, scaling a solution of Eq. 1 on the old graph
 * by n / n_new solves Eq. 1 on the new graph (the sums over in-neighbours
 * scale with it), and a vertex whose only edge is its self-loop solves
 * r = (1 - alpha)/n_new + alpha r, i.e. r = 1/n_new.  So r'[v] = r[v] n/n_new
 * for the vertices kept and 1/n_new for the new ones: a converged graph stays
 * converged, to the rounding of that product.  The last batch's effective
 * change is cleared, so a DF / DF-P update right after the call processes
 * nothing; edges of the new vertices come in later batches.  The tuning
 * settings are kept; the handle stays valid (its device memory is rebuilt:
 * the call costs a graph creation).  Errors: PR_EINVAL (n_new < 1, n_new + m
 * >= 2^31, a removed vertex with edges), PR_ENOMEM, PR_ECUDA; on error the
 * graph is unchanged.
 */
pr_status pr_graph_resize(pr_graph* g, int32_t n_new);

/*
 * Apply one batch update (Sec. 3.2): E_t = (E_{t-1} \ D) u I, deletions
 * first.  D = {(del_src[i], del_dst[i])}, I = {(ins_src[i], ins_dst[i])}, all
 * in host memory.  Repeats, deletions of absent edges, insertions of present
 * edges and self-loop deletions have no effect (self-loops are re-added with
 * every batch, Sec. 5.2.2).  The CSR and its transpose are edited in place on
 * the device, and the effective change Delta- = E_{t-1} \ E_t, Delta+ =
 * E_t \ E_{t-1} is kept for the next pr_update.  Contributions of sources
 * whose out-degree changed are refreshed.  Errors: PR_EINVAL (null pointer
 * with a positive count, negative count), PR_ERANGE (an id outside [0, n);
 * nothing is changed), PR_ENOMEM, PR_ECUDA.
 */
pr_status pr_apply_batch(pr_graph* g, const int32_t* del_src, const int32_t* del_dst, int64_t n_del,
                         const int32_t* ins_src, const int32_t* ins_dst, int64_t n_ins);

/* As pr_apply_batch with the four endpoint arrays in device memory. */
pr_status pr_apply_batch_device(pr_graph* g, const int32_t* del_src, const int32_t* del_dst, int64_t n_del,
                                const int32_t* ins_src, const int32_t* ins_dst, int64_t n_ins);

/*
 * The batches of many graphs at once (one per graph, device arrays as in
 * pr_apply_batch_device; graphs[i] gets del_src[i] .. n_ins[i]).  Each batch
 * has the effect of pr_apply_batch_device on its graph; the difference is
 * scheduling: every graph's work is queued before the host waits for any, so
 * the host round trips of many small batches overlap, and the batches run side
 * by side on a pool of library streams (each first waits for its graph's
 * stream, and the graph's stream waits for its end, so work queued on the
 * graph's stream before and after the call stays ordered with it; graphs of
 * another device than the current one run on their own stream).  A group
 * update of the same graphs usually follows (pr_group_update).  The graphs
 * must be distinct.  The call returns when every batch is applied.
 * Returns the first error; a graph whose batch failed is left as
 * pr_apply_batch_device leaves it on that error, the others are applied.
 * Errors: PR_EINVAL, PR_ERANGE, PR_ENOMEM, PR_ECUDA.
 */
pr_status pr_apply_batches_device(int32_t count, pr_graph* const* graphs, const int32_t* const* del_src,
                                  const int32_t* const* del_dst, const int64_t* n_del, const int32_t* const* ins_src,
                                  const int32_t* const* ins_dst, const int64_t* n_ins);

/* As pr_apply_batches_device with every endpoint array in host memory (ids
 * are checked on the host before anything of that graph is queued; each
 * batch is staged into its graph's device scratch on the pool's stream). */
pr_status pr_apply_batches(int32_t count, pr_graph* const* graphs, const int32_t* const* del_src,
                           const int32_t* const* del_dst, const int64_t* n_del, const int32_t* const* ins_src,
                           const int32_t* const* ins_dst, const int64_t* n_ins);

/*
 * Update the ranks with one method (Sec. 3.1, 2.3, Alg. 1) after the last
 * batch, iterating until the L-inf change of a sweep is <= tau or
 * opts->max_iter sweeps have run.  alpha in [0, 1) is the damping factor
 * (0.85 in the paper), tau >= 0 the iteration tolerance (1e-10, L-inf).
 * Every method runs in the synchronous order: all vertices processed in a
 * sweep read the ranks of the start of the sweep.  PR_STATIC starts from
 * 1/|V|; the others from the current ranks (pr_set_ranks or a previous
 * update; PR_ENORANKS if none).  Not converging is not an error
 * (stats->converged = 0).  opts and stats may be NULL.  Errors: PR_EINVAL,
 * PR_ENORANKS, PR_ECUDA, PR_ETIMEOUT (the one-kernel loop's grid barrier gave
 * up, PR_OPT_ONE_KERNEL; the graph is left without ranks).
 */
pr_status pr_update(pr_graph* g, pr_method method, double alpha, double tau, const pr_options* opts,
                    pr_stats* stats);

/* Copy the n ranks (caller's vertex ids) to host memory out[0..n). */
pr_status pr_ranks(const pr_graph* g, double* out);
/* Copy the n ranks to device memory out[0..n) (complete on the graph's stream). */
pr_status pr_ranks_device(const pr_graph* g, double* out);

/*
 * Set the current ranks R_{t-1} from host memory r[0..n) (caller's ids), for
 * example to run several methods from the same previous ranks.  Errors:
 * PR_EINVAL (a rank that is negative or not finite, or a sum above 2).
 */
pr_status pr_set_ranks(pr_graph* g, const double* r);
/* As pr_set_ranks with r in device memory (checked on the device). */
pr_status pr_set_ranks_device(pr_graph* g, const double* r);

/* n and the current edge count m (self-loops included). */
pr_status pr_graph_info(const pr_graph* g, int32_t* n, int64_t* m);

/*
 * Export one direction of the current graph to host memory in the caller's
 * ids: which = 0 for out-edges, 1 for in-edges.  off[0..n] gets row offsets,
 * adj[0..m) the neighbours of each row in ascending order.
 */
pr_status pr_get_csr(const pr_graph* g, int32_t which, int64_t* off, int32_t* adj);

/*
 * Rows of selected vertices (host memory, caller's ids): which = 0 for
 * out-neighbours, 1 for in-neighbours.  off[0..count] receives the row offsets
 * (off[k+1] - off[k] is the degree of vertices[k]); if adj is not NULL it
 * receives the rows, each sorted ascending (size it from a first call with
 * adj = NULL).  Errors: PR_EINVAL, PR_ERANGE (a vertex outside [0, n)).
 */
pr_status pr_get_rows(const pr_graph* g, int32_t which, int64_t count, const int32_t* vertices, int64_t* off,
                      int32_t* adj);

/* Effective change of the last batch: sizes, then the edges (caller's ids,
 * each array sorted by (src, dst)).  Any output pointer may be NULL. */
pr_status pr_last_delta(const pr_graph* g, int64_t* n_del, int64_t* n_ins, int32_t* del_src, int32_t* del_dst,
                        int32_t* ins_src, int32_t* ins_dst);

/*
 * Affected sets on the device, written as one byte per vertex (caller's ids)
 * to host memory flags[0..n):
 *   which = 0: initial marking of DF / DF-P (Alg. 1): every v' in
 *              (G_{t-1} u G_t).out(u) for (u, v) in Delta- u Delta+;
 *   which = 1: Dynamic Traversal (Sec. 3.3.2): vertices reachable from those
 *              u in G_{t-1}, united with those reachable in G_t.
 */
pr_status pr_affected(pr_graph* g, int32_t which, uint8_t* flags);

/*
 * One synchronous sweep of Eq. 1 over a caller-provided in-CSR, allocating no
 * memory.  The paper has no counterpart: this entry point exists for callers
 * that cannot allocate device memory (code running where cudaMalloc is not
 * allowed or would stall other work, e.g. a serving loop whose device memory
 * is owned by another allocator).  Every pointer is device memory owned by the
 * caller:
 *   in_off[0..n], in_src[0..in_off[n]): in-neighbours u of every vertex v
 *     (self-loops included, as pr_get_csr(g, 1, ...) exports them);
 *   out_deg[0..n): |out(u)| >= 1;  r_in[0..n): current ranks;
 *   r_out[0..n): receives (1-alpha)/n + alpha * sum_u r_in[u]/out_deg[u],
 *     summed exactly in 2^-61 fixed point like pr_update's sweeps;
 *   *delta_out: receives max_v |r_out[v] - r_in[v]|.
 * Work is enqueued on `stream`; the call returns before it completes.  Its
 * scratch memory is a fixed array of PR_NOALLOC_MAX_N + 2 int64 values
 * (about 4 MB) inside the library, whatever n is, present on every GPU that
 * loads it until the process exits; n above PR_NOALLOC_MAX_N is rejected with
 * PR_EINVAL before any device work.  r_out must not overlap r_in (the change
 * of every vertex is measured against r_in): overlapping buffers are rejected
 * with PR_EINVAL.  The
 * first call on a device looks up that array's address (cudaGetSymbolAddress):
 * make it before any stream capture.  All calls share the array, so calls
 * that overlap on the GPU race and must be serialized.  Errors: PR_EINVAL
 * (size, null pointer, r_out overlapping r_in, alpha), PR_ECUDA.
 */
#define PR_NOALLOC_MAX_N 524288
pr_status pr_sweep_noalloc(int32_t n, const int64_t* in_off, const int32_t* in_src, const int32_t* out_deg,
                           const double* r_in, double* r_out, double alpha, double* delta_out, void* stream);

/*
 * Groups: one update of many graphs at once.  The paper updates one graph at
 * a time; a group serves callers that hold many independent graphs (for
 * example one per tenant or per time window) and would otherwise run one
 * launch sequence per graph.  Every iteration sweeps all graphs of the group
 * that have not converged in one launch pair (gather, then the epilogue of
 * Alg. 1 / Eq. 1-2), and the loop over iterations runs on the device (a CUDA
 * graph with a WHILE node), so each graph stops on its own criterion with no
 * host round trip.  A graph's ranks and statistics are bit-identical to those
 * of pr_update on the graph alone.
 *
 * pr_group_create: count in [1, PR_GROUP_MAX] distinct graphs (host array of
 *   handles, read during the call), all on the current device.  The group
 *   refers to the graphs and owns none of them: destroy the group before any
 *   of its graphs.  stream: the CUDA stream of the group's work (NULL: the
 *   legacy default stream).  Errors: PR_EINVAL, PR_ENOMEM, PR_ECUDA.
 * pr_group_update: method PR_STATIC, PR_NAIVE_DYNAMIC, PR_DF or PR_DFP (Dynamic
 *   Traversal is not offered), alpha / tau / opts as in pr_update; the flags
 *   accepted are PR_OPT_MEASURE_* and at most one of PR_OPT_HOST_LOOP (the
 *   same kernels launched one by one with the loop condition read back after
 *   every iteration, for profilers that cannot look into a CUDA graph with
 *   conditional nodes and for drivers without them), PR_OPT_DEVICE_LOOP (the
 *   CUDA graph) and PR_OPT_ONE_KERNEL (one cooperative kernel); with none of
 *   the three the group runs in one kernel below PR_ONE_KERNEL_SLOTS in-CSR
 *   slots over its graphs and as the CUDA graph above.  The update runs after
 *   the work already queued on every graph's stream and is complete on
 *   return.  stats: NULL or count entries, one per graph in creation order;
 *   ms_update is the time of the whole group, ms_sweep is 0.  Errors:
 *   PR_EINVAL, PR_ENORANKS (a dynamic method on a graph without ranks;
 *   nothing is changed), PR_ECUDA, PR_ETIMEOUT (a grid barrier of the
 *   one-kernel loop gave up; the graphs are left without ranks).
 */
#define PR_GROUP_MAX 1024
typedef struct pr_group pr_group;
pr_status pr_group_create(int32_t count, pr_graph* const* graphs, void* stream, pr_group** out);
pr_status pr_group_update(pr_group* grp, pr_method method, double alpha, double tau, const pr_options* opts,
                          pr_stats* stats);
/* The same for the graphs at the given group positions only (count distinct
 * indices in [0, group size)); the others are left as they are.  stats: NULL
 * or one entry per graph of the group, by position; only the members' entries
 * are written. */
pr_status pr_group_update_members(pr_group* grp, pr_method method, double alpha, double tau,
                                  const pr_options* opts, const int32_t* members, int32_t count, pr_stats* stats);
void pr_group_destroy(pr_group* grp);

/*
 * Unit sizes of the group kernels: a gather unit is steps_per_unit warp steps,
 * each over 32 x quads_per_lane in-CSR quads ((quads, steps) one of (2, 1),
 * (4, 1), (8, 1), (2, 4)), an epilogue unit is chunks_per_unit 32-vertex chunks
 * (1, 2 or 4) whose loads a warp issues together.  Smaller units spread small
 * graphs over more warps; larger ones keep more loads in flight per warp or
 * look the graph up less often.  Defaults 4 / 1 / 4.  The setting changes no
 * result (the sums are exact).  It applies to the CUDA-graph and host loops;
 * the one-kernel loop (PR_OPT_ONE_KERNEL) uses units of one warp step of
 * 32 x 2 quads and one chunk.
 * pr_group_autotune: runs reps (0: 1) group updates of the method per
 *   candidate (12 settings; the CUDA-graph device loop, CUDA-event time of the whole update), every
 *   graph starting from its ranks on entry (with its last batch for DF / DF-P),
 *   keeps the fastest, and puts the ranks on entry back at the end (a graph
 *   without ranks keeps those of the last Static trial).  Dynamic methods need
 *   ranks on every graph (PR_ENORANKS).  Errors: PR_EINVAL (Dynamic
 *   Traversal, bad alpha / tau / reps, an update in flight), PR_ENORANKS,
 *   PR_ENOMEM, PR_ECUDA.
 * pr_group_set_tuning: quads_per_lane, steps_per_unit and chunks_per_unit (the
 *   other fields are ignored); other values give PR_EINVAL and no change.
 */
typedef struct {
  int32_t quads_per_lane;
  int32_t steps_per_unit;
  int32_t chunks_per_unit;
  float ms_update;          /* pr_group_autotune: the chosen setting's update time, ms */
  int32_t candidates;       /* pr_group_autotune: settings timed                      */
} pr_group_tuning;
pr_status pr_group_autotune(pr_group* grp, pr_method method, double alpha, double tau, int32_t reps,
                            pr_group_tuning* out);
pr_status pr_group_get_tuning(const pr_group* grp, pr_group_tuning* out);
pr_status pr_group_set_tuning(pr_group* grp, const pr_group_tuning* in);

/*
 * Serving: a request loop over resident graphs.  The paper updates one graph
 * per batch; a server accepts update batches for many graphs as they arrive
 * (from any thread) and turns them into DF / DF-P updates on one worker
 * thread.
 *   PR_SERVE_GROUPED: continuous batching.  Requests of a graph that queue up
 *     are merged in arrival order into one batch (per edge the last operation
 *     wins, deletions of a request before its insertions; the resulting edge
 *     set is the one the requests give one after another, Sec. 3.2).  Batches
 *     are applied while the updates of other graphs run.  A small graph
 *     (below PR_DEVICE_LOOP_SLOTS in-CSR slots) with an applied batch joins
 *     the next group update (one launch pair per iteration for all of them,
 *     the loop on the device); a large graph is updated with pr_update by a
 *     second server thread, large graphs one after another (pr_update picks
 *     the push or pull form per iteration), while group updates and batch
 *     edits of other graphs go on.  A round admits
 *     graphs while their estimated batch scratch leaves hbm_reserve bytes of
 *     device memory free and the round's edges stay within max_round_edges
 *     (0: no cap); the first graph of a round is always admitted.
 *   PR_SERVE_PLAIN: one pr_apply_batch + pr_update per request, in arrival
 *     order (the baseline).
 * While the server runs, each graph's work is on a stream of the server's
 * (pr_set_stream; the previous streams are restored by pr_server_destroy) and
 * the caller must not use the graphs.  Every graph needs ranks.
 */
#define PR_SERVE_GROUPED 0
#define PR_SERVE_PLAIN 1
typedef struct {
  int32_t mode;              /* PR_SERVE_GROUPED or PR_SERVE_PLAIN            */
  int32_t method;            /* PR_DF or PR_DFP                               */
  double alpha, tau;         /* as in pr_update                               */
  pr_options opts;           /* tolerances and max_iter; flags must be 0      */
  int64_t hbm_reserve;       /* device bytes a round leaves free (grouped)    */
  int64_t max_round_edges;   /* batch edges admitted per round, 0: no cap     */
} pr_server_options;

/* Outcome of one request. */
typedef struct {
  int64_t ticket;
  int32_t graph;
  int32_t status;            /* pr_status of the apply / update that served it */
  int64_t round;             /* update round; requests of one graph in one round were merged */
  int32_t merged;            /* requests merged into that round's batch of this graph */
  int32_t pad;
  double t_submit;           /* pr_server_clock() seconds: submitted          */
  double t_start;            /* its batch started to be applied               */
  double t_done;             /* its graph's update finished (ranks ready)     */
  pr_stats stats;            /* that update of its graph                      */
} pr_request_info;

typedef struct pr_server pr_server;
/* count graphs (host array of handles; the server refers to them, destroy it
 * first).  Errors: PR_EINVAL, PR_ENORANKS, PR_ENOMEM, PR_ECUDA. */
pr_status pr_server_create(int32_t count, pr_graph* const* graphs, const pr_server_options* opts, pr_server** out);
/* Queue a batch (host arrays in the caller's ids, copied before the call
 * returns) for graph index `graph`; *ticket identifies the request.  Ids are
 * checked here: PR_ERANGE rejects the request.  Thread-safe. */
pr_status pr_server_submit(pr_server* srv, int32_t graph, const int32_t* del_src, const int32_t* del_dst,
                           int64_t n_del, const int32_t* ins_src, const int32_t* ins_dst, int64_t n_ins,
                           int64_t* ticket);
/* Wait up to timeout_s seconds for a request; PR_ETIMEOUT if it is not done. */
pr_status pr_server_wait(pr_server* srv, int64_t ticket, double timeout_s, pr_request_info* info);
/* Wait up to timeout_s seconds until every submitted request is done. */
pr_status pr_server_drain(pr_server* srv, double timeout_s);
/* Seconds on the steady clock the request times use. */
double pr_server_clock(void);
/* Finish the submitted requests, stop the worker, restore the graphs' streams. */
void pr_server_destroy(pr_server* srv);

/*
 * Autotuning of the every-vertex rank sweep (Static, ND and the pull form of
 * DF / DF-P; Alg. 1's sweep, Eq. 1 / Eq. 2).  The paper schedules its sweep
 * with OpenMP dynamic chunks of 2048 vertices (Sec. 5.1.2); on the GPU the
 * sweep's gather is edge-balanced and its speed depends on three settings
 * that pr_autotune picks by timing them on the graph itself:
 *   threads          threads per block: 256, 512 or 1024;
 *   quads_per_lane   in-CSR quads (4 edge slots each) a lane loads per warp
 *                    step: 2, 4 or 8;
 *   hub_vertices     the contributions R[u]/|out(u)| of this many vertices of
 *                    highest out-degree are staged in shared memory by every
 *                    block (0: none).  This is a degree threshold: every vertex
 *                    of out-degree >= hub_min_degree is staged;
 *   fused_epilogue   1: Eq. 1 / Eq. 2 and the frontier tests run inside the
 *                    gather kernel, for each 128-vertex chunk as soon as its
 *                    rows are summed; 0: in a second kernel after the gather;
 *   ranges           1, 2, 4 or 8: the sweep cut into as many vertex ranges; the
 *                    epilogue of a range runs on a second, high-priority
 *                    stream while the next range is gathered (fused_epilogue 0
 *                    only).
 * The setting changes no result: contribution sums are exact (see the
 * conventions above), so every setting gives the same bits.  It belongs to
 * the graph and survives batches.
 * pr_autotune: times every candidate setting on the graph's stream (CUDA
 *   events) and keeps the fastest, writing it to *out (NULL: not written).
 *   method PR_STATIC or PR_NAIVE_DYNAMIC: reps (0: 3; at most 100) sweeps of
 *   Eq. 1 over every vertex per candidate, from the current contributions;
 *   the graph's ranks and edges are left as they were.  method PR_DF or
 *   PR_DFP: reps (0: 1) whole updates per candidate (the iteration loop on the
 *   host, options at their defaults), each from the ranks the graph has on
 *   entry and with its last batch; the rank-sweep kernel time decides, and the
 *   ranks on entry are put back at the end.  Needs ranks (PR_ENORANKS).  A
 *   graph with ranks below PR_DEVICE_LOOP_SLOTS in-CSR slots, whose pr_update
 *   runs the loop on the device with the group kernels, also has the unit
 *   sizes of those kernels tuned (pr_group_autotune on its one-graph group,
 *   same method, ranks put back).  The trials allocate one n-vector of device memory for the
 *   duration of the call.
 *   Errors: PR_EINVAL (method PR_DYNAMIC_TRAVERSAL, whose sweeps are list
 *   sweeps, or bad alpha / tau / reps), PR_ENORANKS, PR_ENOMEM, PR_ECUDA.
 * pr_get_tuning: the graph's current setting (the defaults 1024 / 2 / 0 / 0 / 1
 *   until tuned or set).  ms_gather and candidates are 0 unless pr_autotune chose it.
 * pr_set_tuning: sets threads, quads_per_lane, hub_vertices, fused_epilogue
 *   and ranges (the other fields are ignored).  hub_vertices above n is clamped; a setting outside
 *   the values above, or a hub too large for one block's shared memory
 *   (about 27.9K vertices), gives PR_EINVAL and no change.
 */
typedef struct {
  int32_t threads;
  int32_t quads_per_lane;
  int32_t hub_vertices;
  int32_t fused_epilogue;
  int32_t ranges;
  int32_t hub_min_degree;   /* out-degree of the last staged vertex (0: none)   */
  float ms_gather;          /* pr_autotune: the chosen setting's time per trial (ms): one sweep, or
                               the rank sweeps of one update                        */
  int32_t candidates;       /* pr_autotune: settings timed                      */
} pr_tuning;
pr_status pr_autotune(pr_graph* g, pr_method method, double alpha, double tau, int32_t reps, pr_tuning* out);
pr_status pr_get_tuning(const pr_graph* g, pr_tuning* out);
pr_status pr_set_tuning(pr_graph* g, const pr_tuning* in);

/*
 * Testing aid for failure handling (the paper has no counterpart): the k-th
 * device memory allocation the library makes from now on (k >= 1, counted
 * over all graphs, groups and servers of the process) fails as if the device
 * were out of memory, so callers can test their handling of PR_ENOMEM without
 * exhausting a real GPU.  k = 0 disarms.  Nothing is launched or faulted on
 * the device.
 */
void pr_debug_fail_alloc(int64_t k);

/* Number of CUDA kernels this library has launched in this process so far
 * (all graphs); the difference across a region counts its launches. */
unsigned long long pr_kernel_launches(void);

/*
 * Per-sweep trace of the last pr_update of a graph that ran with
 * PR_OPT_TIME_SWEEPS and its host loop (the device loop and groups keep no
 * per-sweep times): one record per iteration of Alg. 1, in order.  The paper
 * reports whole-update times (Sec. 5.1.5); the trace splits them into the
 * list (push) sweeps over a frontier and the every-vertex (pull) sweeps, so
 * that each kernel form can be held against its own roofline.
 */
typedef struct {
  int32_t iteration;   /* 0-based                                                  */
  int32_t form;        /* PR_SWEEP_LIST or PR_SWEEP_EVERY_VERTEX                   */
  double ms;           /* CUDA-event time of the sweep's launches on the stream    */
  int64_t edges;       /* in-edges summed by the sweep (vertices processed only)   */
  int64_t vertices;    /* vertices the sweep processed                             */
} pr_sweep_record;
#define PR_SWEEP_LIST 0
#define PR_SWEEP_EVERY_VERTEX 1
/* Copies min(cap, count) records to out (host) and sets *count to the number
 * of records of that update (0 if it kept none).  Errors: PR_EINVAL. */
pr_status pr_sweep_log(const pr_graph* g, pr_sweep_record* out, int32_t cap, int32_t* count);

/* Text of the last error on this graph ("" if none); valid until the next call. */
const char* pr_last_error(const pr_graph* g);

/* Name of a status code. */
const char* pr_status_string(pr_status s);

#ifdef __cplusplus
}
#endif

#endif /* DFPR_H */
