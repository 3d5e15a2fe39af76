// sweep.cuh -- the pull rank sweep and the frontier kernels around it.
#pragma once
#include "graph.cuh"

namespace dfpr {

constexpr int SW_THREADS = 256;
constexpr int SW_QPT = 4;                          // quads per thread per tile
constexpr int SW_TILE_Q = SW_THREADS * SW_QPT;     // 1024 quads = 4096 edge slots per tile
constexpr int SW_MAX_ITEMS = SW_TILE_Q + 2;        // items loaded per tile (those touching it, plus one)

enum SweepMode : int {
  SWEEP_FULL = 0,     // every vertex, Eq. 1, writes R in place and the next contribution buffer (Static, ND)
  SWEEP_LIST = 1,     // a fixed vertex list, Eq. 1, new ranks to rnew (Dynamic Traversal)
  SWEEP_DF = 2,       // frontier list, Eq. 1, expand on a large relative change (DF, push)
  SWEEP_DFP = 3,      // frontier list, Eq. 2, prune on a small one, expand on a large one (DF-P, push)
  SWEEP_PULL_DF = 4,  // every vertex, processed if in the frontier (stay bit or an expanded in-neighbour), DF
  SWEEP_PULL_DFP = 5, // the same for DF-P
};

// The measure of Sec. 4.3 that a DF / DF-P vertex compares with tau_f and
// tau_p, as the factor of the tolerance: dr > tau * measure_base (relative
// change: max(r, R[v]); rank change: 1; contribution factor dr / d: d).
enum Metric : int { METRIC_RELATIVE = 0, METRIC_ABSOLUTE = 1, METRIC_CONTRIB = 2 };
// d >= 1 as a double, assembled from its bits with integer instructions
// (exact: a 31-bit integer fits the 53-bit significand), so the default
// relative measure pays no FP64 conversion even where the compiler evaluates
// both arms of the choice below
__device__ __forceinline__ double degree_as_double(int32_t d) {
  const uint32_t u = (uint32_t)d;
  const int msb = 31 - __clz(u);
  const unsigned long long frac = ((unsigned long long)u << (52 - msb)) & ((1ull << 52) - 1);
  return __longlong_as_double((long long)(((unsigned long long)(1023 + msb) << 52) | frac));
}
__device__ __forceinline__ double measure_base(int metric, double mr, int32_t d) {
  return metric == METRIC_RELATIVE ? mr : (metric == METRIC_ABSOLUTE ? 1.0 : degree_as_double(d));
}

// Eq. 2 as one FMA: r = f (C0 + alpha K 2^-61) with f = 1 / (1 - alpha/d) is
// evaluated as fma(a, K, b), a = f alpha 2^-61, b = f C0, C0 = (1 - alpha)/n;
// the tables hold (a, b) for d < TAB, and larger degrees compute them here
// with the same operations, so both give the same bits
__device__ __forceinline__ double2 closed_coeffs(double alpha, int32_t n, int32_t d) {
  const double f = 1.0 / (1.0 - alpha / (double)d);
  const double C0 = (1.0 - alpha) / (double)n;
  return make_double2(f * (alpha * FIX_INV), f * C0);
}

struct SweepParams {
  int32_t n;
  const int64_t* ioff;
  const int32_t* ideg;
  const int32_t* icol;
  const int32_t* odeg;
  const long long* Ccur;
  long long* Cnext;          // FULL only
  double* R;
  double* rnew;              // LIST / DF / DFP
  const double* tab_sc;      // 2^61 / d
  const double2* tab_ab;     // closed_coeffs(alpha, n, d): Eq. 2 as fma(a, K, b)
  double alpha, C0, tau_f, tau_p;
  // contributions of vertices below `hot` are gathered with an L2 evict-last
  // policy and the rest with evict-first, so the most-read contributions
  // (internal ids are ordered by decreasing out-degree) stay in L2
  int32_t hot;
  int32_t metric;            // Metric (DF / DF-P)
  // the swept list: identity (list == nullptr) over in-CSR capacity quads, or
  // list[0..*count) with quad prefix qs
  const int32_t* list;
  const int32_t* count;
  const int64_t* qs;
  const int32_t* tfirst;
  const int64_t* ntiles_dev;  // device tile count (list mode)
  int64_t ntiles_host;        // identity mode
  long long* gacc;
  int32_t* gcnt;
  // frontier outputs (DF / DFP)
  uint32_t* bits_next;
  uint32_t* ever;
  int32_t* wl_next;
  int32_t* cnt_next;
  int32_t* xl;
  int32_t* cnt_x;
  // pull form of the frontier (PULL_*): F_i = S_cur u out(X_cur); the sweep
  // writes S_next (vertices that stay) and X_next (vertices that expand) and
  // counts them in *cnt_next / *cnt_x
  const uint32_t* S_cur;
  const uint32_t* X_cur;
  uint32_t* S_next;
  uint32_t* X_next;
  int32_t* gany;             // per split item: an in-neighbour expanded (n)
  Ctl* ctl;
};

cudaError_t launch_sweep(int mode, const SweepParams& p, cudaStream_t s);

// Launch configuration of the every-vertex gather (k_gather_rows): threads per
// block (256, 512 or 1024), quads per lane per warp step (2, 4 or 8), and the
// number of hub contributions staged in shared memory by every block (0: none;
// internal ids are ordered by decreasing out-degree, so the hub set is the
// vertices whose out-degree is at least that of vertex hub - 1), and whether
// the epilogue runs inside the gather kernel (k_sweep_rows) or as a second
// launch (k_finish_full / k_finish_pull), and in how many vertex ranges the
// sweep runs.  The defaults are the setting the tuner picks for DF-P on
// R-MAT scale 25 (the pull gather in 32 registers, 64 warps per SM).
struct GatherCfg {
  int32_t threads = 1024;
  int32_t qpt = 2;
  int32_t hub = 0;
  int32_t fused = 0;
  int32_t parts = 1;   // vertex ranges whose epilogue overlaps the next range's gather (1, 2, 4, 8)
};

// the second stream and the events of a sweep cut into vertex ranges
struct SweepAux {
  cudaStream_t stream = nullptr;
  cudaEvent_t ev[9] = {};
};
constexpr int GATHER_SMEM_MAX = 227 * 1024;   // dynamic shared memory of one block on sm_103
size_t gather_hub_bytes(int32_t hub_k, int32_t hub_kx);
bool gather_cfg_valid(const GatherCfg& c);
cudaError_t gather_occupancy(const void* fn, int threads, size_t smem, int* bps);
// the gather alone: adds every row's sum to p.gacc (and, if pull, sets anyb)
cudaError_t launch_gather(bool pull, const SweepParams& p, const GatherCfg& cfg, const uint32_t* rowbits,
                          const int32_t* rowbase, uint32_t* anyb, int64_t nquads, cudaStream_t s);

// every-vertex sweep (FULL, PULL_DF, PULL_DFP); p.ntiles_host is the number of
// quads of the in-CSR capacity, p.gacc the all-zero per-vertex accumulators
// (left zero), rowbits / rowbase the row-start index of the in-CSR
// (launch_row_start_index), anyb an n-bit scratch bitset, done the all-zero
// per-chunk unit counts of the one-launch form (cdiv(n, 128) int32, left zero)
// aux: the second stream of a sweep in several ranges (NULL: one range)
// ordered: the asynchronous order -- the cfg.parts vertex ranges are swept one
// after another on s, each gather followed by its epilogue, and the epilogue
// writes the new contributions in place (p.Cnext == p.Ccur), so every range
// gathers the contributions of the ranges before it as updated in this sweep
// bounds (ordered only): the P + 1 range bounds on the host (P = cfg.parts;
// async_range_bounds below)
cudaError_t launch_full_sweep(int mode, const SweepParams& p, const GatherCfg& cfg, const uint32_t* rowbits,
                              const int32_t* rowbase, uint32_t* anyb, int32_t* done, const SweepAux* aux,
                              cudaStream_t s, bool ordered = false, const int32_t* bounds = nullptr);
// The ranges of the asynchronous order: cut at multiples of 128 vertices
// where the in-degree prefix (in-edges of the vertices below, self-loops
// included) times P first reaches k times all in-edges, k = 1 .. P - 1; one
// range below 128 P vertices.  ideg: n in-degrees on the device; scratch:
// cdiv(n, 128) + 1 + scan_tmp_elems(cdiv(n, 128)) + P int64 on the device;
// bounds: P + 1 host ints, written on return (the call waits for s).
cudaError_t async_range_bounds(const int32_t* ideg, int32_t n, int P, int64_t* scratch, int32_t* bounds,
                               cudaStream_t s);
int64_t async_range_scratch(int32_t n, int P);
// ranges of the asynchronous order (PR_OPT_ASYNC): the vertex set cut at
// multiples of 128 into this many consecutive ranges (one range below 128 x
// this many vertices)
constexpr int ASYNC_RANGES = 8;
// row-start index of the in-CSR: rowbits (nquads/32 + 1 words), rowbase (as
// many int32 + 1); tmp: scan_tmp_elems(nquads/32 + 1) int32
cudaError_t launch_row_start_index(const int64_t* off, int32_t n, int64_t nquads, uint32_t* rowbits, int32_t* rowbase,
                                   int32_t* tmp, cudaStream_t s);

// quad prefix + tile starts of list[0..*count) with quads(v) = ceil(deg[v]/4);
// writes qs[0..K], tfirst[0..ntiles], *qtot_dev, *ntiles_dev.  tmp: >= list_scan_tmp(n) int64
int64_t list_scan_tmp(int32_t n);
cudaError_t launch_list_scan(const int32_t* list, const int32_t* count, const int32_t* deg, int32_t n, int64_t* qs,
                             int32_t* tfirst, int64_t* qtot_dev, int64_t* ntiles_dev, int64_t* tmp, cudaStream_t s);

struct ExpandParams {
  int32_t n;
  const int64_t* ooff;
  const int32_t* ocol;
  const int32_t* list;       // expanding vertices
  const int32_t* count;
  const int64_t* qs;
  const int32_t* tfirst;
  const int64_t* ntiles_dev;
  uint32_t* bits;            // marks (test-and-set)
  uint32_t* ever;            // nullable
  int32_t* wl;               // appended newly marked vertices
  int32_t* cnt;
  // previous-snapshot traversal (Dynamic Traversal on G_{t-1}): skip inserted edges
  const uint32_t* ins_src_bits;   // nullable: sources with effective insertions
  const uint64_t* dplus;          // sorted packed keys of effective insertions
  int64_t n_dplus;
  int id_bits;
};
cudaError_t launch_expand(const ExpandParams& p, cudaStream_t s);

// commit ranks of list[0..*count): R[v] = rnew[k], contribution refreshed;
// clears v's bit in bits_clear when non-null
cudaError_t launch_commit(const int32_t* list, const int32_t* count, const double* rnew, double* R, long long* C,
                          const int32_t* odeg, const double* tab_sc, uint32_t* bits_clear, int32_t n, cudaStream_t s);

}  // namespace dfpr
