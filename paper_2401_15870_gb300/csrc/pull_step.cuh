// pull_step.cuh -- one warp step of the every-vertex sweep (gather and
// epilogue), shared by the single-graph kernels (sweep.cu) and the kernels
// that sweep a group of graphs in one launch (group.cu).
//
// Gather step: a warp takes 32 x SW_QPT consecutive quads of the in-CSR
// capacity (lane = quad), loads them as 128-bit streams, gathers the four
// contributions of each and finds each quad's row from a bitmap of row
// starts (one bit per quad) and the number of rows before every 32-quad word:
// the owner of quad q is rowbase[q/32] + popcount(starts up to q) - 1.  A
// segmented warp reduction leaves one partial sum per row piece, which is
// added to the row's accumulator (exact integer addition, so the order does
// not matter).  In pull form it also records whether any source expanded.
//
// Epilogue step (pull form): a warp owns U consecutive 32-vertex chunks, one
// 32-bit word of every bitset each, so the next frontier's stay / expanded
// words are built with ballots and written whole, with no atomics and no
// clearing beforehand.  Vertices outside F_i keep their rank and copy their
// contribution.  FP64 is the binding pipe of the epilogue on GB300 (about 0.6
// Tops/s), so it is spent only where the formulas need it: the 2^-61 scale is
// folded into alpha (a power of two, so the product is exact), and maxima and
// the threshold tests of non-negative doubles compare their bit patterns as
// integers, which orders them the same way.
#pragma once
#include "fixconv.cuh"
#include "sweep.cuh"

namespace dfpr {

// L2 policies: the streamed CSR columns are read once per sweep (evict first),
// the gathered contributions are reused across the whole sweep (evict last)
__device__ __forceinline__ uint64_t policy_evict_first() {
  uint64_t p;
  asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
  return p;
}
__device__ __forceinline__ uint64_t policy_evict_last() {
  uint64_t p;
  asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
  return p;
}
__device__ __forceinline__ int4 ld_stream4(const int32_t* p, uint64_t pol) {
  int4 v;
  asm volatile("ld.global.nc.L1::no_allocate.L2::cache_hint.v4.s32 {%0, %1, %2, %3}, [%4], %5;"
               : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
               : "l"(p), "l"(pol));
  return v;
}
__device__ __forceinline__ long long ld_hint(const long long* p, uint64_t pol) {
  long long v;
  asm volatile("ld.global.nc.L2::cache_hint.b64 %0, [%1], %2;" : "=l"(v) : "l"(p), "l"(pol));
  return v;
}
// The gather is bound by L2 sector throughput (about 70% of it at R-MAT 24,
// with 19% of its loads hitting L1), so L1 hits matter: internal ids are
// ordered by decreasing out-degree, and the contributions of the sources below
// L1_HUB (128 KB) are the ones many rows on one SM read.  They are cached in
// L1; every other contribution is loaded without allocating an L1 line, so it
// does not evict them.  At R-MAT 25 a DF-P pull sweep took 3.94 ms with every
// load allocating, 3.78 with this cut-off (3.91 at 8192, 3.87 at 32768; an
// evict-first priority instead of no allocation gained nothing).
constexpr int32_t L1_HUB = 16384;
// the contribution at p: one of two predicated loads into the same register
// (allocating in L1 below hub_end, the end of the hub sources'
// contributions, not allocating above)
__device__ __forceinline__ long long ld_contrib(const long long* p, const long long* hub_end, uint64_t pol) {
  long long v;
  asm volatile(
      "{\n\t.reg .pred h;\n\t"
      "setp.lt.u64 h, %1, %2;\n\t"
      "@h ld.global.nc.L2::cache_hint.b64 %0, [%1], %3;\n\t"
      "@!h ld.global.nc.L1::no_allocate.L2::cache_hint.b64 %0, [%1], %3;\n\t}"
      : "=l"(v)
      : "l"(p), "l"(hub_end), "l"(pol));
  return v;
}
// ordinary (weak) loads, for data written earlier in the same launch: the
// read-only path may hold stale lines then, while an ordinary load after the
// grid barrier's acquire sees every write made before the barrier
__device__ __forceinline__ long long ld_weak_hint(const long long* p, uint64_t pol) {
  long long v;
  asm volatile("ld.global.L2::cache_hint.b64 %0, [%1], %2;" : "=l"(v) : "l"(p), "l"(pol) : "memory");
  return v;
}
__device__ __forceinline__ uint32_t ld_weak(const uint32_t* p) {
  uint32_t v;
  asm volatile("ld.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ long long ld_weak(const long long* p) {
  long long v;
  asm volatile("ld.global.b64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ double ld_weak(const double* p) {
  double v;
  asm volatile("ld.global.f64 %0, [%1];" : "=d"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ unsigned long long dbits(double x) { return (unsigned long long)__double_as_longlong(x); }

// Contributions (and, in pull form, expanded-source bits) of the hub vertices
// [0, k) staged in shared memory by the kernel.  Internal ids are ordered by
// decreasing out-degree, so [0, k) are the vertices of out-degree at least
// odeg[k-1]: the sources that the most in-rows gather from.  A shared-memory
// load of random addresses costs a few bank wavefronts per warp, where the
// same loads from global memory cost about one L1TEX wavefront per lane.
struct HubView {
  const long long* c = nullptr;   // c[0..k): C[0..k)
  const uint32_t* x = nullptr;    // x[0..kx): X[0..kx) (pull form)
  int32_t k = 0, kx = 0;
};

// What one gather step touched: the rows of its first and last quads (the
// same in every lane) and whether this lane wrote an accumulator.
struct GatherSpan {
  int first, last;
  bool wrote;
};

// quads [base, base + 32 * QPT) of one in-CSR, those below qlo or from nquads
// on left out; S / X / anyb only in pull form.
// SPAN: also report what the step touched (the one-launch sweep needs it; the
// other callers skip the extra warp operations).
// COH: the contributions and the S / X words were written earlier in the same
// launch (a kernel that runs the whole iteration loop): they are read with
// ordinary loads, not through the read-only path
template <bool PULL, int QPT = SW_QPT, bool HUB = false, bool SPAN = false, bool COH = false>
__device__ __forceinline__ GatherSpan gather_step(const int32_t* __restrict__ icol, const long long* __restrict__ C,
                                                  const uint32_t* __restrict__ X, const uint32_t* __restrict__ S,
                                                  const uint32_t* __restrict__ rowbits,
                                                  const int32_t* __restrict__ rowbase, int64_t nquads, int32_t sent,
                                                  long long* __restrict__ acc, uint32_t* __restrict__ anyb,
                                                  int64_t base, uint64_t pol_stream, uint64_t pol_keep,
                                                  const HubView& hub = HubView(), int64_t qlo = 0) {
  const int lane = threadIdx.x & 31;
  const unsigned upto = lane == 31 ? 0xffffffffu : ((2u << lane) - 1u);
  // sentinel slots (row slack) contribute 0 and issue no load; a hub cache
  // that covers the sentinel id holds C[sent] = 0
  auto contrib = [&](int32_t c) -> long long {
    if (HUB && c < hub.k) return hub.c[c];
    if (c == sent) return 0ll;
    return COH ? ld_weak_hint(C + c, pol_keep) : ld_contrib(C + c, C + L1_HUB, pol_keep);
  };
  auto expanded = [&](int32_t c) -> unsigned {
    if (c == sent) return 0u;
    const uint32_t w = HUB && (c >> 5) < hub.kx ? hub.x[c >> 5] : (COH ? ld_weak(X + (c >> 5)) : __ldg(X + (c >> 5)));
    return w >> (c & 31);
  };
  int4 c[QPT];
  int owner[QPT];
  // the row-start words of the step's QPT 32-quad words in one vector load
  // each: a step starts at a multiple of 32 x QPT quads, and both arrays are
  // padded to a multiple of 8 words, so the loads are aligned and in bounds
  // (words past the last quad are read but not used)
  static_assert(QPT == 2 || QPT % 4 == 0, "quads per lane: 2 or a multiple of 4");
  uint32_t wb[QPT];
  int32_t wr[QPT];
  {
    const int64_t w0 = base >> 5;
    if constexpr (QPT == 2) {
      const uint2 b = __ldg(reinterpret_cast<const uint2*>(rowbits + w0));
      const int2 r = __ldg(reinterpret_cast<const int2*>(rowbase + w0));
      wb[0] = b.x;
      wb[1] = b.y;
      wr[0] = r.x;
      wr[1] = r.y;
    } else {
#pragma unroll
      for (int j = 0; j < QPT; j += 4) {
        const uint4 b = __ldg(reinterpret_cast<const uint4*>(rowbits + w0 + j));
        const int4 r = __ldg(reinterpret_cast<const int4*>(rowbase + w0 + j));
        wb[j] = b.x;
        wb[j + 1] = b.y;
        wb[j + 2] = b.z;
        wb[j + 3] = b.w;
        wr[j] = r.x;
        wr[j + 1] = r.y;
        wr[j + 2] = r.z;
        wr[j + 3] = r.w;
      }
    }
  }
#pragma unroll
  for (int j = 0; j < QPT; j++) {
    const int64_t q = base + 32 * j + lane;
    const bool valid = q >= qlo && q < nquads;
    c[j] = valid ? ld_stream4(icol + 4 * q, pol_stream) : make_int4(sent, sent, sent, sent);
    owner[j] = valid ? wr[j] + __popc(wb[j] & upto) - 1 : -1;
  }
  long long s[QPT];
  unsigned x[QPT];
#pragma unroll
  for (int j = 0; j < QPT; j++) {
    s[j] = contrib(c[j].x) + contrib(c[j].y) + contrib(c[j].z) + contrib(c[j].w);
    x[j] = 0;
    // a row whose vertex stays in the frontier is processed anyway: its
    // sources' expanded bits are not needed
    if (PULL && owner[j] >= 0 &&
        !(((COH ? ld_weak(S + (owner[j] >> 5)) : __ldg(S + (owner[j] >> 5))) >> (owner[j] & 31)) & 1u))
      x[j] = (expanded(c[j].x) | expanded(c[j].y) | expanded(c[j].z) | expanded(c[j].w)) & 1u;
  }
  GatherSpan span{0, 0, false};
  if (SPAN) {
    span.first = __shfl_sync(0xffffffffu, owner[0], 0);
    int hi = owner[0];
#pragma unroll
    for (int j = 1; j < QPT; j++) hi = max(hi, owner[j]);
    span.last = __reduce_max_sync(0xffffffffu, hi);
  }
  // Segmented reduction of each 32-quad word: a row piece's sum ends up in its
  // first lane.  Warp shuffles move data through the same L1TEX data pipe as
  // the gathers, so only the sums are shuffled: whether two lanes hold the same
  // row follows from the word's row-start bits (and the edges of the valid
  // quads), and whether any source of a row piece expanded from one ballot.
#pragma unroll
  for (int j = 0; j < QPT; j++) {
    const int own = owner[j];
    long long sum = s[j];
    // segment starts: lane 0, the row starts, and where the valid quads
    // ([qlo, nquads), owner >= 0) begin and end
    const unsigned vm = __ballot_sync(0xffffffffu, own >= 0);
    const unsigned long long st = (unsigned long long)(wb[j] | 1u | (vm ^ (vm << 1)));
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const long long os = __shfl_down_sync(0xffffffffu, sum, o);
      // lane + o holds the same row piece when no segment starts in (lane, lane + o]
      if (lane + o < 32 && ((st >> (lane + 1)) & ((1ull << o) - 1ull)) == 0) sum += os;
    }
    unsigned any = 0u;
    if (PULL) {
      const unsigned xm = __ballot_sync(0xffffffffu, x[j] != 0u);
      const unsigned long long later = (st >> (lane + 1)) << (lane + 1);   // starts after this lane
      const int end = later ? __ffsll((long long)later) - 1 : 32;         // this lane's segment ends before it
      const unsigned seg = (unsigned)(((1ull << end) - 1ull) & ~((1ull << lane) - 1ull));
      any = (xm & seg) != 0u;
    }
    if (own >= 0 && ((st >> lane) & 1ull)) {
      if (sum) atomicAdd(reinterpret_cast<unsigned long long*>(acc + own), (unsigned long long)sum);
      if (PULL && any) atomicOr(anyb + (own >> 5), 1u << (own & 31));
      if (SPAN) span.wrote = span.wrote || sum != 0 || (PULL && any);
    }
  }
  return span;
}

constexpr int FIN_U = 4;   // chunks per warp step of the epilogue: their loads are issued together

// per-thread totals of the epilogue (lane 0 holds the frontier counts)
struct PullTotals {
  unsigned long long dmax = 0ull;   // max |r - R[v]| as the bits of a non-negative double
  long long edges = 0, verts = 0;
  long long ever_new = 0;           // vertices processed for the first time in this update
  int stays = 0, exps = 0;
};

// chunks [ch0, ch0 + U) of one graph.  P provides n, odeg, ideg, R, Ccur,
// Cnext, S_cur, S_next, X_next, ever, tab_sc, tab_ab, alpha, C0, tau_f, tau_p,
// metric (unless REL).
// The accumulators and the expanded-source words it reads are left zero for
// the next sweep.  L2: read them from L2 (they were written by other SMs in
// the same launch).  COH: also the frontier words, ranks, own contributions
// and ever-affected words, which earlier phases of the same launch wrote
// (a kernel that runs the whole iteration loop).
// REL: the relative measure of Alg. 1 fixed at compile time (the default);
// otherwise p.metric chooses.  SAME: tau_p == tau_f known at compile time (the
// default tolerances), which saves the FP64 product of the prune threshold
template <bool CLOSED, class P, bool L2 = false, int U = FIN_U, bool REL = false, bool SAME = false,
          bool COH = false>
__device__ __forceinline__ void finish_pull_step(const P& p, long long* __restrict__ acc, uint32_t* __restrict__ anyb,
                                                 int64_t ch0, int64_t nchunks, PullTotals& t) {
  const int lane = threadIdx.x & 31;
  const double alpha_fix = p.alpha * FIX_INV;
  const bool same_tau = p.tau_f == p.tau_p;
  // contributions updated in place (the gather that read them has finished):
  // a vertex outside F_i keeps its entry and copies nothing
  const bool inplace = p.Cnext == p.Ccur;
  long long sum[U], cself[U];
  double Rv[U];
  int32_t d[U], din[U];
  bool member[U], valid[U];
  // every load of a vertex is issued up front, whether or not it turns out
  // to be a member: waiting for the membership words before loading the
  // members' data would chain two global-memory latencies, which is what
  // bounds this epilogue (long scoreboard stalls), not the extra bytes
#pragma unroll
  for (int u = 0; u < U; u++) {
    const int64_t ch = ch0 + u;
    const int64_t v = ch * 32 + lane;
    valid[u] = ch < nchunks && v < p.n;
    const uint32_t ab = ch < nchunks ? (L2 || COH ? __ldcg(anyb + ch) : anyb[ch]) : 0u;
    const uint32_t sw = ch < nchunks ? (COH ? ld_weak(p.S_cur + ch) : __ldg(p.S_cur + ch)) : 0u;
    const uint32_t in_f = ab | sw;
    member[u] = valid[u] && ((in_f >> lane) & 1u);
    sum[u] = valid[u] ? (L2 || COH ? __ldcg(acc + v) : acc[v]) : 0;
    // the own contribution: Eq. 2's self term, or the entry a non-member copies
    cself[u] = (CLOSED || !inplace) && valid[u] ? (COH ? ld_weak(p.Ccur + v) : p.Ccur[v]) : 0;
    Rv[u] = valid[u] ? (COH ? ld_weak(p.R + v) : p.R[v]) : 0.0;
    d[u] = valid[u] ? p.odeg[v] : 1;
    din[u] = valid[u] ? p.ideg[v] : 0;
  }
#pragma unroll
  for (int u = 0; u < U; u++) {
    const int64_t ch = ch0 + u;
    const int64_t v = ch * 32 + lane;
    bool stay = false, expand = false;
    if (valid[u]) acc[v] = 0;
    if (member[u]) {
      double r;
      if (CLOSED) {
        // Eq. 2, the self term removed exactly in fixed point, as one FMA
        const long long K = sum[u] - cself[u];
        const double2 ab = d[u] < TAB ? p.tab_ab[d[u]] : closed_coeffs(p.alpha, p.n, d[u]);
        r = fma(ab.x, (double)K, ab.y);
      } else {
        r = fma(alpha_fix, (double)sum[u], p.C0);   // Eq. 1
      }
      const unsigned long long drb = dbits(fabs(r - Rv[u]));
      t.dmax = drb > t.dmax ? drb : t.dmax;
      t.edges += din[u];
      t.verts += 1;
      p.R[v] = r;
      const double sc = d[u] < TAB ? p.tab_sc[d[u]] : FIX_ONE / (double)d[u];
      p.Cnext[v] = fixconv::f64_to_i64_rn(r * sc);   // the FP64 pipe bounds this epilogue
      // Alg. 1: prune when dr / max(r, R[v]) <= tau_p (DF-P), expand when it
      // is > tau_f (or the other measures of Sec. 4.3); compared without the
      // division
      const double mx = dbits(r) > dbits(Rv[u]) ? r : Rv[u];
      const double mr = REL ? mx : measure_base(p.metric, mx, d[u]);
      const unsigned long long tf = dbits(p.tau_f * mr);
      const unsigned long long tp = SAME || same_tau ? tf : dbits(p.tau_p * mr);
      stay = !CLOSED || drb > tp;
      expand = drb > tf;
    } else if (valid[u] && !inplace) {
      p.Cnext[v] = cself[u];
    }
    const unsigned ms = __ballot_sync(0xffffffffu, stay);
    const unsigned mx = __ballot_sync(0xffffffffu, expand);
    const unsigned mm = __ballot_sync(0xffffffffu, member[u]);
    if (lane == 0 && ch < nchunks) {
      anyb[ch] = 0u;
      p.S_next[ch] = ms;
      p.X_next[ch] = mx;
      if (mm) {
        const uint32_t old = COH ? ld_weak(p.ever + ch) : p.ever[ch];
        if (mm & ~old) {
          p.ever[ch] = old | mm;
          t.ever_new += __popc(mm & ~old);
        }
      }
      t.stays += __popc(ms);
      t.exps += __popc(mx);
    }
  }
}

}  // namespace dfpr
