// batch.cu -- a batch of edge deletions and insertions applied to the device
// CSR and transpose-CSR in place (Sec. 3.2).
//
//   E_t = (E_{t-1} \ D) u I      (deletions first; self-loop deletions are
//                                 ignored because self-loops are re-added with
//                                 every batch, Sec. 5.1.4 / 4.2.2)
//   Delta- = E_{t-1} \ E_t,  Delta+ = E_t \ E_{t-1}   (the effective change)
//
// Steps: packed keys -> radix sort -> first occurrences -> effective flags by
// binary search in the sorted rows -> compaction (Delta-, Delta+ sorted by
// (src, dst)).  Each touched row is rewritten by one warp: the old row is
// copied to scratch, every surviving element and every insertion computes its
// output position by counting smaller deletions / insertions / old elements,
// and is written back in place; padding slots get the sentinel.  A row whose
// new degree exceeds its capacity triggers a repack of that direction (a full
// rebuild with fresh slack).
#include <algorithm>
#include "batch.cuh"
#include "frontier.cuh"
#include "prim.cuh"
#include "sweep.cuh"

namespace dfpr {

constexpr uint64_t DROP = ~0ull;

struct Carve {
  char* p;
  size_t used = 0;
  explicit Carve(void* base) : p((char*)base) {}
  template <typename T>
  T* take(int64_t n) {
    size_t off = (used + 255) & ~(size_t)255;
    used = off + sizeof(T) * (size_t)(n > 0 ? n : 1);
    return (T*)(p + off);
  }
};

#define GRID_STRIDE(i, n) \
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < (n); i += (int64_t)gridDim.x * blockDim.x)

#define TRY(x)                                          \
  do {                                                  \
    cudaError_t _e = (x);                               \
    if (_e != cudaSuccess) return cuda_fail(g, _e, #x); \
  } while (0)

// ------------------------------------------------------------------ kernels

__global__ void k_validate(const int32_t* __restrict__ s, const int32_t* __restrict__ d, int64_t k, int32_t n,
                           unsigned long long* bad) {
  unsigned long long c = 0;
  GRID_STRIDE(i, k) c += (s[i] < 0 || s[i] >= n || d[i] < 0 || d[i] >= n) ? 1 : 0;
  if (c) atomicAdd(bad, c);
}

// user ids -> packed internal keys; self-loops become DROP
__global__ void k_make_keys(const int32_t* __restrict__ s, const int32_t* __restrict__ d, int64_t k,
                            const int32_t* __restrict__ perm, int bits, uint64_t* __restrict__ out) {
  GRID_STRIDE(i, k) {
    int32_t u = s[i], v = d[i];
    out[i] = (u == v) ? DROP : (((uint64_t)perm[u] << bits) | (uint64_t)perm[v]);
  }
}

__device__ __forceinline__ bool in_row(const int32_t* col, int64_t base, int32_t deg, int32_t x) {
  int32_t lo = 0, hi = deg;
  while (lo < hi) {
    int32_t mid = (lo + hi) >> 1;
    if (col[base + mid] < x) lo = mid + 1;
    else hi = mid;
  }
  return lo < deg && col[base + lo] == x;
}

__device__ __forceinline__ bool key_in(const uint64_t* k, int64_t len, uint64_t x) {
  int64_t lo = 0, hi = len;
  while (lo < hi) {
    int64_t mid = (lo + hi) >> 1;
    if (k[mid] < x) lo = mid + 1;
    else hi = mid;
  }
  return lo < len && k[lo] == x;
}

__device__ __forceinline__ int64_t lower_key(const uint64_t* k, int64_t lo, int64_t hi, uint64_t x) {
  while (lo < hi) {
    int64_t mid = (lo + hi) >> 1;
    if (k[mid] < x) lo = mid + 1;
    else hi = mid;
  }
  return lo;
}

// effective deletion: first occurrence, present in E_{t-1}, not re-inserted
__global__ void k_flag_del(const uint64_t* __restrict__ dk, int64_t nd, const uint64_t* __restrict__ ik, int64_t ni,
                           const int64_t* __restrict__ oo, const int32_t* __restrict__ od,
                           const int32_t* __restrict__ oc, int bits, uint8_t* __restrict__ f) {
  uint64_t mask = (1ull << bits) - 1;
  GRID_STRIDE(i, nd) {
    uint64_t k = dk[i];
    bool e = k != DROP && (i == 0 || dk[i - 1] != k);
    if (e) {
      int32_t u = (int32_t)(k >> bits), v = (int32_t)(k & mask);
      e = in_row(oc, oo[u], od[u], v) && !key_in(ik, ni, k);
    }
    f[i] = e;
  }
}

// effective insertion: first occurrence, absent from E_{t-1}
__global__ void k_flag_ins(const uint64_t* __restrict__ ik, int64_t ni, const int64_t* __restrict__ oo,
                           const int32_t* __restrict__ od, const int32_t* __restrict__ oc, int bits,
                           uint8_t* __restrict__ f) {
  uint64_t mask = (1ull << bits) - 1;
  GRID_STRIDE(i, ni) {
    uint64_t k = ik[i];
    bool e = k != DROP && (i == 0 || ik[i - 1] != k);
    if (e) {
      int32_t u = (int32_t)(k >> bits), v = (int32_t)(k & mask);
      e = !in_row(oc, oo[u], od[u], v);
    }
    f[i] = e;
  }
}

__global__ void k_swap_keys(const uint64_t* __restrict__ in, int64_t k, int bits, uint64_t* __restrict__ out) {
  uint64_t mask = (1ull << bits) - 1;
  GRID_STRIDE(i, k) out[i] = ((in[i] & mask) << bits) | (in[i] >> bits);
}

__global__ void k_row_keys(const uint64_t* __restrict__ a, int64_t na, const uint64_t* __restrict__ b, int64_t nb,
                           int bits, uint64_t* __restrict__ out) {
  GRID_STRIDE(i, na + nb) out[i] = (i < na ? a[i] : b[i - na]) >> bits;
}

// per touched row: ranges in the deletion / insertion lists, old degree,
// chunk counts of the copy and write passes, overflow
constexpr int RW_CH = 1024;   // row elements per chunk (one warp works on a chunk)

__global__ void k_row_plan(const uint64_t* __restrict__ rows, int64_t nr, const uint64_t* __restrict__ dl, int64_t nd,
                           const uint64_t* __restrict__ il, int64_t ni, int bits, const int64_t* __restrict__ off,
                           const int32_t* __restrict__ deg, int64_t* __restrict__ plan, int64_t* __restrict__ olddeg,
                           int64_t* __restrict__ cchunks, int64_t* __restrict__ wchunks, unsigned long long* overflow) {
  GRID_STRIDE(j, nr) {
    uint64_t r = rows[j];
    int64_t d0 = lower_key(dl, 0, nd, r << bits), d1 = lower_key(dl, d0, nd, (r + 1) << bits);
    int64_t i0 = lower_key(il, 0, ni, r << bits), i1 = lower_key(il, i0, ni, (r + 1) << bits);
    int64_t dg = deg[r];
    int64_t nd2 = dg - (d1 - d0) + (i1 - i0);
    plan[4 * j + 0] = d0;
    plan[4 * j + 1] = d1;
    plan[4 * j + 2] = i0;
    plan[4 * j + 3] = i1;
    olddeg[j] = dg;
    cchunks[j] = cdiv(dg, RW_CH);
    wchunks[j] = cdiv(round4(dg > nd2 ? dg : nd2), RW_CH);
    if (round4(nd2) > off[r + 1] - off[r]) atomicAdd(overflow, 1ull);
  }
}

// row j of chunk c: largest j with pre[j] <= c
__device__ __forceinline__ int64_t chunk_row(const int64_t* pre, int64_t nr, int64_t c) {
  int64_t lo = 0, hi = nr - 1;
  while (lo < hi) {
    int64_t mid = (lo + hi + 1) >> 1;
    if (pre[mid] <= c) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

// copy pass: the old elements of every touched row into scratch, one warp per chunk
__global__ void k_row_copy(const uint64_t* __restrict__ rows, const int64_t* __restrict__ nrp,
                           const int64_t* __restrict__ sofs, const int64_t* __restrict__ cpre,
                           const int64_t* __restrict__ off, const int32_t* __restrict__ deg,
                           const int32_t* __restrict__ col, int32_t* __restrict__ scratch, const int32_t* skip) {
  if (skip && *skip) return;
  const int64_t nr = *nrp;
  const int lane = threadIdx.x & 31;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int64_t total = cpre[nr];
  for (int64_t c = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; c < total; c += nw) {
    const int64_t j = chunk_row(cpre, nr, c);
    const int64_t r = (int64_t)rows[j];
    const int64_t x0 = (c - cpre[j]) * RW_CH;
    const int64_t x1 = min(x0 + (int64_t)RW_CH, (int64_t)deg[r]);
    const int64_t base = off[r];
    int32_t* S = scratch + sofs[j];
    for (int64_t x = x0 + lane; x < x1; x += 32) S[x] = col[base + x];
  }
}

// write pass over old positions: every surviving element moves to
// x - (#deletions below it) + (#insertions below it); slots from the new degree
// up to the old end get the sentinel
__global__ void k_row_survivors(const uint64_t* __restrict__ rows, const int64_t* __restrict__ nrp,
                                const int64_t* __restrict__ plan, const int64_t* __restrict__ sofs,
                                const int64_t* __restrict__ wpre, const uint64_t* __restrict__ dl,
                                const uint64_t* __restrict__ il, int bits, const int64_t* __restrict__ off,
                                const int32_t* __restrict__ deg, int32_t* __restrict__ col,
                                const int32_t* __restrict__ scratch, int32_t sent, const int32_t* skip) {
  if (skip && *skip) return;
  const int64_t nr = *nrp;
  const int lane = threadIdx.x & 31;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int64_t total = wpre[nr];
  for (int64_t c = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; c < total; c += nw) {
    const int64_t j = chunk_row(wpre, nr, c);
    const int64_t r = (int64_t)rows[j];
    const int64_t d0 = plan[4 * j], d1 = plan[4 * j + 1], i0 = plan[4 * j + 2], i1 = plan[4 * j + 3];
    const int64_t d_old = deg[r];
    const int64_t d_new = d_old - (d1 - d0) + (i1 - i0);
    const int64_t pad_end = round4(d_old > d_new ? d_old : d_new);
    const int64_t base = off[r], cap = off[r + 1] - base;
    const int32_t* S = scratch + sofs[j];
    const int64_t x0 = (c - wpre[j]) * RW_CH;
    const int64_t x1 = min(x0 + (int64_t)RW_CH, pad_end);
    for (int64_t x = x0 + lane; x < x1; x += 32) {
      if (x < d_old) {
        const int32_t v = S[x];
        const uint64_t key = ((uint64_t)r << bits) | (uint64_t)v;
        const int64_t dl_lt = lower_key(dl, d0, d1, key);
        if (!(dl_lt < d1 && dl[dl_lt] == key)) {
          const int64_t pos = x - (dl_lt - d0) + (lower_key(il, i0, i1, key) - i0);
          if (pos >= 0 && pos < cap) col[base + pos] = v;
        }
      }
      if (x >= d_new && x < cap) col[base + x] = sent;
    }
  }
}

// write pass over insertions: insertion k of row r goes to
// (#insertions below it) + (#old elements below it) - (#deletions below it)
__global__ void k_row_insertions(const uint64_t* __restrict__ rows, const int64_t* __restrict__ nrp,
                                 const int64_t* __restrict__ plan, const int64_t* __restrict__ sofs,
                                 const uint64_t* __restrict__ dl, const uint64_t* __restrict__ il,
                                 const int64_t* __restrict__ nip, int bits, const int64_t* __restrict__ off,
                                 const int32_t* __restrict__ deg, int32_t* __restrict__ col,
                                 const int32_t* __restrict__ scratch, const int32_t* skip) {
  if (skip && *skip) return;
  const int64_t nr = *nrp, ni = *nip;
  const uint64_t mask = (1ull << bits) - 1;
  GRID_STRIDE(k, ni) {
    const uint64_t r = il[k] >> bits;
    int64_t lo = 0, hi = nr - 1;   // touched-row index of r
    while (lo < hi) {
      int64_t mid = (lo + hi) >> 1;
      if (rows[mid] < r) lo = mid + 1;
      else hi = mid;
    }
    const int64_t j = lo;
    const int64_t d0 = plan[4 * j], d1 = plan[4 * j + 1], i0 = plan[4 * j + 2];
    const int32_t y = (int32_t)(il[k] & mask);
    const int32_t* S = scratch + sofs[j];
    int32_t a = 0, b = deg[r];
    while (a < b) {
      int32_t mid = (a + b) >> 1;
      if (S[mid] < y) a = mid + 1;
      else b = mid;
    }
    const int64_t dl_lt = lower_key(dl, d0, d1, (r << bits) | (uint64_t)y);
    const int64_t pos = (k - i0) + a - (dl_lt - d0);
    const int64_t base = off[r], cap = off[r + 1] - base;
    if (pos >= 0 && pos < cap) col[base + pos] = y;
  }
}

__global__ void k_row_degrees(const uint64_t* __restrict__ rows, const int64_t* __restrict__ nrp,
                              const int64_t* __restrict__ plan, int32_t* __restrict__ deg, const int32_t* skip) {
  if (skip && *skip) return;
  const int64_t nr = *nrp;
  GRID_STRIDE(j, nr) {
    const uint64_t r = rows[j];
    deg[r] = deg[r] - (int32_t)(plan[4 * j + 1] - plan[4 * j]) + (int32_t)(plan[4 * j + 3] - plan[4 * j + 2]);
  }
}

constexpr int32_t REPACK_SHORT = 64;     // rows of at most this degree are rewritten by one thread
constexpr int32_t REPACK_HUB = 16384;    // rows above this degree are spread over many blocks
constexpr int64_t REPACK_CHUNK = 8192;   // elements of a hub row per block

// repack of a direction, pass 1: per row the new degree and the new capacity:
// round4(degree) + 8 slots of slack, a quarter of the degree more for a row
// that received insertions (rows that grew tend to grow again -- a hub of a
// temporal stream -- and geometric slack makes their repacks rare), an eighth
// more for every row of degree >= 64 once the direction has been repacked
// before (the graph keeps growing), and never less than the row had
// (also each row's first deletion and insertion, dstart / istart[0..n], and
// the list of rows above REPACK_HUB with their count and largest degree in
// hinfo[0..1], for pass 2)
__global__ void k_repack_plan(const int64_t* __restrict__ off, const int32_t* __restrict__ deg, int32_t n,
                              const uint64_t* __restrict__ dl, int64_t nd, const uint64_t* __restrict__ il, int64_t ni,
                              int bits, bool growing, int32_t* __restrict__ newdeg, int64_t* __restrict__ cap,
                              int64_t* __restrict__ dstart, int64_t* __restrict__ istart, int32_t* __restrict__ hubs,
                              int32_t* __restrict__ hinfo) {
  GRID_STRIDE(r, n) {
    const int32_t od = deg[r];
    const int slot = warp_append(hinfo, od > REPACK_HUB);
    if (od > REPACK_HUB) {
      hubs[slot] = (int32_t)r;
      atomicMax(hinfo + 1, od);
    }
    const uint64_t rk = (uint64_t)r << bits, rk1 = (uint64_t)(r + 1) << bits;
    const int64_t d0 = lower_key(dl, 0, nd, rk), d1 = lower_key(dl, d0, nd, rk1);
    const int64_t i0 = lower_key(il, 0, ni, rk), i1 = lower_key(il, i0, ni, rk1);
    dstart[r] = d0;
    istart[r] = i0;
    if (r == n - 1) {
      dstart[n] = nd;
      istart[n] = ni;
    }
    const int64_t d = deg[r] - (d1 - d0) + (i1 - i0);
    newdeg[r] = (int32_t)d;
    const int64_t extra = i1 > i0 ? round4(d >> 2) : (growing && d >= 64 ? round4(d >> 3) : 0);
    const int64_t want = round4(d) + 8 + extra, had = off[r + 1] - off[r];
    cap[r] = want > had ? want : had;
  }
}

// pass 2 for the rows longer than REPACK_SHORT: the surviving old elements
// and the insertions merged into the new column array (both are sorted, so
// each element's output position is its rank: survivors x -> i - #deletions
// below x + #insertions below x, insertion y -> k + #old below y - #deletions
// below y), then the padding slots get the sentinel.  part / nparts: this
// call's share of the row -- elements [part * chunk, (part + 1) * chunk) and
// the same share of its insertions and of its padding -- worked by `step`
// threads from t0.
__device__ __forceinline__ void repack_row_part(int64_t r, int64_t part, int64_t nparts, int64_t chunk, int64_t t0,
                                                int64_t step, const int64_t* __restrict__ off,
                                                const int32_t* __restrict__ deg, const int32_t* __restrict__ col,
                                                int32_t n, const uint64_t* __restrict__ dl,
                                                const uint64_t* __restrict__ il, const int64_t* __restrict__ dstart,
                                                const int64_t* __restrict__ istart, int bits,
                                                const int64_t* __restrict__ noff, const int32_t* __restrict__ ndeg,
                                                int32_t* __restrict__ ncol) {
  const uint64_t mask = (1ull << bits) - 1;
  const int64_t dg = deg[r];
  const uint64_t rk = (uint64_t)r << bits;
  const int64_t d0 = dstart[r], d1 = dstart[r + 1];
  const int64_t i0 = istart[r], i1 = istart[r + 1];
  const int64_t base = off[r], nbase = noff[r];
  const int32_t* row = col + base;
  const int64_t x1 = min(dg, (part + 1) * chunk);
  for (int64_t x = part * chunk + t0; x < x1; x += step) {
    const int32_t v = row[x];
    const uint64_t key = rk | (uint64_t)v;
    const int64_t dlt = lower_key(dl, d0, d1, key);
    if (dlt < d1 && dl[dlt] == key) continue;   // deleted
    ncol[nbase + x - (dlt - d0) + (lower_key(il, i0, i1, key) - i0)] = v;
  }
  const int64_t ish = cdiv(i1 - i0, nparts);
  const int64_t k1 = min(i1, i0 + (part + 1) * ish);
  for (int64_t k = i0 + part * ish + t0; k < k1; k += step) {
    const int32_t y = (int32_t)(il[k] & mask);
    int64_t a = 0, b = dg;   // old elements below y
    while (a < b) {
      const int64_t mid = (a + b) >> 1;
      if (row[mid] < y) a = mid + 1;
      else b = mid;
    }
    ncol[nbase + (k - i0) + a - (lower_key(dl, d0, d1, rk | (uint64_t)y) - d0)] = y;
  }
  const int64_t f0 = ndeg[r], f1 = noff[r + 1] - nbase;
  const int64_t fsh = cdiv(f1 - f0, nparts);
  const int64_t e1 = min(f1, f0 + (part + 1) * fsh);
  for (int64_t x = f0 + part * fsh + t0; x < e1; x += step) ncol[nbase + x] = n;
}

// rows of degree in (REPACK_SHORT, REPACK_HUB], one warp per row
__global__ void k_repack_rows(const int64_t* __restrict__ off, const int32_t* __restrict__ deg,
                              const int32_t* __restrict__ col, int32_t n, const uint64_t* __restrict__ dl,
                              const uint64_t* __restrict__ il, const int64_t* __restrict__ dstart,
                              const int64_t* __restrict__ istart, int bits, const int64_t* __restrict__ noff,
                              const int32_t* __restrict__ ndeg, int32_t* __restrict__ ncol) {
  const int lane = threadIdx.x & 31;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t r = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; r < n; r += nw) {
    const int64_t dg = deg[r];
    if (dg <= REPACK_SHORT || dg > REPACK_HUB) continue;   // k_repack_short / k_repack_hub
    repack_row_part(r, 0, 1, dg, lane, 32, off, deg, col, n, dl, il, dstart, istart, bits, noff, ndeg, ncol);
  }
}

// rows of degree above REPACK_HUB (listed by k_repack_plan): block (x, y)
// works share x of hub row hubs[y], REPACK_CHUNK elements each, so a row of
// a million edges is spread over the grid instead of one warp
__global__ void k_repack_hub(const int32_t* __restrict__ hubs, const int64_t* __restrict__ off,
                             const int32_t* __restrict__ deg, const int32_t* __restrict__ col, int32_t n,
                             const uint64_t* __restrict__ dl, const uint64_t* __restrict__ il,
                             const int64_t* __restrict__ dstart, const int64_t* __restrict__ istart, int bits,
                             const int64_t* __restrict__ noff, const int32_t* __restrict__ ndeg,
                             int32_t* __restrict__ ncol) {
  const int64_t r = hubs[blockIdx.y];
  const int64_t nparts = cdiv((int64_t)deg[r], REPACK_CHUNK);
  if ((int64_t)blockIdx.x >= nparts) return;
  repack_row_part(r, blockIdx.x, nparts, REPACK_CHUNK, threadIdx.x, blockDim.x, off, deg, col, n, dl, il, dstart,
                  istart, bits, noff, ndeg, ncol);
}

// pass 2 for the short rows (degree <= REPACK_SHORT), one thread per row: an
// untouched row is copied as whole quads (both offsets are multiples of four
// slots, so the copies are aligned 16-byte moves), a touched one is merged
// element by element (old elements ascending, deletions skipped, insertions
// placed in order: the effective deletions are present and the effective
// insertions absent, so the merge never meets an equal pair).  The rest of the
// new capacity gets the sentinel.  Longer rows are left to k_repack_rows.
__global__ void k_repack_short(const int64_t* __restrict__ off, const int32_t* __restrict__ deg,
                               const int32_t* __restrict__ col, int32_t n, const uint64_t* __restrict__ dl,
                               const uint64_t* __restrict__ il, const int64_t* __restrict__ dstart,
                               const int64_t* __restrict__ istart, int bits, const int64_t* __restrict__ noff,
                               int32_t* __restrict__ ncol) {
  const uint64_t mask = (1ull << bits) - 1;
  GRID_STRIDE(r, n) {
    const int32_t dg = deg[r];
    if (dg > REPACK_SHORT) continue;
    const int64_t d0 = dstart[r], d1 = dstart[r + 1], i0 = istart[r], i1 = istart[r + 1];
    const int32_t* row = col + off[r];
    int32_t* out = ncol + noff[r];
    const int64_t ncap = noff[r + 1] - noff[r];
    int64_t o = 0;
    if (d0 == d1 && i0 == i1) {
      const int64_t q = round4(dg);   // the last quad's slack slots already hold the sentinel
      for (int64_t k = 0; k < q; k += 4)
        *reinterpret_cast<int4*>(out + k) = *reinterpret_cast<const int4*>(row + k);
      o = q;
    } else {
      int64_t di = d0, ii = i0;
      for (int32_t x = 0; x < dg; x++) {
        const int32_t v = row[x];
        while (ii < i1 && (int32_t)(il[ii] & mask) < v) out[o++] = (int32_t)(il[ii++] & mask);
        while (di < d1 && (int32_t)(dl[di] & mask) < v) di++;
        if (di < d1 && (int32_t)(dl[di] & mask) == v) {
          di++;
          continue;
        }
        out[o++] = v;
      }
      while (ii < i1) out[o++] = (int32_t)(il[ii++] & mask);
    }
    for (; o < ncap; o++) out[o] = n;
  }
}

__global__ void k_u64_to_i32_low(const uint64_t* __restrict__ in, int64_t k, int32_t* __restrict__ out) {
  GRID_STRIDE(i, k) out[i] = (int32_t)in[i];
}

// ------------------------------------------------------------------ host

// a direction whose new rows do not fit their capacity is rebuilt with fresh
// slack: new degrees and capacities, their prefix as the new offsets, and the
// rows merged straight into a new column array (no sort: the old rows and the
// insertions are both sorted)
static int repack_direction(Graph* g, Csr* c, const uint64_t* dl, int64_t nd, const uint64_t* il, int64_t ni) {
  cudaStream_t s = g->stream;
  const int bits = g->id_bits;
  const int32_t n = g->n;
  int32_t* ndeg = nullptr;
  int64_t *cap = nullptr, *noff = nullptr, *scr = nullptr, *dstart = nullptr, *istart = nullptr;
  int32_t *ncol = nullptr, *hubs = nullptr, *hinfo = nullptr;
  auto release = [&] {
    cudaFree(ndeg);
    cudaFree(cap);
    cudaFree(noff);
    cudaFree(scr);
    cudaFree(dstart);
    cudaFree(istart);
    cudaFree(hubs);
    cudaFree(hinfo);
  };
  // rows above REPACK_HUB, each holding more than REPACK_HUB of the old edges
  const int64_t hub_cap = std::min<int64_t>(n, c->cap / REPACK_HUB + 1);
  cudaError_t e;
  if ((e = dev_malloc(&ndeg, sizeof(int32_t) * n)) != cudaSuccess ||
      (e = dev_malloc(&cap, sizeof(int64_t) * (n + 1))) != cudaSuccess ||
      (e = dev_malloc(&noff, sizeof(int64_t) * (n + 1))) != cudaSuccess ||
      (e = dev_malloc(&scr, sizeof(int64_t) * scan_tmp_elems(n))) != cudaSuccess ||
      (e = dev_malloc(&dstart, sizeof(int64_t) * (n + 1))) != cudaSuccess ||
      (e = dev_malloc(&istart, sizeof(int64_t) * (n + 1))) != cudaSuccess ||
      (e = dev_malloc(&hubs, sizeof(int32_t) * hub_cap)) != cudaSuccess ||
      (e = dev_malloc(&hinfo, sizeof(int32_t) * 2)) != cudaSuccess ||
      (e = cudaMemsetAsync(hinfo, 0, sizeof(int32_t) * 2, s)) != cudaSuccess) {
    release();
    return cuda_fail(g, e, "cudaMalloc(repack)");
  }
  note_launch(); k_repack_plan<<<grid_for(n, 256), 256, 0, s>>>(c->off, c->deg, n, dl, nd, il, ni, bits, c->repacks > 0,
                                                                 ndeg, cap, dstart, istart, hubs, hinfo);
  e = scan_excl<int64_t>(cap, noff, n, scr, s);
  int64_t total = 0;
  int32_t hinfo_h[2] = {0, 0};
  if (e == cudaSuccess) e = cudaMemcpyAsync(&total, noff + n, sizeof(int64_t), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(hinfo_h, hinfo, sizeof(hinfo_h), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e == cudaSuccess && (hinfo_h[0] < 0 || hinfo_h[0] > hub_cap || hinfo_h[0] > 65535)) e = cudaErrorUnknown;
  if (e == cudaSuccess) e = dev_malloc(&ncol, sizeof(int32_t) * (size_t)total);
  if (e != cudaSuccess) {
    release();
    return cuda_fail(g, e, "repack");
  }
  note_launch(); k_repack_short<<<grid_for(n, 256), 256, 0, s>>>(c->off, c->deg, c->col, n, dl, il, dstart, istart,
                                                                  bits, noff, ncol);
  note_launch(); k_repack_rows<<<num_sms() * 16, 256, 0, s>>>(c->off, c->deg, c->col, n, dl, il, dstart, istart, bits,
                                                              noff, ndeg, ncol);
  if (hinfo_h[0] > 0) {
    const dim3 hgrid((unsigned)cdiv(hinfo_h[1], REPACK_CHUNK), (unsigned)hinfo_h[0]);
    note_launch(); k_repack_hub<<<hgrid, 256, 0, s>>>(hubs, c->off, c->deg, c->col, n, dl, il, dstart, istart, bits, noff,
                                                       ndeg, ncol);
  }
  e = cudaMemcpyAsync(c->off, noff, sizeof(int64_t) * (n + 1), cudaMemcpyDeviceToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(c->deg, ndeg, sizeof(int32_t) * n, cudaMemcpyDeviceToDevice, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  release();
  if (e != cudaSuccess) {
    cudaFree(ncol);
    return cuda_fail(g, e, "repack");
  }
  // the new column array replaces the old one in the graph's allocations
  bool owned = false;
  for (auto& p : g->allocs)
    if (p == c->col) {
      cudaFree(p);
      p = ncol;
      owned = true;
    }
  if (!owned) g->allocs.push_back(ncol);
  c->col = ncol;
  c->cap = total;
  c->repacks++;
  return OK;
}

static int edit_direction(Graph* g, Csr* c, const uint64_t* dl, int64_t nd, const uint64_t* il, int64_t ni,
                          const int64_t* ni_dev, bool* repacked) {
  cudaStream_t s = g->stream;
  int bits = g->id_bits;
  *repacked = false;
  int64_t nrk = nd + ni;
  if (nrk == 0) return OK;
  // touched rows: sorted distinct row ids
  size_t need = 0;
  {
    Carve probe(nullptr);
    probe.take<uint64_t>(nrk);
    probe.take<uint64_t>(nrk);
    probe.take<uint64_t>(nrk);
    probe.take<uint8_t>(nrk);
    probe.take<char>((int64_t)std::max(radix_tmp_bytes(nrk), compact_tmp_bytes(nrk)));
    probe.take<int64_t>(1);
    need = probe.used + 4096;
  }
  void* base;
  TRY(scratch_get(g, 3, need, &base));
  Carve cv(base);
  uint64_t* rk = cv.take<uint64_t>(nrk);
  uint64_t* alt = cv.take<uint64_t>(nrk);
  uint64_t* rows = cv.take<uint64_t>(nrk);
  uint8_t* flag = cv.take<uint8_t>(nrk);
  void* tmp = cv.take<char>((int64_t)std::max(radix_tmp_bytes(nrk), compact_tmp_bytes(nrk)));
  int64_t* cnt = cv.take<int64_t>(1);
  note_launch(); k_row_keys<<<grid_for(nrk, 256), 256, 0, s>>>(dl, nd, il, ni, bits, rk);
  TRY(radix_sort_u64(rk, alt, nrk, bits, tmp, s));
  TRY(flag_unique_sorted(rk, nrk, flag, s));
  TRY(compact_u64(rk, flag, nrk, rows, cnt, tmp, s));
  int64_t nr = 0;
  TRY(cudaMemcpyAsync(&nr, cnt, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
  TRY(cudaStreamSynchronize(s));

  void* base2;
  size_t need2 = 0;
  {
    Carve probe(nullptr);
    probe.take<int64_t>(4 * nr);
    for (int i = 0; i < 3; i++) probe.take<int64_t>(nr + 1);
    probe.take<int64_t>(scan_tmp_elems(nr));
    probe.take<unsigned long long>(1);
    need2 = probe.used + 4096;
  }
  TRY(scratch_get(g, 4, need2, &base2));
  Carve c2(base2);
  int64_t* plan = c2.take<int64_t>(4 * nr);
  int64_t* sofs = c2.take<int64_t>(nr + 1);
  int64_t* cpre = c2.take<int64_t>(nr + 1);
  int64_t* wpre = c2.take<int64_t>(nr + 1);
  int64_t* sscr = c2.take<int64_t>(scan_tmp_elems(nr));
  unsigned long long* ovf = c2.take<unsigned long long>(1);
  TRY(cudaMemsetAsync(ovf, 0, sizeof(unsigned long long), s));
  note_launch(); k_row_plan<<<grid_for(nr, 256), 256, 0, s>>>(rows, nr, dl, nd, il, ni, bits, c->off, c->deg, plan, sofs,
                                                              cpre, wpre, ovf);
  TRY(scan_excl<int64_t>(sofs, sofs, nr, sscr, s));
  TRY(scan_excl<int64_t>(cpre, cpre, nr, sscr, s));
  TRY(scan_excl<int64_t>(wpre, wpre, nr, sscr, s));
  unsigned long long ovf_h = 0;
  int64_t stot = 0;
  TRY(cudaMemcpyAsync(&ovf_h, ovf, sizeof(ovf_h), cudaMemcpyDeviceToHost, s));
  TRY(cudaMemcpyAsync(&stot, sofs + nr, sizeof(stot), cudaMemcpyDeviceToHost, s));
  TRY(cudaStreamSynchronize(s));

  if (ovf_h == 0) {
    void* sp;
    TRY(scratch_get(g, 5, sizeof(int32_t) * (size_t)(stot + 1), &sp));
    int32_t* S = (int32_t*)sp;
    const int wgrid = num_sms() * 16;
    note_launch(); k_row_copy<<<wgrid, 256, 0, s>>>(rows, cnt, sofs, cpre, c->off, c->deg, c->col, S, nullptr);
    note_launch(); k_row_survivors<<<wgrid, 256, 0, s>>>(rows, cnt, plan, sofs, wpre, dl, il, bits, c->off, c->deg, c->col,
                                                         S, g->n, nullptr);
    if (ni) {
      note_launch(); k_row_insertions<<<grid_for(ni, 256), 256, 0, s>>>(rows, cnt, plan, sofs, dl, il, ni_dev, bits,
                                                                        c->off, c->deg, c->col, S, nullptr);
    }
    note_launch(); k_row_degrees<<<grid_for(nr, 256), 256, 0, s>>>(rows, cnt, plan, c->deg, nullptr);
    TRY(cudaGetLastError());
    return OK;
  }

  // repack this direction: survivors + insertions, sorted, rebuilt with more slack
  *repacked = true;
  return repack_direction(g, c, dl, nd, il, ni);
}

// ------------------------------------------------------------------ small batches
//
// A batch of at most SMALL_MAX edges is ingested by one thread block with the
// keys in shared memory: validation, packed keys, sort (bitonic), effective
// flags, compaction, the same lists keyed (dst, src), and for each direction
// the touched rows with their edit plans and prefix sums.  The row rewrite
// kernels above then read every count from the device, so the whole batch
// costs about ten launches and one host synchronisation (the status read at
// the end) instead of ~170 launches and six synchronisations.  A direction
// whose rows overflow their capacity, or whose staging buffer is too small,
// is skipped by the device and finished by the host after the status read.
constexpr int SMALL_MAX = 4096;                 // edges of a batch (deletions + insertions)
constexpr int SMALL_THREADS = 1024;
constexpr int SMALL_SORT = 2 * SMALL_MAX;       // sort slots (each side padded to a power of two)

struct SmallStatus {
  int64_t n_del, n_ins;   // effective deletions / insertions
  int64_t nr[2];          // touched rows, out (0) and in (1)
  int64_t stot[2];        // staging elements (old degrees of the touched rows)
  int32_t skip[2];        // the device left this direction's rows unchanged
  int32_t bad, ovf[2], need[2], pad;
};

struct SmallBufs {
  uint64_t edl[SMALL_MAX], eil[SMALL_MAX];   // Delta-, Delta+ sorted by (src, dst)
  uint64_t sdl[SMALL_MAX], sil[SMALL_MAX];   // the same sorted by (dst, src)
  uint64_t rows[2][SMALL_MAX];
  int64_t plan[2][4 * SMALL_MAX];
  int64_t sofs[2][SMALL_MAX + 1], cpre[2][SMALL_MAX + 1], wpre[2][SMALL_MAX + 1];
  SmallStatus st;
};

constexpr size_t SMALL_SMEM = sizeof(uint64_t) * (2 * SMALL_SORT + SMALL_MAX) + sizeof(int64_t) * SMALL_MAX;

__host__ __device__ __forceinline__ int pow2_at_least(int x) {
  int p = x > 0 ? 1 : 0;
  while (p < x) p <<= 1;
  return p;
}

// ascending bitonic sort of a[0..N), N a power of two (or 0), whole block
__device__ void block_bitonic(uint64_t* a, int N) {
  for (int k = 2; k <= N; k <<= 1)
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int i = threadIdx.x; i < N; i += blockDim.x) {
        const int x = i ^ j;
        if (x > i) {
          const uint64_t p = a[i], q = a[x];
          if ((p > q) == ((i & k) == 0)) {
            a[i] = q;
            a[x] = p;
          }
        }
      }
      __syncthreads();
    }
}

// exclusive prefix sum of w[0..len) in place, whole block; returns the total
__device__ int64_t block_excl_scan(int64_t* w, int len, int64_t* wsum /* 32 */) {
  const int T = blockDim.x, tid = threadIdx.x, lane = tid & 31, wp = tid >> 5;
  const int per = (len + T - 1) / T;
  const int b = min(tid * per, len), e = min(b + per, len);
  int64_t loc = 0;
  for (int i = b; i < e; i++) loc += w[i];
  int64_t x = loc;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    int64_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) wsum[wp] = x;
  __syncthreads();
  if (wp == 0) {
    int64_t z = lane < (T >> 5) ? wsum[lane] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      int64_t y = __shfl_up_sync(0xffffffffu, z, o);
      if (lane >= o) z += y;
    }
    wsum[lane] = z;
  }
  __syncthreads();
  int64_t before = (wp ? wsum[wp - 1] : 0) + x - loc;
  const int64_t total = wsum[(T >> 5) - 1];
  for (int i = b; i < e; i++) {
    const int64_t v = w[i];
    w[i] = before;
    before += v;
  }
  __syncthreads();
  return total;
}

// touched rows of one direction and their edit plans; L holds the deletions
// [0, nde) and insertions [nde, nde + nie), each sorted by (row, col)
__device__ void small_plan(int dir, const uint64_t* L, int nde, int nie, int bits, const int64_t* __restrict__ off,
                           const int32_t* __restrict__ deg, int64_t scap, uint64_t* R, int64_t* W, int64_t* wsum,
                           SmallBufs* B) {
  __shared__ int ovf;
  const int tid = threadIdx.x, T = blockDim.x;
  const int tot = nde + nie, P = pow2_at_least(tot);
  if (tid == 0) ovf = 0;
  for (int i = tid; i < P; i += T) R[i] = i < tot ? (L[i] >> bits) : DROP;
  __syncthreads();
  block_bitonic(R, P);
  for (int i = tid; i < tot; i += T) W[i] = (i == 0 || R[i - 1] != R[i]) ? 1 : 0;
  __syncthreads();
  const int nr = (int)block_excl_scan(W, tot, wsum);
  uint64_t* rows = B->rows[dir];
  for (int i = tid; i < tot; i += T)
    if (i == 0 || R[i - 1] != R[i]) rows[W[i]] = R[i];
  __syncthreads();
  int64_t* plan = B->plan[dir];
  for (int j = tid; j < nr; j += T) {
    const uint64_t r = rows[j];
    const int64_t d0 = lower_key(L, 0, nde, r << bits), d1 = lower_key(L, d0, nde, (r + 1) << bits);
    const int64_t i0 = lower_key(L + nde, 0, nie, r << bits), i1 = lower_key(L + nde, i0, nie, (r + 1) << bits);
    const int64_t dg = deg[r];
    const int64_t nd2 = dg - (d1 - d0) + (i1 - i0);
    plan[4 * j + 0] = d0;
    plan[4 * j + 1] = d1;
    plan[4 * j + 2] = i0;
    plan[4 * j + 3] = i1;
    if (round4(nd2) > off[r + 1] - off[r]) ovf = 1;
    W[j] = dg;
  }
  __syncthreads();
  const int64_t stot = block_excl_scan(W, nr, wsum);
  for (int j = tid; j < nr; j += T) B->sofs[dir][j] = W[j];
  for (int j = tid; j < nr; j += T) W[j] = cdiv((int64_t)deg[rows[j]], RW_CH);
  __syncthreads();
  const int64_t ctot = block_excl_scan(W, nr, wsum);
  for (int j = tid; j < nr; j += T) B->cpre[dir][j] = W[j];
  for (int j = tid; j < nr; j += T) {
    const int64_t dg = deg[rows[j]];
    const int64_t nd2 = dg - (plan[4 * j + 1] - plan[4 * j]) + (plan[4 * j + 3] - plan[4 * j + 2]);
    W[j] = cdiv(round4(dg > nd2 ? dg : nd2), RW_CH);
  }
  __syncthreads();
  const int64_t wtot = block_excl_scan(W, nr, wsum);
  for (int j = tid; j < nr; j += T) B->wpre[dir][j] = W[j];
  if (tid == 0) {
    B->sofs[dir][nr] = stot;
    B->cpre[dir][nr] = ctot;
    B->wpre[dir][nr] = wtot;
    SmallStatus& st = B->st;
    st.nr[dir] = nr;
    st.stot[dir] = stot;
    st.ovf[dir] = ovf;
    st.need[dir] = stot > scap ? 1 : 0;
    st.skip[dir] = (ovf || stot > scap) ? 1 : 0;
  }
  __syncthreads();
}

__global__ void __launch_bounds__(SMALL_THREADS) k_small_ingest(
    const int32_t* __restrict__ ds, const int32_t* __restrict__ dd, int nd, const int32_t* __restrict__ is,
    const int32_t* __restrict__ id, int ni, int32_t n, int bits, const int32_t* __restrict__ perm,
    const int64_t* __restrict__ ooff, const int32_t* __restrict__ odeg, const int32_t* __restrict__ ocol,
    const int64_t* __restrict__ ioff, const int32_t* __restrict__ ideg, int64_t scap_out, int64_t scap_in,
    SmallBufs* B) {
  extern __shared__ uint64_t smem[];
  uint64_t* A = smem;                           // SMALL_SORT: sorts
  uint64_t* L = A + SMALL_SORT;                 // SMALL_MAX: effective lists of the current direction
  uint64_t* R = L + SMALL_MAX;                  // SMALL_SORT: row ids, flags
  int64_t* W = reinterpret_cast<int64_t*>(R + SMALL_SORT);   // SMALL_MAX: scans
  __shared__ int64_t wsum[32];
  __shared__ int bad;
  const int tid = threadIdx.x, T = blockDim.x;
  const uint64_t mask = (1ull << bits) - 1;
  if (tid == 0) bad = 0;
  __syncthreads();
  const int Pd = pow2_at_least(nd), Pi = pow2_at_least(ni);
  uint64_t* dk = A;
  uint64_t* ik = A + Pd;
  // keys in internal ids; self-loops and padding sort last as DROP
  for (int i = tid; i < Pd + Pi; i += T) {
    const bool del = i < Pd;
    const int k = del ? i : i - Pd;
    uint64_t key = DROP;
    if (k < (del ? nd : ni)) {
      const int32_t u = del ? ds[k] : is[k], v = del ? dd[k] : id[k];
      if (u < 0 || u >= n || v < 0 || v >= n) bad = 1;
      else if (u != v) key = ((uint64_t)perm[u] << bits) | (uint64_t)perm[v];
    }
    A[i] = key;
  }
  __syncthreads();
  if (bad) {
    if (tid == 0) {
      SmallStatus& st = B->st;
      memset(&st, 0, sizeof(st));
      st.bad = 1;
      st.skip[0] = st.skip[1] = 1;
    }
    return;
  }
  block_bitonic(dk, Pd);
  block_bitonic(ik, Pi);
  // effective flags (Sec. 3.2): a deletion is a first occurrence, present in
  // E_{t-1} and not re-inserted; an insertion is a first occurrence absent from E_{t-1}
  for (int i = tid; i < nd + ni; i += T) {
    const bool del = i < nd;
    const uint64_t key = del ? dk[i] : ik[i - nd];
    const uint64_t prev = del ? (i > 0 ? dk[i - 1] : DROP) : (i > nd ? ik[i - nd - 1] : DROP);
    bool e = key != DROP && key != prev;
    if (e) {
      const int32_t u = (int32_t)(key >> bits), v = (int32_t)(key & mask);
      const bool present = in_row(ocol, ooff[u], odeg[u], v);
      e = del ? (present && !key_in(ik, ni, key)) : !present;
    }
    R[i] = e;
    W[i] = e;
  }
  __syncthreads();
  const int nde = (int)block_excl_scan(W, nd, wsum);
  const int nie = (int)block_excl_scan(W + nd, ni, wsum);
  for (int i = tid; i < nd + ni; i += T) {
    if (!R[i]) continue;
    if (i < nd) {
      L[W[i]] = dk[i];
      B->edl[W[i]] = dk[i];
    } else {
      L[nde + W[i]] = ik[i - nd];
      B->eil[W[i]] = ik[i - nd];
    }
  }
  __syncthreads();
  small_plan(0, L, nde, nie, bits, ooff, odeg, scap_out, R, W, wsum, B);
  // the same lists keyed (dst, src) for the in-CSR
  const int Pde = pow2_at_least(nde), Pie = pow2_at_least(nie);
  for (int i = tid; i < Pde + Pie; i += T) {
    const bool del = i < Pde;
    const int k = del ? i : i - Pde;
    uint64_t key = DROP;
    if (k < (del ? nde : nie)) {
      const uint64_t x = L[del ? k : nde + k];
      key = ((x & mask) << bits) | (x >> bits);
    }
    A[i] = key;
  }
  __syncthreads();
  block_bitonic(A, Pde);
  block_bitonic(A + Pde, Pie);
  for (int i = tid; i < nde + nie; i += T) {
    const bool del = i < nde;
    const uint64_t key = del ? A[i] : A[Pde + i - nde];
    L[i] = key;
    if (del) B->sdl[i] = key;
    else B->sil[i - nde] = key;
  }
  __syncthreads();
  small_plan(1, L, nde, nie, bits, ioff, ideg, scap_in, R, W, wsum, B);
  if (tid == 0) {
    B->st.n_del = nde;
    B->st.n_ins = nie;
    B->st.bad = 0;
  }
}

// contributions of the touched out-rows' vertices (the sources of the change)
__global__ void k_small_contrib(const uint64_t* __restrict__ rows, const int64_t* __restrict__ nrp,
                                const int32_t* skip, const double* __restrict__ R, long long* __restrict__ C,
                                const int32_t* __restrict__ odeg, const double* __restrict__ tab_sc) {
  if (*skip) return;
  const int64_t nr = *nrp;
  GRID_STRIDE(j, nr) {
    const int32_t u = (int32_t)rows[j];
    const int32_t d = odeg[u];
    const double sc = d < TAB ? tab_sc[d] : FIX_ONE / (double)d;
    C[u] = __double2ll_rn(R[u] * sc);
  }
}

static void launch_small_edit(Graph* g, Csr* c, SmallBufs* B, int dir, int32_t* S, int64_t nk) {
  cudaStream_t s = g->stream;
  const int bits = g->id_bits;
  const uint64_t* dl = dir == 0 ? B->edl : B->sdl;
  const uint64_t* il = dir == 0 ? B->eil : B->sil;
  const int32_t* skip = &B->st.skip[dir];
  const int64_t* nrp = &B->st.nr[dir];
  const int wgrid = num_sms() * 4;
  note_launch(); k_row_copy<<<wgrid, 256, 0, s>>>(B->rows[dir], nrp, B->sofs[dir], B->cpre[dir], c->off, c->deg, c->col,
                                                 S, skip);
  note_launch(); k_row_survivors<<<wgrid, 256, 0, s>>>(B->rows[dir], nrp, B->plan[dir], B->sofs[dir], B->wpre[dir], dl,
                                                      il, bits, c->off, c->deg, c->col, S, g->n, skip);
  note_launch(); k_row_insertions<<<grid_for(nk, 256), 256, 0, s>>>(B->rows[dir], nrp, B->plan[dir], B->sofs[dir], dl, il,
                                                                   &B->st.n_ins, bits, c->off, c->deg, c->col, S, skip);
  note_launch(); k_row_degrees<<<grid_for(nk, 256), 256, 0, s>>>(B->rows[dir], nrp, B->plan[dir], c->deg, skip);
}

// grow-only staging buffer of one direction (scratch slot 5: out, 7: in)
static cudaError_t small_staging(Graph* g, int dir, int64_t elems, int32_t** out, int64_t* cap) {
  const int slot = dir == 0 ? 5 : 7;
  void* p;
  cudaError_t e = scratch_get(g, slot, sizeof(int32_t) * (size_t)(elems + 1), &p);
  if (e != cudaSuccess) return e;
  *out = (int32_t*)p;
  *cap = (int64_t)(g->scr[slot].bytes / sizeof(int32_t)) - 1;
  return cudaSuccess;
}

// phase 1 of a small batch: everything up to the status copy to the host,
// queued on the graph's stream without waiting
static int small_launch(Graph* g, const int32_t* ds, const int32_t* dd, int64_t nd, const int32_t* is,
                        const int32_t* id, int64_t ni, SmallApply* A) {
  cudaStream_t s = g->stream;
  const int32_t n = g->n;
  const int64_t nk = nd + ni;
  void* bp;
  TRY(scratch_get(g, 6, sizeof(SmallBufs), &bp));
  SmallBufs* B = (SmallBufs*)bp;
  if (!g->small_h) TRY(cudaMallocHost(&g->small_h, sizeof(SmallStatus)));
  SmallStatus* h = (SmallStatus*)g->small_h;
  int32_t** S = A->S;
  int64_t* cap = A->cap;
  // staging of at least 64K elements per direction; larger rows are handled by growing it
  TRY(small_staging(g, 0, 65536, &S[0], &cap[0]));
  TRY(small_staging(g, 1, 65536, &S[1], &cap[1]));
  static bool attr_set[64] = {false};
  const bool known = g->dev >= 0 && g->dev < 64;
  if (!known || !attr_set[g->dev]) {
    TRY(cudaFuncSetAttribute(k_small_ingest, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SMALL_SMEM));
    if (known) attr_set[g->dev] = true;
  }
  note_launch();
  k_small_ingest<<<1, SMALL_THREADS, SMALL_SMEM, s>>>(ds, dd, (int)nd, is, id, (int)ni, n, g->id_bits, g->perm,
                                                      g->out.off, g->out.deg, g->out.col, g->in.off, g->in.deg, cap[0],
                                                      cap[1], B);
  TRY(cudaGetLastError());
  launch_small_edit(g, &g->out, B, 0, S[0], nk);
  launch_small_edit(g, &g->in, B, 1, S[1], nk);
  if (g->has_ranks) {
    note_launch();
    k_small_contrib<<<grid_for(nk, 256), 256, 0, s>>>(B->rows[0], &B->st.nr[0], &B->st.skip[0], g->R, g->C[g->ccur],
                                                      g->out.deg, g->tab_sc);
  }
  TRY(cudaMemcpyAsync(h, &B->st, sizeof(SmallStatus), cudaMemcpyDeviceToHost, s));
  A->B = B;
  A->nk = nk;
  return OK;
}

// phase 2: wait for the status, keep the effective change, and finish on the
// host what the device left (a larger staging buffer, or a repack)
static int small_complete(Graph* g, SmallApply* A) {
  cudaStream_t s = g->stream;
  const int32_t n = g->n;
  SmallBufs* B = A->B;
  SmallStatus* h = (SmallStatus*)g->small_h;
  int32_t** S = A->S;
  int64_t* cap = A->cap;
  const int64_t nk = A->nk;
  TRY(cudaStreamSynchronize(s));
  if (h->bad) return set_error(g, ERANGE_, "pr_apply_batch: vertex id out of range");
  const int64_t a = h->n_del, b = h->n_ins;
  // the effective change, kept for the update (grow-only buffers owned by the graph)
  if (g->cap_dmin < a) {
    if (g->dmin) cudaFree(g->dmin);
    g->dmin = nullptr;
    g->cap_dmin = 0;
    TRY(dev_malloc(&g->dmin, sizeof(uint64_t) * (a + 1)));
    g->cap_dmin = a;
  }
  if (g->cap_dplus < b) {
    if (g->dplus) cudaFree(g->dplus);
    g->dplus = nullptr;
    g->cap_dplus = 0;
    TRY(dev_malloc(&g->dplus, sizeof(uint64_t) * (b + 1)));
    g->cap_dplus = b;
  }
  if (a) TRY(cudaMemcpyAsync(g->dmin, B->edl, sizeof(uint64_t) * a, cudaMemcpyDeviceToDevice, s));
  if (b) TRY(cudaMemcpyAsync(g->dplus, B->eil, sizeof(uint64_t) * b, cudaMemcpyDeviceToDevice, s));
  g->n_dmin = a;
  g->n_dplus = b;
  if (a + b == 0) return OK;
  // directions the device skipped: a larger staging buffer, or a repack
  bool redo_out = false, rep_in = false;
  for (int dir = 0; dir < 2; dir++) {
    if (!h->skip[dir]) continue;
    Csr* c = dir == 0 ? &g->out : &g->in;
    if (h->ovf[dir]) {
      int rc = repack_direction(g, c, dir == 0 ? B->edl : B->sdl, a, dir == 0 ? B->eil : B->sil, b);
      if (rc) return rc;
      if (dir == 1) rep_in = true;
    } else {
      TRY(small_staging(g, dir, h->stot[dir], &S[dir], &cap[dir]));
      TRY(cudaMemsetAsync(&B->st.skip[dir], 0, sizeof(int32_t), s));
      launch_small_edit(g, c, B, dir, S[dir], nk);
    }
    if (dir == 0) redo_out = true;
  }
  if (rep_in) {
    int rc = refresh_full_tiles(g);
    if (rc) return rc;
  }
  if (redo_out && g->has_ranks) {
    TRY(cudaMemsetAsync(g->aux, 0, sizeof(uint32_t) * (size_t)(cdiv(n, 32) + 1), s));
    TRY(cudaMemsetAsync(&g->ctl->count[0], 0, sizeof(int32_t), s));
    TRY(launch_mark_sources(g->dmin, a, g->dplus, b, g->id_bits, g->aux, g->wl[0], &g->ctl->count[0], s));
    TRY(launch_contrib_list(g->wl[0], &g->ctl->count[0], g->R, g->C[g->ccur], g->out.deg, g->tab_sc, n, s));
    TRY(cudaMemsetAsync(&g->ctl->count[0], 0, sizeof(int32_t), s));
  }
  TRY(cudaGetLastError());
  return OK;
}

int apply_batch_launch(Graph* g, const int32_t* ds, const int32_t* dd, int64_t nd, const int32_t* is,
                       const int32_t* id, int64_t ni, bool validated, SmallApply* pending) {
  const int64_t nk = nd + ni;
  pending->B = nullptr;
  if (nk > 0 && nk <= SMALL_MAX) return small_launch(g, ds, dd, nd, is, id, ni, pending);
  return apply_batch_device(g, ds, dd, nd, is, id, ni, validated);
}

int apply_batch_complete(Graph* g, SmallApply* pending) {
  if (!pending->B) return OK;
  return small_complete(g, pending);
}

int apply_batch_device(Graph* g, const int32_t* ds, const int32_t* dd, int64_t nd, const int32_t* is,
                       const int32_t* id, int64_t ni, bool validated) {
  cudaStream_t s = g->stream;
  int bits = g->id_bits;
  int32_t n = g->n;
  int64_t nk = nd + ni;
  if (nk > 0 && nk <= SMALL_MAX) {
    SmallApply A;
    const int rc = small_launch(g, ds, dd, nd, is, id, ni, &A);
    return rc != OK ? rc : small_complete(g, &A);
  }
  size_t need;
  {
    Carve probe(nullptr);
    probe.take<uint64_t>(nd);
    probe.take<uint64_t>(ni);
    probe.take<uint64_t>(nk);
    probe.take<uint8_t>(nk);
    probe.take<char>((int64_t)std::max(radix_tmp_bytes(nk), compact_tmp_bytes(nk)));
    probe.take<unsigned long long>(4);
    need = probe.used + 4096;
  }
  void* base;
  TRY(scratch_get(g, 2, need, &base));
  Carve cv(base);
  uint64_t* dk = cv.take<uint64_t>(nd);
  uint64_t* ik = cv.take<uint64_t>(ni);
  uint64_t* alt = cv.take<uint64_t>(nk);
  uint8_t* flag = cv.take<uint8_t>(nk);
  void* tmp = cv.take<char>((int64_t)std::max(radix_tmp_bytes(nk), compact_tmp_bytes(nk)));
  unsigned long long* small = cv.take<unsigned long long>(4);
  if (!validated && nk) {
    TRY(cudaMemsetAsync(small, 0, sizeof(unsigned long long), s));
    if (nd) { note_launch(); k_validate<<<grid_for(nd, 256), 256, 0, s>>>(ds, dd, nd, n, small); }
    if (ni) { note_launch(); k_validate<<<grid_for(ni, 256), 256, 0, s>>>(is, id, ni, n, small); }
    unsigned long long bad = 0;
    TRY(cudaMemcpyAsync(&bad, small, sizeof(bad), cudaMemcpyDeviceToHost, s));
    TRY(cudaStreamSynchronize(s));
    if (bad) return set_error(g, ERANGE_, "pr_apply_batch: vertex id out of range");
  }
  // effective change lists (grow-only buffers owned by the graph)
  if (g->cap_dmin < nd) {
    if (g->dmin) cudaFree(g->dmin);
    g->dmin = nullptr;
    g->cap_dmin = 0;
    TRY(dev_malloc(&g->dmin, sizeof(uint64_t) * (nd + 1)));
    g->cap_dmin = nd;
  }
  if (g->cap_dplus < ni) {
    if (g->dplus) cudaFree(g->dplus);
    g->dplus = nullptr;
    g->cap_dplus = 0;
    TRY(dev_malloc(&g->dplus, sizeof(uint64_t) * (ni + 1)));
    g->cap_dplus = ni;
  }
  if (nd) {
    note_launch(); k_make_keys<<<grid_for(nd, 256), 256, 0, s>>>(ds, dd, nd, g->perm, bits, dk);
    TRY(radix_sort_u64(dk, alt, nd, 2 * bits, tmp, s));
  }
  if (ni) {
    note_launch(); k_make_keys<<<grid_for(ni, 256), 256, 0, s>>>(is, id, ni, g->perm, bits, ik);
    TRY(radix_sort_u64(ik, alt, ni, 2 * bits, tmp, s));
  }
  int64_t* cnts = (int64_t*)(small + 1);
  TRY(cudaMemsetAsync(cnts, 0, 2 * sizeof(int64_t), s));
  if (nd) {
    note_launch(); k_flag_del<<<grid_for(nd, 256), 256, 0, s>>>(dk, nd, ik, ni, g->out.off, g->out.deg, g->out.col, bits, flag);
    TRY(compact_u64(dk, flag, nd, g->dmin, cnts, tmp, s));
  }
  if (ni) {
    note_launch(); k_flag_ins<<<grid_for(ni, 256), 256, 0, s>>>(ik, ni, g->out.off, g->out.deg, g->out.col, bits, flag + nd);
    TRY(compact_u64(ik, flag + nd, ni, g->dplus, cnts + 1, tmp, s));
  }
  int64_t hc[2] = {0, 0};
  TRY(cudaMemcpyAsync(hc, cnts, sizeof(hc), cudaMemcpyDeviceToHost, s));
  TRY(cudaStreamSynchronize(s));
  g->n_dmin = hc[0];
  g->n_dplus = hc[1];
  if (hc[0] + hc[1] == 0) return OK;

  // out-CSR: lists are sorted by (src, dst)
  bool rep_out = false, rep_in = false;
  int rc = edit_direction(g, &g->out, g->dmin, hc[0], g->dplus, hc[1], cnts + 1, &rep_out);
  if (rc) return rc;
  // in-CSR: the same lists keyed (dst, src)
  {
    int64_t a = hc[0], b = hc[1];
    void* base2;
    size_t need2;
    {
      Carve probe(nullptr);
      probe.take<uint64_t>(a);
      probe.take<uint64_t>(b);
      probe.take<uint64_t>(a + b);
      probe.take<char>((int64_t)radix_tmp_bytes(a + b));
      need2 = probe.used + 4096;
    }
    TRY(scratch_get(g, 1, need2, &base2));
    Carve c2(base2);
    uint64_t* sd = c2.take<uint64_t>(a);
    uint64_t* si = c2.take<uint64_t>(b);
    uint64_t* alt2 = c2.take<uint64_t>(a + b);
    void* tmp2 = c2.take<char>((int64_t)radix_tmp_bytes(a + b));
    if (a) {
      note_launch(); k_swap_keys<<<grid_for(a, 256), 256, 0, s>>>(g->dmin, a, bits, sd);
      TRY(radix_sort_u64(sd, alt2, a, 2 * bits, tmp2, s));
    }
    if (b) {
      note_launch(); k_swap_keys<<<grid_for(b, 256), 256, 0, s>>>(g->dplus, b, bits, si);
      TRY(radix_sort_u64(si, alt2, b, 2 * bits, tmp2, s));
    }
    rc = edit_direction(g, &g->in, sd, a, si, b, cnts + 1, &rep_in);
    if (rc) return rc;
  }
  if (rep_in) {
    rc = refresh_full_tiles(g);
    if (rc) return rc;
  }
  // contributions of sources whose out-degree changed (a3)
  if (g->has_ranks) {
    // the sources: reuse worklist 0 and the aux bitset
    TRY(cudaMemsetAsync(g->aux, 0, sizeof(uint32_t) * (size_t)(cdiv(n, 32) + 1), s));
    TRY(cudaMemsetAsync(&g->ctl->count[0], 0, sizeof(int32_t), s));
    TRY(launch_mark_sources(g->dmin, hc[0], g->dplus, hc[1], bits, g->aux, g->wl[0], &g->ctl->count[0], s));
    TRY(launch_contrib_list(g->wl[0], &g->ctl->count[0], g->R, g->C[g->ccur], g->out.deg, g->tab_sc, n, s));
    TRY(cudaMemsetAsync(&g->ctl->count[0], 0, sizeof(int32_t), s));
  }
  TRY(cudaGetLastError());
  return OK;
}

}  // namespace dfpr
