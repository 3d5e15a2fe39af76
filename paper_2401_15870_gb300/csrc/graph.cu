// graph.cu -- building the device CSR + transpose-CSR from an edge list.
//
// Graph construction (Sec. 5.1.3: a self-loop on every vertex, the edge set
// with repeats collapsed) runs on the device: radix sort of packed edge keys,
// first-occurrence compaction, then one CSR per direction with rows rounded to
// whole 16-byte quads plus slack quads for later in-place batch edits.
//
// Vertex relabelling (a GB300 layout choice, not from the paper): internal ids
// are assigned by decreasing out-degree, so the contributions of the vertices
// that are gathered most often sit together in a few MB that stay resident in
// L2 / L1.  Random 8-byte gathers over a 256 MB array reach ~72 Gedge/s on
// GB300, while gathers within a 64 MB L2-resident range reach ~290 Gedge/s.
#include <cstdio>
#include "graph.cuh"
#include "prim.cuh"
#include "sweep.cuh"

namespace dfpr {

int set_error(Graph* g, int code, const char* msg) {
  if (g) g->err = msg;
  return code;
}

int cuda_fail(Graph* g, cudaError_t e, const char* where) {
  char buf[256];
  snprintf(buf, sizeof(buf), "%s: %s", where, cudaGetErrorString(e));
  if (g) g->err = buf;
  return e == cudaErrorMemoryAllocation ? ENOMEM_ : ECUDA_;
}

cudaError_t dalloc(Graph* g, void** p, size_t bytes) {
  cudaError_t e = dev_malloc(p, bytes > 0 ? bytes : 16);
  if (e == cudaSuccess) g->allocs.push_back(*p);
  return e;
}

void dfree_all(Graph* g) {
  for (void* p : g->allocs) cudaFree(p);
  g->allocs.clear();
  for (auto& s : g->scr) {
    if (s.p) cudaFree(s.p);
    s.p = nullptr;
    s.bytes = 0;
  }
}

cudaError_t scratch_get(Graph* g, int slot, size_t bytes, void** out) {
  Scratch& s = g->scr[slot];
  if (s.bytes < bytes) {
    if (s.p) {
      cudaStreamSynchronize(g->stream);
      cudaFree(s.p);
      s.p = nullptr;
      s.bytes = 0;
    }
    size_t want = bytes + bytes / 4 + 256;
    cudaError_t e = dev_malloc(&s.p, want);
    if (e != cudaSuccess) return e;
    s.bytes = want;
  }
  *out = s.p;
  return cudaSuccess;
}

// ------------------------------------------------------------------ kernels

// rowstart[key_row(i)] = i at the first key of each row (every row non-empty)
__global__ void k_row_starts(const uint64_t* __restrict__ keys, int64_t m, int bits, int64_t* __restrict__ rowstart,
                             int32_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x) {
    int32_t r = (int32_t)(keys[i] >> bits);
    if (i == 0 || (int32_t)(keys[i - 1] >> bits) != r) rowstart[r] = i;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) rowstart[n] = m;
}

__global__ void k_deg_cap(const int64_t* __restrict__ rowstart, int32_t n, int slack_quads, int32_t* __restrict__ deg,
                          int64_t* __restrict__ cap) {
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
    int64_t d = rowstart[v + 1] - rowstart[v];
    deg[v] = (int32_t)d;
    cap[v] = round4(d) + 4 * (int64_t)slack_quads;
  }
}

__global__ void k_fill_cols(const uint64_t* __restrict__ keys, int64_t m, int bits, const int64_t* __restrict__ rowstart,
                            const int64_t* __restrict__ off, int32_t* __restrict__ col) {
  uint64_t mask = (1ull << bits) - 1;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x) {
    int32_t r = (int32_t)(keys[i] >> bits);
    col[off[r] + (i - rowstart[r])] = (int32_t)(keys[i] & mask);
  }
}

__global__ void k_pad_rows(const int64_t* __restrict__ off, const int32_t* __restrict__ deg, int32_t n,
                           int32_t* __restrict__ col) {
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x)
    for (int64_t s = off[v] + deg[v]; s < off[v + 1]; s++) col[s] = n;
}

// relabel keys: (-(outdeg), id) ascending = outdeg descending, ties by id
__global__ void k_relabel_keys(const int64_t* __restrict__ rowstart, int32_t n, int bits, uint64_t* __restrict__ vk) {
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
    uint64_t d = (uint64_t)(rowstart[v + 1] - rowstart[v]);
    vk[v] = ((0xFFFFFFFFull - d) << bits) | (uint64_t)v;
  }
}

__global__ void k_perm_from_sorted(const uint64_t* __restrict__ vk, int32_t n, int bits, int32_t* __restrict__ perm,
                                   int32_t* __restrict__ iperm) {
  uint64_t mask = (1ull << bits) - 1;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    int32_t v = (int32_t)(vk[i] & mask);
    iperm[i] = v;
    perm[v] = (int32_t)i;
  }
}

// keys_out[i] = (perm[u] << bits | perm[v]) or, if swap, (perm[v] << bits | perm[u])
__global__ void k_remap_keys(const uint64_t* __restrict__ in, int64_t m, int bits, const int32_t* __restrict__ perm,
                             bool swap, uint64_t* __restrict__ out) {
  uint64_t mask = (1ull << bits) - 1;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x) {
    uint64_t u = (uint64_t)perm[in[i] >> bits], v = (uint64_t)perm[in[i] & mask];
    out[i] = swap ? (v << bits | u) : (u << bits | v);
  }
}

// tile starts of the identity list over capacity quads
__global__ void k_full_tiles(const int64_t* __restrict__ off, int32_t n, int32_t* __restrict__ tfirst, int64_t ntiles) {
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
    int64_t q0 = off[v] >> 2, q1 = off[v + 1] >> 2;
    for (int64_t t = cdiv(q0, SW_TILE_Q); t * SW_TILE_Q < q1; t++) tfirst[t] = (int32_t)v;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) tfirst[ntiles] = n;
}

// ------------------------------------------------------------------ host

struct Tmp {
  std::vector<void*> ptrs;
  ~Tmp() {
    for (void* p : ptrs) cudaFree(p);
  }
  template <typename T>
  cudaError_t get(T** p, size_t elems) {
    cudaError_t e = dev_malloc((void**)p, sizeof(T) * (elems > 0 ? elems : 1));
    if (e == cudaSuccess) ptrs.push_back(*p);
    return e;
  }
};

#define TRY(x)                                         \
  do {                                                 \
    cudaError_t _e = (x);                              \
    if (_e != cudaSuccess) return cuda_fail(g, _e, #x); \
  } while (0)

int build_csr_from_sorted(Graph* g, Csr* c, const uint64_t* keys, int64_t m, bool in_dir, int slack_quads) {
  (void)in_dir;
  cudaStream_t s = g->stream;
  int32_t n = g->n;
  Tmp t;
  int64_t *rowstart, *cap, *scr;
  TRY(t.get(&rowstart, n + 1));
  TRY(t.get(&cap, n + 1));
  TRY(t.get(&scr, scan_tmp_elems(n)));
  note_launch(); k_row_starts<<<grid_for(m, 256), 256, 0, s>>>(keys, m, g->id_bits, rowstart, n);
  if (!c->deg) TRY(dalloc(g, (void**)&c->deg, sizeof(int32_t) * n));
  if (!c->off) TRY(dalloc(g, (void**)&c->off, sizeof(int64_t) * (n + 1)));
  note_launch(); k_deg_cap<<<grid_for(n, 256), 256, 0, s>>>(rowstart, n, slack_quads, c->deg, cap);
  TRY(scan_excl<int64_t>(cap, c->off, n, scr, s));
  int64_t total = 0;
  TRY(cudaMemcpyAsync(&total, c->off + n, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
  TRY(cudaStreamSynchronize(s));
  if (c->col) {
    // replace the column array (repack)
    for (auto& p : g->allocs)
      if (p == c->col) {
        cudaFree(p);
        p = nullptr;
      }
    c->col = nullptr;
  }
  TRY(dalloc(g, (void**)&c->col, sizeof(int32_t) * total));
  c->cap = total;
  note_launch(); k_fill_cols<<<grid_for(m, 256), 256, 0, s>>>(keys, m, g->id_bits, rowstart, c->off, c->col);
  note_launch(); k_pad_rows<<<grid_for(n, 256), 256, 0, s>>>(c->off, c->deg, n, c->col);
  TRY(cudaGetLastError());
  TRY(cudaStreamSynchronize(s));
  return OK;
}

int refresh_full_tiles(Graph* g) {
  int64_t quads = g->in.cap >> 2;
  int64_t nt = cdiv(quads, SW_TILE_Q);
  // row-start index of the in-CSR for the two-phase full sweep
  for (auto& p : g->allocs)
    if (p == g->rowbits || p == g->rowbase) {
      cudaFree(p);
      p = nullptr;
    }
  int64_t words = cdiv(quads, 32) + 1;
  // padded to a multiple of 8 words, plus 8: a sweep step reads the words of
  // its quads (up to 8) with vector loads from a multiple of its width
  const int64_t padded = (cdiv(quads, 32) + 7) / 8 * 8 + 8;
  TRY(dalloc(g, (void**)&g->rowbits, sizeof(uint32_t) * padded));
  TRY(dalloc(g, (void**)&g->rowbase, sizeof(int32_t) * padded));
  TRY(cudaMemsetAsync(g->rowbits, 0, sizeof(uint32_t) * padded, g->stream));
  TRY(cudaMemsetAsync(g->rowbase, 0, sizeof(int32_t) * padded, g->stream));
  {
    int32_t* tmp;
    TRY(dev_malloc(&tmp, sizeof(int32_t) * scan_tmp_elems(words)));
    cudaError_t e = launch_row_start_index(g->in.off, g->n, quads, g->rowbits, g->rowbase, tmp, g->stream);
    cudaStreamSynchronize(g->stream);
    cudaFree(tmp);
    TRY(e);
  }
  if (g->full_tfirst) {
    for (auto& p : g->allocs)
      if (p == g->full_tfirst) {
        cudaFree(p);
        p = nullptr;
      }
    g->full_tfirst = nullptr;
  }
  TRY(dalloc(g, (void**)&g->full_tfirst, sizeof(int32_t) * (nt + 1)));
  g->full_ntiles = nt;
  note_launch(); k_full_tiles<<<grid_for(g->n, 256), 256, 0, g->stream>>>(g->in.off, g->n, g->full_tfirst, nt);
  TRY(cudaGetLastError());
  return OK;
}

// keys: device array of nkeys packed user-id edge keys, which already include
// one self-loop key per vertex; the buffer is consumed.
int build_graph_from_user_keys(Graph* g, uint64_t* keys, int64_t nkeys) {
  cudaStream_t s = g->stream;
  int32_t n = g->n;
  int bits = g->id_bits;
  Tmp t;
  uint64_t *alt, *ukeys;
  uint8_t* flag;
  void *rtmp, *ctmp;
  int64_t* cnt;
  TRY(t.get(&alt, nkeys));
  TRY(t.get((char**)&rtmp, radix_tmp_bytes(nkeys)));
  TRY(radix_sort_u64(keys, alt, nkeys, 2 * bits, rtmp, s));
  TRY(t.get(&flag, nkeys));
  TRY(flag_unique_sorted(keys, nkeys, flag, s));
  ukeys = alt;   // alt is free again after the sort
  TRY(t.get((char**)&ctmp, compact_tmp_bytes(nkeys)));
  TRY(t.get(&cnt, 1));
  TRY(compact_u64(keys, flag, nkeys, ukeys, cnt, ctmp, s));
  int64_t m = 0;
  TRY(cudaMemcpyAsync(&m, cnt, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
  TRY(cudaStreamSynchronize(s));
  g->m = m;

  TRY(dalloc(g, (void**)&g->perm, sizeof(int32_t) * n));
  TRY(dalloc(g, (void**)&g->iperm, sizeof(int32_t) * n));
  if (g->relabel) {
    int64_t* rowstart;
    uint64_t *vk, *vk_alt;
    void* vtmp;
    TRY(t.get(&rowstart, n + 1));
    TRY(t.get(&vk, n));
    TRY(t.get(&vk_alt, n));
    TRY(t.get((char**)&vtmp, radix_tmp_bytes(n)));
    note_launch(); k_row_starts<<<grid_for(m, 256), 256, 0, s>>>(ukeys, m, bits, rowstart, n);
    note_launch(); k_relabel_keys<<<grid_for(n, 256), 256, 0, s>>>(rowstart, n, bits, vk);
    TRY(radix_sort_u64(vk, vk_alt, n, 32 + bits, vtmp, s));
    note_launch(); k_perm_from_sorted<<<grid_for(n, 256), 256, 0, s>>>(vk, n, bits, g->perm, g->iperm);
  } else {
    TRY(iota_i32(g->perm, n, s));
    TRY(iota_i32(g->iperm, n, s));
  }
  // out-CSR on internal ids
  note_launch(); k_remap_keys<<<grid_for(m, 256), 256, 0, s>>>(ukeys, m, bits, g->perm, false, keys);
  {
    uint64_t* alt2;
    TRY(t.get(&alt2, m));
    TRY(radix_sort_u64(keys, alt2, m, 2 * bits, rtmp, s));
    int rc = build_csr_from_sorted(g, &g->out, keys, m, false, 1);
    if (rc) return rc;
    // in-CSR: swapped keys
    note_launch(); k_remap_keys<<<grid_for(m, 256), 256, 0, s>>>(ukeys, m, bits, g->perm, true, keys);
    TRY(radix_sort_u64(keys, alt2, m, 2 * bits, rtmp, s));
    rc = build_csr_from_sorted(g, &g->in, keys, m, true, 1);
    if (rc) return rc;
  }
  TRY(cudaGetLastError());
  return refresh_full_tiles(g);
}

}  // namespace dfpr
