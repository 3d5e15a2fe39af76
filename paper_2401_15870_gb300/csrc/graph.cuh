// graph.cuh -- the device-resident graph state behind the opaque pr_graph.
#pragma once
#include <string>
#include <vector>
#include "common.cuh"

namespace dfpr {

// One direction of adjacency: rows with capacity slack (see common.cuh).
struct Csr {
  int64_t* off = nullptr;   // n+1 capacity offsets, multiples of 4
  int32_t* deg = nullptr;   // n
  int32_t* col = nullptr;   // off[n] slots, SENT beyond deg
  int64_t cap = 0;          // off[n] (host copy)
  int32_t repacks = 0;      // times this direction was rebuilt after an overflow
};

// Per-iteration control block, device resident; the host reads a copy.
struct Ctl {
  int32_t count[2];             // worklist sizes
  int32_t nexp;                 // expander list size
  int32_t cur;                  // current worklist / bitset index
  int32_t iter;                 // iterations done
  int32_t done;                 // converged (1) or not (0)
  unsigned long long dR;        // bit pattern of this iteration's L-inf change (non-negative double)
  unsigned long long dR_last;   // of the last finished iteration
  int64_t qtot;                 // quads of the list being swept
  int64_t ntiles;               // tiles of the list being swept
  int64_t xqtot, xntiles;       // quads / tiles of the expander list
  int64_t edges;                // in-edges processed (all iterations)
  int64_t verts;                // vertices processed (all iterations)
  int32_t status;               // device-detected error (0 = none)
  int32_t nexp_last;            // expander count of the last finished iteration
  int32_t nbig;                 // rows deferred to the long-row pass of a full sweep
  int32_t pad;
};

struct Scratch {
  void* p = nullptr;
  size_t bytes = 0;
};

struct Graph {
  int32_t n = 0;
  int id_bits = 1;              // bits of a vertex id (packed edge keys are src << id_bits | dst)
  int64_t m = 0;                // edges, one self-loop per vertex included
  int dev = 0;
  cudaStream_t stream = nullptr;
  bool relabel = true;

  Csr out, in;
  int32_t* perm = nullptr;      // user id -> internal id
  int32_t* iperm = nullptr;     // internal id -> user id

  double* R = nullptr;          // ranks, internal ids
  long long* C[2] = {nullptr, nullptr};  // fixed-point contributions, n+1 each
  int ccur = 0;                 // which C buffer is current
  bool has_ranks = false;

  // tables indexed by out-degree d in [0, TAB): 2^61/d, and the coefficients
  // of Eq. 2 as one FMA (closed_coeffs, for this graph's n and tab_alpha)
  double* tab_sc = nullptr;
  double2* tab_ab = nullptr;
  double tab_alpha = -1.0;

  // frontier state
  uint32_t* bits[2] = {nullptr, nullptr};   // membership of worklist 0 / 1
  uint32_t* ever = nullptr;                 // vertices ever affected
  uint32_t* aux = nullptr;                  // scratch bitset (sources, BFS visited)
  uint32_t* aux2 = nullptr;
  int32_t* wl[2] = {nullptr, nullptr};      // worklists
  int32_t* xl = nullptr;                    // expander list
  double* rnew = nullptr;                   // new rank per worklist slot
  int64_t* qs = nullptr;                    // quad prefix of the swept list (n+1)
  int32_t* tfirst = nullptr;                // first item of every tile of the swept list
  int64_t* xqs = nullptr;                   // quad prefix of the expander list
  int32_t* xtfirst = nullptr;
  long long* gacc = nullptr;                // partial sums of items split across tiles (n)
  int32_t* gcnt = nullptr;                  // tiles that finished each split item (n)
  int32_t* gany = nullptr;                  // pull sweeps: an in-neighbour of a split item expanded (n)
  int32_t* full_tfirst = nullptr;           // tile starts for the identity list over in-CSR capacity
  int64_t full_ntiles = 0;
  uint32_t* rowbits = nullptr;              // full sweeps: in-CSR quads where a row starts
  int32_t* rowbase = nullptr;               // rows starting before each 32-quad word
  uint32_t* anyb = nullptr;                 // full pull sweeps: an in-neighbour expanded (n bits)
  int32_t* done = nullptr;                  // one-launch full sweeps: gather units counted per 128-vertex chunk

  // effective change of the last batch, packed keys sorted by (src, dst), internal ids
  uint64_t* dmin = nullptr;
  uint64_t* dplus = nullptr;
  int64_t n_dmin = 0, n_dplus = 0;
  int64_t cap_dmin = 0, cap_dplus = 0;

  Ctl* ctl = nullptr;       // device
  Ctl* ctl_h = nullptr;     // pinned host mirror

  Scratch scr[8];
  void* small_h = nullptr;  // pinned host copy of the small-batch status (batch.cu)
  std::vector<void*> allocs;
  std::string err;
};

constexpr int TAB = 4096;

// scratch slot helper: grows slot i to at least `bytes`
cudaError_t scratch_get(Graph* g, int slot, size_t bytes, void** out);

cudaError_t dalloc(Graph* g, void** p, size_t bytes);
void dfree_all(Graph* g);

// graph.cu
int build_graph_from_user_keys(Graph* g, uint64_t* keys, int64_t nkeys);   // keys: packed user-id edge keys (device)
int build_csr_from_sorted(Graph* g, Csr* c, const uint64_t* keys, int64_t m, bool in_dir, int slack_quads);
int refresh_full_tiles(Graph* g);
int set_error(Graph* g, int code, const char* msg);
int cuda_fail(Graph* g, cudaError_t e, const char* where);

}  // namespace dfpr
