// frontier.cuh -- marking, reachability and bookkeeping kernels.
#pragma once
#include "graph.cuh"

namespace dfpr {

// sources of the packed keys a[0..na) and b[0..nb): first occurrence in `seen`
// is appended to list / *count
cudaError_t launch_mark_sources(const uint64_t* a, int64_t na, const uint64_t* b, int64_t nb, int id_bits,
                                uint32_t* seen, int32_t* list, int32_t* count, cudaStream_t s);
// targets of the packed keys d[0..nd): test-and-set in bits, append, set ever
cudaError_t launch_mark_targets(const uint64_t* d, int64_t nd, int id_bits, uint32_t* bits, uint32_t* ever,
                                int32_t* list, int32_t* count, cudaStream_t s);
// edges (u, w) of d[0..nd) with u marked in vis: mark w (reachability through deleted edges)
cudaError_t launch_follow_edges(const uint64_t* d, int64_t nd, int id_bits, uint32_t* vis, int32_t* list,
                                int32_t* count, cudaStream_t s);
// set the bit of every source of d[0..nd)
cudaError_t launch_source_bits(const uint64_t* d, int64_t nd, int id_bits, uint32_t* bits, cudaStream_t s);
// list = ascending ids of set bits of (a | b) over [0, n); *count = size.  tmp: n/32+2 int32 + scan tmp
cudaError_t launch_bits_to_list(const uint32_t* a, const uint32_t* b, int32_t n, int32_t* list, int32_t* count,
                                int32_t* tmp, cudaStream_t s);
int64_t bits_to_list_tmp(int32_t n);
// *out = number of set bits of a[0..words)
cudaError_t launch_popcount(const uint32_t* a, int64_t words, long long* out, cudaStream_t s);
// out = a | b over `words` 32-bit words
cudaError_t launch_bits_or(const uint32_t* a, const uint32_t* b, uint32_t* out, int64_t words, cudaStream_t s);

// end-of-iteration bookkeeping (one thread); frontier != 0 swaps the worklists
cudaError_t launch_control(Ctl* ctl, int frontier, cudaStream_t s);

// tables for d in [1, TAB): tab_sc[d] = 2^61 / d and, unless tab_ab is NULL,
// tab_ab[d] = closed_coeffs(alpha, n, d) (the coefficients of Eq. 2 as one FMA)
cudaError_t launch_tables(double* tab_sc, double2* tab_ab, double alpha, int32_t n, cudaStream_t s);
// R = 1/n for all v; C from R
cudaError_t launch_init_uniform(double* R, long long* C, const int32_t* odeg, const double* tab_sc, int32_t n,
                                cudaStream_t s);
// C[v] from R[v] for all v (C[n] = 0)
cudaError_t launch_contrib_all(const double* R, long long* C, const int32_t* odeg, const double* tab_sc, int32_t n,
                               cudaStream_t s);
// C[u] from R[u] for u = list[0..*count)
cudaError_t launch_contrib_list(const int32_t* list, const int32_t* count, const double* R, long long* C,
                                const int32_t* odeg, const double* tab_sc, int32_t n, cudaStream_t s);

// internal <-> user id maps of a vector
cudaError_t launch_gather_f64(const double* in, const int32_t* idx, double* out, int32_t n, cudaStream_t s);
cudaError_t launch_scatter_f64(const double* in, const int32_t* idx, double* out, int32_t n, cudaStream_t s);

}  // namespace dfpr
