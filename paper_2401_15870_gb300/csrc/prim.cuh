// prim.cuh -- device-wide primitives written for this library: exclusive scan,
// LSD radix sort of 64-bit keys, stream compaction, fills.
#pragma once
#include "common.cuh"

namespace dfpr {

// ------------------------------------------------------------------ scan
// Exclusive prefix sum of in[0..n) into out[0..n], out[n] = total.
// tmp must hold scan_tmp_elems(n) elements of T.  in and out may alias.
int64_t scan_tmp_elems(int64_t n);
template <typename T>
cudaError_t scan_excl(const T* in, T* out, int64_t n, T* tmp, cudaStream_t s);

// ------------------------------------------------------------------ radix sort
// Sorts keys[0..n) ascending on bits [0, nbits); alt is a same-size buffer.
// The result ends in keys.  n < 2^31.  tmp: radix_tmp_bytes(n) bytes.
size_t radix_tmp_bytes(int64_t n);
cudaError_t radix_sort_u64(uint64_t* keys, uint64_t* alt, int64_t n, int nbits, void* tmp, cudaStream_t s);

// ------------------------------------------------------------------ compaction
// out[0..c) = in[i] for which flag[i] != 0, in order; *count_dev = c.
// tmp: compact_tmp_bytes(n) bytes.
size_t compact_tmp_bytes(int64_t n);
cudaError_t compact_u64(const uint64_t* in, const uint8_t* flag, int64_t n, uint64_t* out, int64_t* count_dev,
                        void* tmp, cudaStream_t s);

// flags of first occurrences in a sorted array (flag[i] = i == 0 || k[i] != k[i-1])
cudaError_t flag_unique_sorted(const uint64_t* k, int64_t n, uint8_t* flag, cudaStream_t s);

// ------------------------------------------------------------------ fills
cudaError_t fill_i32(int32_t* p, int32_t v, int64_t n, cudaStream_t s);
cudaError_t fill_i64(int64_t* p, int64_t v, int64_t n, cudaStream_t s);
cudaError_t iota_i32(int32_t* p, int64_t n, cudaStream_t s);

// grid size for grid-stride kernels over n items with `block` threads
int grid_for(int64_t n, int block);
int num_sms();

}  // namespace dfpr
