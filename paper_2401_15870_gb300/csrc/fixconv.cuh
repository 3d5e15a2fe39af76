// fixconv.cuh -- the rounding of a new contribution to the nearest multiple of
// 2^-61, in integer arithmetic.
//
// The DF / DF-P epilogue turns every processed vertex's new rank times
// 2^61 / |out(v)| into the nearest integer (its next fixed-point
// contribution).  The epilogue is bound by GB300's narrow FP64 pipe, and this
// conversion is one of its FP64 instructions; doing it with integer
// instructions moves it to the integer pipes.  It follows the IEEE 754
// definition (IEEE 754-2019 Sec. 5.8 convertToIntegerTiesToEven, rounding
// direction roundTiesToEven of Sec. 4.3.1) for the non-negative values below
// 2^63 the sweep produces, so it gives the same integer as the hardware
// conversion; tests/test_fixconv.py checks it against the C library's llrint
// on every exponent and every kind of tie, and the GPU tests check that
// sweeps using it agree bit for bit with sweeps using the hardware
// conversion.
#pragma once
#include <cstdint>
#include <cstring>

#if defined(__CUDACC__)
#define FIXCONV_FN __host__ __device__ __forceinline__
#else
#define FIXCONV_FN inline
#endif

namespace fixconv {

FIXCONV_FN uint64_t bits_of(double x) {
#if defined(__CUDA_ARCH__)
  return (uint64_t)__double_as_longlong(x);
#else
  uint64_t b;
  std::memcpy(&b, &x, sizeof b);
  return b;
#endif
}

// y in [0, 2^63) (finite) to the nearest integer, ties to even
FIXCONV_FN int64_t f64_to_i64_rn(double y) {
  const uint64_t b = bits_of(y);
  const int ex = (int)(b >> 52);       // biased exponent (the sign bit is 0)
  if (ex < 1022) return 0;             // y < 0.5
  const uint64_t sig = (b & ((1ull << 52) - 1)) | (1ull << 52);
  const int sh = 1075 - ex;            // fraction bits of sig: 52 - (ex - 1023)
  if (sh <= 0) return (int64_t)(sig << -sh);   // already an integer
  const uint64_t q = sig >> sh;        // sh in [1, 53]
  const uint64_t rem = sig & ((1ull << sh) - 1);
  const uint64_t half = 1ull << (sh - 1);
  return (int64_t)(q + ((rem > half || (rem == half && (q & 1ull))) ? 1ull : 0ull));
}

}  // namespace fixconv
