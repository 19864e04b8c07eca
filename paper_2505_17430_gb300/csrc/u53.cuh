// u53.cuh -- the double m * 2^-53 of a 53-bit integer m, built from integer
// operations only.  m < 2^53 is exactly representable, so the value is the
// same as a (rounding-free) integer-to-double conversion followed by the
// exact scaling by 2^-53; on this GPU that conversion and the scaling run on
// the FP64 pipe, which the DE/PSO operators already saturate, while these
// operations run on the integer pipe.  For m > 0 with leading bit L (0..52):
// m * 2^-53 = (1 + f) * 2^(L - 53), so the biased exponent is L - 53 + 1023
// and the 52 fraction bits are m shifted left by 52 - L with the leading bit
// dropped.
#pragma once
#include <stdint.h>
#include <string.h>

#ifdef __CUDACC__
#define SV_U53_FN __host__ __device__ __forceinline__
#else
#define SV_U53_FN static inline
#endif

SV_U53_FN double sv_u53_of(uint64_t m) {
#ifdef __CUDA_ARCH__
  const int L = 63 - __clzll((long long)m);
#else
  const int L = m ? 63 - __builtin_clzll(m) : -1;
#endif
  const uint64_t frac = (m << ((52 - L) & 63)) & 0x000FFFFFFFFFFFFFull;
  const uint64_t bits = m ? (((uint64_t)(L + 970) << 52) | frac) : 0ull;
#ifdef __CUDA_ARCH__
  return __longlong_as_double((long long)bits);
#else
  double d;
  memcpy(&d, &bits, sizeof d);
  return d;
#endif
}
