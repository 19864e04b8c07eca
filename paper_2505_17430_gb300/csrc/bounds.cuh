// bounds.cuh -- IEEE comparisons of a double against a box bound (x < b,
// x > b; NaN compares false, -0 equals +0) built from 32-bit integer
// instructions on the two halves of the encodings.  The trial repair and the
// PSO / CSO clamps test every coordinate against lb and ub; done as FP64
// compares (or as 64-bit integer keys, which cost the same here) the two
// tests took about as many FP64-pipe instructions as the update itself, and
// the FP64 pipe is what bounds these kernels on GB300.
//
// Sign-magnitude order: for x and b of different signs, x < b exactly when
// x is the negative one, unless both are zeros; for equal signs the
// magnitudes (high word without the sign, then the low word, unsigned)
// decide, reversed for negatives.  A NaN on either side (exponent all ones,
// nonzero significand) makes the comparison false.
//
// The header also compiles as plain C++ (host), so that the comparison can be
// checked against the compiler's own double compares on the CPU.
#pragma once
#include <stdint.h>
#include <string.h>

#ifdef __CUDACC__
#define SV_BOUND_FN __host__ __device__ __forceinline__
#else
#define SV_BOUND_FN static inline
#endif

struct SvBound {
  int32_t hi;       // high word of b (sign, exponent, top of the significand)
  uint32_t lo;      // low word of b
  uint32_t mag_hi;  // hi without the sign bit
  int32_t zero;     // b is +0 or -0
  int32_t nan;      // b is a NaN (every comparison is then false)
};

SV_BOUND_FN void sv_words(double x, int32_t& hi, uint32_t& lo) {
#ifdef __CUDA_ARCH__
  hi = __double2hiint(x);
  lo = (uint32_t)__double2loint(x);
#else
  uint64_t b;
  memcpy(&b, &x, 8);
  hi = (int32_t)(uint32_t)(b >> 32);
  lo = (uint32_t)b;
#endif
}

SV_BOUND_FN SvBound sv_bound(double b) {
  SvBound r;
  sv_words(b, r.hi, r.lo);
  r.mag_hi = (uint32_t)r.hi & 0x7FFFFFFFu;
  r.zero = (r.mag_hi | r.lo) == 0u;
  r.nan = r.mag_hi > 0x7FF00000u || (r.mag_hi == 0x7FF00000u && r.lo != 0u);
  return r;
}

// x < b
SV_BOUND_FN bool sv_lt_bound(double x, const SvBound& b) {
  int32_t hx;
  uint32_t lx;
  sv_words(x, hx, lx);
  const uint32_t ax = (uint32_t)hx & 0x7FFFFFFFu;
  const bool nan = ax > 0x7FF00000u || (ax == 0x7FF00000u && lx != 0u);
  const bool zeros = ((ax | lx) == 0u) && b.zero;
  const bool sx = hx < 0, sb = b.hi < 0;
  const bool mlt = ax < b.mag_hi || (ax == b.mag_hi && lx < b.lo);  // |x| < |b|
  const bool mgt = ax > b.mag_hi || (ax == b.mag_hi && lx > b.lo);  // |x| > |b|
  const bool r = (sx != sb) ? (sx && !zeros) : (sx ? mgt : mlt);
  return r && !nan && !b.nan;
}

// x > b
SV_BOUND_FN bool sv_gt_bound(double x, const SvBound& b) {
  int32_t hx;
  uint32_t lx;
  sv_words(x, hx, lx);
  const uint32_t ax = (uint32_t)hx & 0x7FFFFFFFu;
  const bool nan = ax > 0x7FF00000u || (ax == 0x7FF00000u && lx != 0u);
  const bool zeros = ((ax | lx) == 0u) && b.zero;
  const bool sx = hx < 0, sb = b.hi < 0;
  const bool mlt = ax < b.mag_hi || (ax == b.mag_hi && lx < b.lo);
  const bool mgt = ax > b.mag_hi || (ax == b.mag_hi && lx > b.lo);
  const bool r = (sx != sb) ? (sb && !zeros) : (sx ? mlt : mgt);
  return r && !nan && !b.nan;
}
