// sevo_internal.cuh -- types and helpers shared by the library's translation
// units (host and device).  Nothing here is shared with the CPU oracle.
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>

#include "../../include/sevo.h"
#include "u53.cuh"

#define SV_MAXG SEVO_MAX_GROUPS
#define SV_MAXC SEVO_MAX_COMPONENTS

// Philox purposes: high byte of counter word 3 (the low 24 bits carry a salt,
// the component index for instance data).
enum : uint32_t {
  SV_P_INIT = 1, SV_P_PART = 2, SV_P_CROSS = 3, SV_P_ARCH = 4, SV_P_PSO = 5, SV_P_SHADE = 6, SV_P_CSO = 7,
  SV_P_SHIFT = 16, SV_P_ROT = 17, SV_P_PERM = 18, SV_P_HYB = 19, SV_P_COMP = 20
};

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon et al., SC'11): 10 rounds; each round multiplies
// words 0 and 2 by 0xD2511F53 / 0xCD9E8D57 (64-bit products split hi/lo),
// xors the high halves into words 1 and 3 with the key, and the key advances
// by 0x9E3779B9 / 0xBB67AE85 after every round.
// ---------------------------------------------------------------------------
__host__ __device__ __forceinline__ uint32_t sv_mulhi(uint32_t a, uint32_t b) {
#ifdef __CUDA_ARCH__
  return __umulhi(a, b);
#else
  return (uint32_t)(((uint64_t)a * b) >> 32);
#endif
}

__host__ __device__ __forceinline__ uint4 sv_philox(uint4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint32_t lo0 = 0xD2511F53u * c.x, hi0 = sv_mulhi(0xD2511F53u, c.x);
    const uint32_t lo1 = 0xCD9E8D57u * c.z, hi1 = sv_mulhi(0xCD9E8D57u, c.z);
    c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
  return c;
}

// draw(seed; c0, c1, c2, purpose, salt)
__host__ __device__ __forceinline__ uint4 sv_draw(uint64_t seed, uint32_t c0, uint32_t c1,
                                                  uint32_t c2, uint32_t purpose,
                                                  uint32_t salt = 0) {
  return sv_philox(make_uint4(c0, c1, c2, (purpose << 24) | (salt & 0xFFFFFFu)),
                   (uint32_t)seed, (uint32_t)(seed >> 32));
}

// 53-bit uniform in [0,1) from two words (27 + 26 high bits), exact.
__host__ __device__ __forceinline__ double sv_u53(uint32_t w0, uint32_t w1) {
  const uint64_t m = ((uint64_t)(w0 >> 5) << 26) | (uint64_t)(w1 >> 6);
#ifdef __CUDA_ARCH__
  return sv_u53_of(m);  // integer operations only (u53.cuh)
#else
  return (double)m * 0x1p-53;
#endif
}

// integer in [0,n): high word of w*n
__host__ __device__ __forceinline__ uint32_t sv_below(uint32_t w, uint32_t n) {
  return sv_mulhi(w, n);
}

// ---------------------------------------------------------------------------
// Device-resident instance descriptor.  A single-family instance is one
// component with one group; a hybrid is one component with K groups; a
// composition is Nc components of one group each; a composition of hybrids is
// Nc components of K_c groups each.  Groups are contiguous ranges of the
// (permuted) output coordinates of their component.
// ---------------------------------------------------------------------------
struct ProblemDev {
  int32_t family, D, ncomp;
  int32_t weighted;  // composition kinds: component values are weighted (compose)
  int32_t kpad;   // K (input) extent padded for the tensor-core operands
  int32_t npad;   // N (output) extent padded for the tensor-core operands
  double fstar;
  double sch_s, sch_c;                  // Schwefel shift s and c = s sin sqrt s
  float sch_s32, sch_B32, sch_sinB32, sch_cosB32, sch_h032, sch_c32;
  const double* o[SV_MAXC];             // D
  const double* MT64[SV_MAXC];          // D x D, MT[j*D+i] = M_ij
  const float* MT32[SV_MAXC];           // D x D, FP32 copy of MT
  const float* M32[SV_MAXC];            // npad x kpad row-major, TF32-rounded, zero pad
  const __nv_bfloat16* Mhi[SV_MAXC];    // npad x kpad
  const __nv_bfloat16* Mlo[SV_MAXC];    // npad x kpad
  const double* aux64[SV_MAXC];         // D: ellipsoid coefficient or sqrt(position)
  const float* aux32[SV_MAXC];
  const int32_t* gid[SV_MAXC];          // D: group index of output coordinate i
  const CUtensorMap* tmap32[SV_MAXC];   // device copies of the TMA descriptors
  const CUtensorMap* tmaphi[SV_MAXC];
  const CUtensorMap* tmaplo[SV_MAXC];
  const CUtensorMap* tmap32h[SV_MAXC];  // the same with 64-row boxes (D > 128)
  const CUtensorMap* tmaphih[SV_MAXC];
  const CUtensorMap* tmaploh[SV_MAXC];
  const float* oh32[SV_MAXC];           // D: o split as oh + ol (see sv_split_hi_lo)
  const float* ol32[SV_MAXC];
  int32_t ngc[SV_MAXC];                 // groups of component c
  int32_t gstart[SV_MAXC][SV_MAXG + 1]; // component c's group ranges
  int32_t gbody[SV_MAXC][SV_MAXG];      // component c's group bodies
  double sigma[SV_MAXC], lambda[SV_MAXC], bias[SV_MAXC];
};

struct sevo_problem {
  int32_t family, D, ncomp, ngroups, device;
  double fstar;
  // host copies
  double* o_h;      // ncomp x D
  double* M_h;      // ncomp x D x D (row-major; hybrid rows permuted)
  int32_t* perm_h;  // D (hybrid), ncomp x D (composition of hybrids)
  int32_t gsize[SV_MAXG], gbody[SV_MAXG];   // hybrid groups
  int32_t cbody[SV_MAXC];                    // composition component bodies
  int32_t cK[SV_MAXC];                       // composition of hybrids: groups,
  int32_t cgsize[SV_MAXC][SV_MAXG], cgbody[SV_MAXC][SV_MAXG];  // sizes, bodies
  double sigma[SV_MAXC], lambda[SV_MAXC], bias[SV_MAXC];
  // device
  ProblemDev host_desc;   // descriptor with device pointers (host copy)
  ProblemDev* desc_d;     // same, in device memory
  void* dev_block;        // one allocation holding all device arrays
  size_t dev_bytes;
  // TMA descriptors of the padded rotation operands (built on first use)
  bool tmaps_ready;
  CUtensorMap tmap_f32[SV_MAXC];   // M32: npad x kpad fp32, box (32, rows)
  CUtensorMap tmap_hi[SV_MAXC];    // Mhi: npad x kpad bf16, box (64, rows)
  CUtensorMap tmap_lo[SV_MAXC];
  CUtensorMap tmap_f32h[SV_MAXC];  // 64-row boxes (D > 128: 64-column GEMM tiles)
  CUtensorMap tmap_hih[SV_MAXC];
  CUtensorMap tmap_loh[SV_MAXC];
  int32_t tmap_rows;               // box rows used when the maps were built
};

// Split a double into float hi + lo with integer operations only:
// hi = x with the significand truncated to 24 bits (exact as a float),
// lo = the remaining low 29 significand bits, rounded to a float.  For
// |x| < 2^-74 both are 0 (such x are 0 to any precision the mixed path
// uses).  Used for x and for the shift o alike, so x == o gives hi == oh and
// lo == ol exactly.
__host__ __device__ __forceinline__ void sv_split_hi_lo(double x, float& hi, float& lo) {
#ifdef __CUDA_ARCH__
  const long long b = __double_as_longlong(x);
#else
  long long b;
  __builtin_memcpy(&b, &x, 8);
#endif
  const uint32_t h = (uint32_t)((unsigned long long)b >> 32), l = (uint32_t)b;
  const int e = (int)((h >> 20) & 0x7FF);
  // branch-free: the bits are formed for every input and replaced by 0 when
  // |x| < 2^-74 (or beyond the float range, which the callers never pass)
  const bool ok = (e >= 949) && (e <= 1150);
  const uint32_t sign = h & 0x80000000u;
  const uint32_t hb = sign | ((uint32_t)(e - 896) << 23) | ((h & 0xFFFFFu) << 3) | (l >> 29);
  const uint32_t r = l & 0x1FFFFFFFu;
  const uint32_t sb = (uint32_t)(e - 948) << 23;  // 2^(e - 1075) as float bits
#ifdef __CUDA_ARCH__
  const float hv = __uint_as_float(hb);
  const float v = __fmul_rn(__uint2float_rn(r), __uint_as_float(sb));
#else
  float hv, scl;
  __builtin_memcpy(&hv, &hb, 4);
  __builtin_memcpy(&scl, &sb, 4);
  const float v = (float)r * scl;
#endif
  hi = ok ? hv : 0.f;
  lo = ok ? (sign ? -v : v) : 0.f;
}

#ifdef __CUDACC__
// One coordinate of the tensor-core operand: d = x - o, formed from the
// float hi/lo splits of x and of o (oh, ol) as (xh - oh) + (xl - ol) in
// round-to-nearest FP32 (no contraction).  The fused evaluation's producers
// and the operators that hand their rows to it both call this, so the operand
// has the same bits whichever forms it.
__device__ __forceinline__ float sv_operand_d(double x, float oh, float ol) {
  float xh, xl;
  sv_split_hi_lo(x, xh, xl);
  return __fadd_rn(__fsub_rn(xh, oh), __fsub_rn(xl, ol));
}
#endif

// status helpers --------------------------------------------------------
#define SV_CUDA(call)                                     \
  do {                                                    \
    cudaError_t _e = (call);                              \
    if (_e != cudaSuccess) {                              \
      sv_set_last_cuda_error(_e);                         \
      return _e == cudaErrorMemoryAllocation ? SEVO_ERR_OOM : SEVO_ERR_CUDA; \
    }                                                     \
  } while (0)

void sv_set_last_cuda_error(cudaError_t e);
// kernel launch accounting (see sevo_kernel_launches)
void sv_note_launch(int64_t n = 1);
// kernel tracing: a token from sv_trace_begin (before the launch; -1 when
// tracing is off or the stream is capturing) is closed by sv_trace_end
// (after the launch), which also counts the launch
int sv_trace_begin(int kind, cudaStream_t st);
void sv_trace_end(int token, cudaStream_t st);
// upload the instance to the current device on first use (thread-safe);
// SEVO_ERR_STATE if it already lives on another device
int32_t sv_problem_ready(const sevo_problem* p);
// SEVO_OK if p's device copy exists on device dev (read under the lock that
// guards its upload), else SEVO_ERR_STATE
int32_t sv_problem_has_device_copy(const sevo_problem* p, int dev);
// composition kinds: the row error is a distance-weighted sum of components
inline bool sv_weighted_family(int f) { return f == SEVO_COMPOSITION || f == SEVO_COMP_HYBRID; }

// error flags set by device code (bitmask in a device word)
enum : uint32_t { SV_DEVERR_TIMEOUT = 1u, SV_DEVERR_BOUNDS = 2u, SV_DEVERR_NAN = 4u };
