// bodies.cuh -- per-coordinate terms and per-group finalisation of the six
// function bodies.  Every body is bias-free (g(0) = 0 exactly; f = g + f*).
//
// A group's value is built from three per-row accumulators (a0, a1, a2):
//   ellipsoid  a0 = sum c_p z^2            (c_p = 10^{6(p-1)/(n-1)}, table)
//   rosenbrock a0 = sum_{p<n} term(z_p, z_{p+1})
//   rastrigin  a0 = sum term(z)
//   schwefel   a0 = sum term(z)
//   ackley     a0 = sum z^2, a1 = sum cos(2 pi z)        [FP64]
//                                a1 = sum sin^2(pi z)       [FP32]
//   griewank   a0 = sum z^2, a1 = prod cos(z/sqrt p)     [FP64]
//                                a1 = sum log|cos|, a2 = #negative cos [FP32]
// Slot combine rules: sum, except FP64 griewank a1 (product).
#pragma once
#include "sevo_internal.cuh"

#define SV_TWO_PI 6.28318530717958647692
#define SV_E 2.71828182845904523536

// ------------------------------------------------------------------ FP64
// Plain textbook forms, term for term the same expressions as the
// definitions (the FP64 path is compared with the oracle at 1e-12 rel).
struct Acc64 {
  double a0, a1, a2;
};

__device__ __forceinline__ void acc64_init(int body, Acc64& a) {
  a.a0 = 0.0;
  a.a1 = (body == SEVO_GRIEWANK) ? 1.0 : 0.0;
  a.a2 = 0.0;
}

__device__ __forceinline__ bool slot1_is_product64(int body) { return body == SEVO_GRIEWANK; }

// one coordinate's contribution; aux = ellipsoid coefficient or sqrt(p);
// has_next/znext: Rosenbrock pairs stay inside a group
__device__ __forceinline__ void term64(int body, double z, double aux, bool has_next,
                                       double znext, const ProblemDev& P, Acc64& a) {
  switch (body) {
    case SEVO_ELLIPSOID:
      a.a0 += aux * z * z;
      break;
    case SEVO_ROSENBROCK:
      if (has_next) {
        double yi = z + 1.0, yn = znext + 1.0;
        double u = yi * yi - yn, v = yi - 1.0;
        a.a0 += 100.0 * u * u + v * v;
      }
      break;
    case SEVO_RASTRIGIN:
      a.a0 += z * z - 10.0 * cos(SV_TWO_PI * z) + 10.0;
      break;
    case SEVO_SCHWEFEL: {
      double y = z + P.sch_s, ay = fabs(y);
      // the product is rounded on its own (no fused multiply-add), as in
      // c = s sin sqrt s, so the term is exactly 0 at z = 0
      if (ay <= 500.0) {
        a.a0 += P.sch_c - __dmul_rn(y, sin(sqrt(ay)));
      } else {
        double b = (y > 0.0) ? 500.0 : -500.0;
        a.a0 += P.sch_c - __dmul_rn(b, sin(sqrt(500.0))) + 1e-4 * (ay - 500.0) * (ay - 500.0);
      }
      break;
    }
    case SEVO_ACKLEY:
      a.a0 += z * z;
      a.a1 += cos(SV_TWO_PI * z);
      break;
    case SEVO_GRIEWANK:
      a.a0 += z * z;
      a.a1 *= cos(z / aux);
      break;
  }
}

__device__ __forceinline__ double finalize64(int body, const Acc64& a, int n) {
  if (n <= 0) return 0.0;
  switch (body) {
    case SEVO_ACKLEY: {
      double ea = exp(-0.2 * sqrt(a.a0 / (double)n));
      double eb = exp(a.a1 / (double)n);
      return (20.0 - 20.0 * ea) + (exp(1.0) - eb);
    }
    case SEVO_GRIEWANK:
      return a.a0 / 4000.0 + (1.0 - a.a1);
    default:
      return a.a0;
  }
}

// ------------------------------------------------------------------ FP32
// Algebraically equal forms without catastrophic cancellation near z = 0,
// so that errors near the 1e-4 refinement threshold are resolved in FP32:
//   rastrigin  z^2 - 10 cos 2 pi z + 10 = z^2 + 20 sin^2(pi z)
//   rosenbrock (z+1)^2 - (z'+1) = z^2 + 2z - z';  (y-1)^2 = z^2
//   ackley     20(1 - e^{-0.2 r}) + e(1 - e^{-2 sum sin^2(pi z)/n})  via expm1
//   griewank   1 - prod cos(z/sqrt p) = -expm1(sum log cos), log cos x =
//              log1p(-2 sin^2(x/2)), sign tracked for negative cosines
//   schwefel   c - (s+t) sin sqrt(s+t) expanded around the optimum (t = z,
//              B = sqrt s, A = sqrt(s+t), d = A - B = t/(A+B), c = s sin B):
//              sin A = sin B cos d + cos B sin d, cos d = 1 - 2 sin^2(d/2),
//              sin d = d + (sin d - d), so with s + t = A^2
//                c - A^2 sin A = A^2 sin B 2 sin^2(d/2)
//                              - A^2 cos B (sin d - d)
//                              - t sin B - A^2 d cos B.
//              Writing -t sin B = t (B/2) cos B - t h0 with h0 = sin B +
//              (B/2) cos B (zero at the exact argmax, its FP32 residual
//              kept) and using B(A+B) - 2A^2 = -(2A+B) d, the last two
//              pieces become -t cos B (2A+B) d / (2(A+B)) - t h0.  Every
//              piece but t h0 is second order in t and none cancels.
struct Acc32 {
  float a0, a1, a2;
};

__device__ __forceinline__ void acc32_init(Acc32& a) { a.a0 = a.a1 = a.a2 = 0.f; }

// sin(d) - d without cancellation for small |d| (Taylor to d^9)
__device__ __forceinline__ float sin_minus_x(float d) {
  const float d2 = d * d;
  const float series =
      d * d2 * (-1.f / 6.f + d2 * (1.f / 120.f + d2 * (-1.f / 5040.f + d2 * (1.f / 362880.f))));
  return (fabsf(d) < 0.25f) ? series : (sinf(d) - d);
}

__device__ __forceinline__ float schwefel_term32(float z, const ProblemDev& P) {
  const float s = P.sch_s32;
  float y = z + s;
  float ay = fabsf(y);
  if (y > 0.f && ay <= 500.f) {
    const float B = P.sch_B32, sB = P.sch_sinB32, cB = P.sch_cosB32;
    float A = sqrtf(s + z);
    float apb = A + B;
    float d = z / apb;
    float h = sinf(0.5f * d);
    float spt = s + z;
    float t1 = spt * sB * 2.f * h * h;                  // (s+t) sin B (1 - cos d)
    float t2 = -cB * spt * sin_minus_x(d);              // -(s+t) cos B (sin d - d)
    float t3 = -z * cB * (2.f * A + B) * d / (2.f * apb);
    float t4 = -z * P.sch_h032;
    return t1 + t2 + t3 + t4;
  }
  if (ay <= 500.f) return P.sch_c32 - y * sinf(sqrtf(ay));
  float b = (y > 0.f) ? 500.f : -500.f;
  float e = ay - 500.f;
  return P.sch_c32 - b * sinf(sqrtf(500.f)) + 1e-4f * e * e;
}

__device__ __forceinline__ void term32(int body, float z, float aux, bool has_next, float znext,
                                       const ProblemDev& P, Acc32& a) {
  switch (body) {
    case SEVO_ELLIPSOID:
      a.a0 += aux * z * z;
      break;
    case SEVO_ROSENBROCK:
      if (has_next) {
        float u = fmaf(z, z + 2.f, -znext);
        a.a0 += 100.f * u * u + z * z;
      }
      break;
    case SEVO_RASTRIGIN: {
      float sp = sinpif(z);
      a.a0 += z * z + 20.f * sp * sp;
      break;
    }
    case SEVO_SCHWEFEL:
      a.a0 += schwefel_term32(z, P);
      break;
    case SEVO_ACKLEY: {
      float sp = sinpif(z);
      a.a0 += z * z;
      a.a1 += sp * sp;
      break;
    }
    case SEVO_GRIEWANK: {
      float x = z / aux;
      float h = sinf(0.5f * x);
      float c = 1.f - 2.f * h * h;  // cos x
      a.a0 += z * z;
      if (c > 0.f) {
        a.a1 += log1pf(-2.f * h * h);
      } else {
        a.a1 += logf(fmaxf(-c, 1e-30f));
        a.a2 += 1.f;
      }
      break;
    }
  }
}

// Fast variant for the TF32 path (operands carry 2^-11 relative rounding, far
// above these approximations' error): sin^2(pi z) from the reduced argument
// z - rint(z) with the hardware sine, hardware sine / fast divide in
// Schwefel.  Same algebraic forms as term32.
__device__ __forceinline__ float sin_pi_red(float z) {
  const float r = z - rintf(z);  // exact for |z| < 2^23; sin^2(pi z) has period 1
  return __sinf(3.14159265358979f * r);
}

__device__ __forceinline__ float schwefel_term32f(float z, const ProblemDev& P) {
  const float s = P.sch_s32;
  const float y = z + s;
  if (fabsf(z) < 1.0f) {
    // near the optimum the term is O(z^2) next to c ~ 418: the expansion
    // around s avoids the cancellation (y > 0 and |y| <= 500 here)
    const float B = P.sch_B32, sB = P.sch_sinB32, cB = P.sch_cosB32;
    const float spt = y;
    const float A = sqrtf(spt);
    const float apb = A + B;
    const float d = __fdividef(z, apb);
    const float h = __sinf(0.5f * d);
    const float t1 = spt * sB * 2.f * h * h;
    const float t2 = -cB * spt * sin_minus_x(d);
    const float t3 = -z * cB * (2.f * A + B) * __fdividef(d, 2.f * apb);
    const float t4 = -z * P.sch_h032;
    return t1 + t2 + t3 + t4;
  }
  const float ay = fabsf(y);
  const float yc = fminf(ay, 500.f);
  const float bsgn = (y > 0.f) ? 1.f : -1.f;
  const float e = fmaxf(ay - 500.f, 0.f);
  return P.sch_c32 - bsgn * yc * __sinf(sqrtf(yc)) + 1e-4f * e * e;
}

__device__ __forceinline__ void term32f(int body, float z, float aux, bool has_next, float znext,
                                        const ProblemDev& P, Acc32& a) {
  switch (body) {
    case SEVO_RASTRIGIN: {
      float sp = sin_pi_red(z);
      a.a0 += z * z + 20.f * sp * sp;
      break;
    }
    case SEVO_SCHWEFEL:
      a.a0 += schwefel_term32f(z, P);
      break;
    case SEVO_ACKLEY: {
      float sp = sin_pi_red(z);
      a.a0 += z * z;
      a.a1 += sp * sp;
      break;
    }
    case SEVO_GRIEWANK: {
      // sin^2(x/2) has period pi in x/2: reduce before the hardware sine
      const float hx = 0.5f * __fdividef(z, aux);
      const float h = __sinf(hx - 3.14159265358979f * rintf(hx * 0.318309886183791f));
      float c = 1.f - 2.f * h * h;
      a.a0 += z * z;
      if (c > 0.f) {
        a.a1 += log1pf(-2.f * h * h);
      } else {
        a.a1 += __logf(fmaxf(-c, 1e-30f));
        a.a2 += 1.f;
      }
      break;
    }
    default:
      term32(body, z, aux, has_next, znext, P, a);
  }
}

template <bool FAST>
__device__ __forceinline__ void term32t(int body, float z, float aux, bool has_next, float znext,
                                        const ProblemDev& P, Acc32& a) {
  if (FAST)
    term32f(body, z, aux, has_next, znext, P, a);
  else
    term32(body, z, aux, has_next, znext, P, a);
}

__device__ __forceinline__ float finalize32(int body, const Acc32& a, int n) {
  if (n <= 0) return 0.f;
  switch (body) {
    case SEVO_ACKLEY: {
      float r = sqrtf(a.a0 / (float)n);
      return 20.f * (-expm1f(-0.2f * r)) + (float)SV_E * (-expm1f(-2.f * a.a1 / (float)n));
    }
    case SEVO_GRIEWANK: {
      bool neg = ((int)a.a2) & 1;
      float one_minus_prod = neg ? 1.f + expf(a.a1) : -expm1f(a.a1);
      return a.a0 / 4000.f + one_minus_prod;
    }
    default:
      return a.a0;
  }
}

// ------------------------------------------------------------------ composition
// w_c = s_c^{-1/2} exp(-s_c / (2 D sigma_c^2)); s_c = |x - o_c|^2 (FP64).
// If some s_c == 0 the weight vector is e_c (first such c); if every w_c
// underflows the weights are uniform.
__device__ __forceinline__ double compose(const ProblemDev& P, const double* s, const double* g) {
  const int nc = P.ncomp;
  int exact = -1;
  for (int c = 0; c < nc; ++c)
    if (s[c] == 0.0 && exact < 0) exact = c;
  double out = 0.0;
  if (exact >= 0) return P.lambda[exact] * g[exact] + P.bias[exact];
  double w[SV_MAXC], W = 0.0;
  for (int c = 0; c < nc; ++c) {
    double sg = P.sigma[c];
    w[c] = (1.0 / sqrt(s[c])) * exp(-s[c] / (2.0 * (double)P.D * sg * sg));
    W += w[c];
  }
  for (int c = 0; c < nc; ++c) {
    double om = (W > 0.0) ? w[c] / W : 1.0 / (double)nc;
    out += om * (P.lambda[c] * g[c] + P.bias[c]);
  }
  return out;
}
