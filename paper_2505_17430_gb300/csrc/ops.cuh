// ops.cuh -- the DE and PSO operators on one row quad / coordinate, shared
// by the operator kernels (evo.cu) and the fused evaluation's producer warps
// (eval_tc.cu), which form trial rows and moved particles in place of
// loading them: the same functions, hence the same bits, either way.
#pragma once
#include "bounds.cuh"
#include "sevo_internal.cuh"

namespace {

// exact 53-bit uniform from two Philox words (the same value as sv_u53;
// integer operations only, u53.cuh)
__device__ __forceinline__ double u53_int(uint32_t w0, uint32_t w1) { return sv_u53(w0, w1); }

// v * 0.5, exactly as IEEE multiplication rounds it, with integer
// instructions: a normal result only loses one from the exponent; when the
// result is subnormal the significand shifts right once with round to nearest
// even; zeros, infinities and NaN are returned unchanged (all exact halves).
__device__ __forceinline__ double half_exact(double v) {
  const long long b = __double_as_longlong(v);
  const long long sign = b & (long long)0x8000000000000000ull;
  const long long mag = b & 0x7FFFFFFFFFFFFFFFll;
  const int e = (int)(mag >> 52);
  if (e > 1 && e < 0x7FF) return __longlong_as_double(b - (1ll << 52));
  if (e == 0x7FF || mag == 0) return v;
  // e == 1 or subnormal: the significand with its implicit bit, halved
  const long long s = mag;  // for e == 1 the exponent bit is the implicit 1
  long long h = s >> 1;
  if ((s & 1) && (h & 1)) ++h;  // tie: round to even
  return __longlong_as_double(sign | h);
}

// four consecutive coordinates j0..j0+3 of a row (16-byte loads when the
// quad is whole: rows start 16-byte aligned and j0 is a multiple of 4)
__device__ __forceinline__ void load_quad(const double* __restrict__ row, int j0, int D,
                                          double (&v)[4]) {
  if (j0 + 3 < D) {
    const double2 a = *reinterpret_cast<const double2*>(row + j0);
    const double2 b = *reinterpret_cast<const double2*>(row + j0 + 2);
    v[0] = a.x;
    v[1] = a.y;
    v[2] = b.x;
    v[3] = b.y;
  } else {
#pragma unroll
    for (int q = 0; q < 4; ++q) v[q] = (j0 + q < D) ? row[j0 + q] : 0.0;
  }
}

// ---------------------------------------------------------------- DE trials
// one quad (coordinates 4 jq .. 4 jq + 3) of run r's trial row i, written to
// U and, when uq is given, also returned in uq[0..3] (0 past D)
template <int ALG>
__device__ __forceinline__ void de_trial_elem(const double* __restrict__ X, double* __restrict__ U,
                                              const double* __restrict__ A,
                                              const int32_t* __restrict__ asize,
                                              const int32_t* __restrict__ order,
                                              int32_t* __restrict__ part,
                                              const uint64_t* __restrict__ seeds, int NP, int D,
                                              int ld, double F, unsigned long long cr_thr,
                                              double lb, double ub, int pk,
                                              unsigned long long gen, int r, int i, int jq,
                                              const double* __restrict__ Fi = nullptr,
                                              const double* __restrict__ CRi = nullptr,
                                              const int32_t* __restrict__ kpb = nullptr,
                                              double* uq = nullptr) {
  // SHADE: this row's F, crossover threshold and pbest pool
  if (ALG == SEVO_DE_SHADE) {
    const int64_t row = (int64_t)r * NP + i;
    F = Fi[row];
    cr_thr = (unsigned long long)ceil(__dmul_rn(CRi[row], 4294967296.0));
    pk = kpb[row];
  }
  const uint64_t seed = seeds[r];
  const uint4 w = sv_draw(seed, 0u, (uint32_t)i, (uint32_t)gen, SV_P_PART);
  const double* Xr = X + (int64_t)r * NP * ld;
  const double* xi = Xr + (int64_t)i * ld;
  const double *d1, *d2, *d3;
  int p0, p1, p2, jr;
  if (ALG == SEVO_DE_RAND1) {
    int a = (int)sv_below(w.x, (uint32_t)(NP - 1));
    if (a >= i) ++a;
    const int lo = min(i, a), hi = max(i, a);
    int b = (int)sv_below(w.y, (uint32_t)(NP - 2));
    if (b >= lo) ++b;
    if (b >= hi) ++b;
    int e0 = lo, e1 = hi, e2 = b;  // sort {i, a, b}
    if (e2 < e1) {
      int tt = e1;
      e1 = e2;
      e2 = tt;
    }
    if (e1 < e0) {
      int tt = e0;
      e0 = e1;
      e1 = tt;
    }
    int c = (int)sv_below(w.z, (uint32_t)(NP - 3));
    if (c >= e0) ++c;
    if (c >= e1) ++c;
    if (c >= e2) ++c;
    p0 = a;
    p1 = b;
    p2 = c;
    d1 = Xr + (int64_t)a * ld;
    d2 = Xr + (int64_t)b * ld;
    d3 = Xr + (int64_t)c * ld;
  } else {
    const int as = (ALG == SEVO_DE_CTPB) ? asize[r] : 0;  // SHADE: no archive
    const int pb = order[(int64_t)r * NP + (int)sv_below(w.x, (uint32_t)pk)];
    int r1 = (int)sv_below(w.y, (uint32_t)(NP - 1));
    if (r1 >= i) ++r1;
    const int lo = min(i, r1), hi = max(i, r1);
    int r2 = (int)sv_below(w.z, (uint32_t)(NP + as - 2));
    if (r2 >= lo) ++r2;
    if (r2 >= hi) ++r2;
    p0 = pb;
    p1 = r1;
    p2 = r2;
    d1 = Xr + (int64_t)pb * ld;
    d2 = Xr + (int64_t)r1 * ld;
    d3 = (r2 < NP) ? Xr + (int64_t)r2 * ld : A + ((int64_t)r * NP + (r2 - NP)) * ld;
  }
  jr = (int)sv_below(w.w, (uint32_t)D);
  if (jq == 0 && part) {
    int32_t* pp = part + ((int64_t)r * NP + i) * 4;
    pp[0] = p0;
    pp[1] = p1;
    pp[2] = p2;
    pp[3] = jr;
  }
  const uint4 cw = sv_draw(seed, (uint32_t)jq, (uint32_t)i, (uint32_t)gen, SV_P_CROSS);
  const uint32_t cws[4] = {cw.x, cw.y, cw.z, cw.w};
  double* ui = U + ((int64_t)r * NP + i) * ld;
  const int j0 = jq * 4;
  double xv[4], v1[4], v2[4], v3[4];
  load_quad(xi, j0, D, xv);
  load_quad(d1, j0, D, v1);
  load_quad(d2, j0, D, v2);
  load_quad(d3, j0, D, v3);
  const SvBound lbb = sv_bound(lb), ubb = sv_bound(ub);
  if (uq) uq[0] = uq[1] = uq[2] = uq[3] = 0.0;
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int j = j0 + q;
    if (j >= D) break;
    const double x = xv[q];
    double u = x;
    if ((unsigned long long)cws[q] < cr_thr || j == jr) {
      if (ALG == SEVO_DE_RAND1)
        u = __fma_rn(F, __dsub_rn(v2[q], v3[q]), v1[q]);
      else
        u = __fma_rn(F, __dsub_rn(v2[q], v3[q]), __fma_rn(F, __dsub_rn(v1[q], x), x));
    }
    // repair: if u < lb then u = (lb + x) / 2; then if u > ub, u = (ub + x) / 2.
    // With the parent inside the bounds at most one of them applies, so one
    // FP64 add with the bound chosen by a select; the second check only
    // fires for parents outside the bounds (populations set by the caller)
    const bool lo = sv_lt_bound(u, lbb), hi = sv_gt_bound(u, ubb);
    if (lo || hi) {
      u = half_exact(__dadd_rn(lo ? lb : ub, x));
      if (lo && sv_gt_bound(u, ubb)) u = half_exact(__dadd_rn(ub, x));
    }
    ui[j] = u;
    if (uq) uq[q] = u;
  }
}

// ---------------------------------------------------------------- PSO
// coordinate j of run r's particle i (row ri = r * NP + i), element e:
// the moved position (returned) and velocity (*vn)
__device__ __forceinline__ double pso_moved(const double* __restrict__ X,
                                            const double* __restrict__ V,
                                            const double* __restrict__ P,
                                            const int32_t* __restrict__ guide,
                                            const uint64_t* __restrict__ seeds,
                                            unsigned long long gen, int NP, int ld, double w,
                                            double c1, double c2, double lb, double ub, int r,
                                            int i, int j, int64_t ri, int64_t e, double* vn) {
  const uint4 rw = sv_draw(seeds[r], (uint32_t)j, (uint32_t)i, (uint32_t)gen, SV_P_PSO);
  const double r1 = u53_int(rw.x, rw.y), r2 = u53_int(rw.z, rw.w);
  const double a = __dmul_rn(c1, r1), b = __dmul_rn(c2, r2);
  const int gi = guide[ri];
  const double x = X[e];
  const double gj = P[((int64_t)r * NP + gi) * ld + j];
  double v = __fma_rn(w, V[e], __fma_rn(a, __dsub_rn(P[e], x), __dmul_rn(b, __dsub_rn(gj, x))));
  double xn = __dadd_rn(x, v);
  if (sv_lt_bound(xn, sv_bound(lb))) {
    xn = lb;
    v = 0.0;
  }
  if (sv_gt_bound(xn, sv_bound(ub))) {
    xn = ub;
    v = 0.0;
  }
  *vn = v;
  return xn;
}

}  // namespace
