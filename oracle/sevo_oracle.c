/*
 * sevo_oracle.c -- plain FP64 CPU oracle (TEST INFRASTRUCTURE ONLY).
 *
 * Everything here is the direct, sequential statement of each step: direct
 * matrix-vector products, textbook body formulas, loops in index order.
 * No blocking, no SIMD, no reordering beyond what a definition states.
 * Shares no source with the product library or its CUDA kernels.
 *
 * Built with -ffp-contract=off so that "a*b + c" is two roundings unless the
 * definition says fma() (the DE/PSO operator readings fix where an fma is
 * used, so both sides can agree bit-for-bit on trial vectors).
 */
#include "sevo_oracle.h"

#include <math.h>
#include <pthread.h>
#include <stdlib.h>
#include <string.h>

#define ORC_PI 3.14159265358979323846
#define ORC_TWO_PI 6.28318530717958647692

/* ======================================================================
 * Philox4x32-10, from its published definition (Salmon et al., "Parallel
 * random numbers: as easy as 1, 2, 3", SC'11): ten rounds of two 32x32->64
 * multiplies with constants 0xD2511F53 / 0xCD9E8D57, key bumped by the
 * Weyl constants 0x9E3779B9 / 0xBB67AE85 between rounds.
 * ====================================================================== */
void orc_philox(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                uint32_t k0, uint32_t k1, uint32_t out[4]) {
  uint32_t c[4] = {c0, c1, c2, c3};
  uint32_t k[2] = {k0, k1};
  for (int round = 0; round < 10; ++round) {
    if (round > 0) {
      k[0] += 0x9E3779B9u;
      k[1] += 0xBB67AE85u;
    }
    uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)c[0];
    uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)c[2];
    uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    uint32_t n0 = hi1 ^ c[1] ^ k[0];
    uint32_t n2 = hi0 ^ c[3] ^ k[1];
    c[0] = n0;
    c[1] = lo1;
    c[2] = n2;
    c[3] = lo0;
  }
  out[0] = c[0];
  out[1] = c[1];
  out[2] = c[2];
  out[3] = c[3];
}

/* 53-bit uniform in [0,1): 27 high bits of w0 and 26 high bits of w1 */
double orc_u53(uint32_t w0, uint32_t w1) {
  uint64_t a = w0 >> 5, b = w1 >> 6;
  return ((double)a * 67108864.0 + (double)b) * (1.0 / 9007199254740992.0);
}

/* integer in [0,n): high word of the 64-bit product w*n */
uint32_t orc_below(uint32_t w, uint32_t n) {
  return (uint32_t)(((uint64_t)w * (uint64_t)n) >> 32);
}

static void draw(uint64_t seed, uint32_t c0, uint32_t c1, uint32_t c2,
                 uint32_t purpose, uint32_t salt, uint32_t out[4]) {
  orc_philox(c0, c1, c2, (purpose << 24) | (salt & 0xFFFFFFu),
             (uint32_t)seed, (uint32_t)(seed >> 32), out);
}

/* ======================================================================
 * Bodies (plain FP64 forms; all bias-free, g(0) = 0 exactly).
 * ====================================================================== */

/* Schwefel shift s = argmax_{t in [0,500]} t*sin(sqrt t), by Newton on
 * h(u) = sin u + (u/2) cos u (u = sqrt t), the stationarity condition. */
static double g_schwefel_s;
static pthread_once_t g_schwefel_once = PTHREAD_ONCE_INIT;
static void schwefel_s_init(void) {
  double u = 20.5;
  for (int it = 0; it < 60; ++it) {
    double h = sin(u) + 0.5 * u * cos(u);
    double dh = 1.5 * cos(u) - 0.5 * u * sin(u);
    double step = h / dh;
    u -= step;
    if (fabs(step) < 1e-15) break;
  }
  g_schwefel_s = u * u;
}
static double schwefel_s(void) {
  pthread_once(&g_schwefel_once, schwefel_s_init);
  return g_schwefel_s;
}

static double schwefel_term(double z, double s, double c) {
  double y = z + s;
  double ay = fabs(y);
  if (ay <= 500.0) return c - y * sin(sqrt(ay));
  double b = (y > 0.0) ? 500.0 : -500.0;
  return c - b * sin(sqrt(500.0)) + 1e-4 * (ay - 500.0) * (ay - 500.0);
}

static double body_impl(int family, const double* z, int n) {
  double g = 0.0;
  if (n <= 0) return 0.0;
  switch (family) {
    case ORC_ELLIPSOID:
      for (int i = 1; i <= n; ++i) {
        double coef = (n > 1) ? pow(10.0, 6.0 * (double)(i - 1) / (double)(n - 1)) : 1.0;
        g += coef * z[i - 1] * z[i - 1];
      }
      break;
    case ORC_ROSENBROCK:
      for (int i = 0; i + 1 < n; ++i) {
        double yi = z[i] + 1.0, yn = z[i + 1] + 1.0;
        double a = yi * yi - yn, b = yi - 1.0;
        g += 100.0 * a * a + b * b;
      }
      break;
    case ORC_RASTRIGIN:
      for (int i = 0; i < n; ++i) {
        double cz = cos(ORC_TWO_PI * z[i]);
        g += z[i] * z[i] - 10.0 * cz + 10.0;
      }
      break;
    case ORC_SCHWEFEL: {
      double s = schwefel_s();
      double c = s * sin(sqrt(s));
      for (int i = 0; i < n; ++i) g += schwefel_term(z[i], s, c);
      break;
    }
    case ORC_ACKLEY: {
      double sq = 0.0, sc = 0.0;
      for (int i = 0; i < n; ++i) {
        sq += z[i] * z[i];
        sc += cos(ORC_TWO_PI * z[i]);
      }
      double a = exp(-0.2 * sqrt(sq / (double)n));
      double b = exp(sc / (double)n);
      double e = exp(1.0);
      g = (20.0 - 20.0 * a) + (e - b);
      break;
    }
    case ORC_GRIEWANK: {
      double sq = 0.0, pr = 1.0;
      for (int i = 1; i <= n; ++i) {
        sq += z[i - 1] * z[i - 1];
        pr *= cos(z[i - 1] / sqrt((double)i));
      }
      g = sq / 4000.0 + (1.0 - pr);
      break;
    }
    default:
      g = NAN;
  }
  return g;
}

/* ======================================================================
 * Rounding-error bound of the plain FP64 evaluation (used only to state
 * parity tolerances; not part of any definition).
 *
 * Linearised running-error analysis: every rounded intermediate r of the
 * plain form contributes |dg/dr| * |r| * (its relative error).  The sums
 * below are in units of u = 2^-53 and count two implementations of the same
 * form (this oracle and any other), each IEEE operation <= u on either side
 * (weight B_OP = 2), each libm / device transcendental <= 1 ulp on the host
 * plus 2 ulp on a GPU (weight B_TR = 6); a sum of n terms adds n * sum|t|
 * per side in any summation order.  The rotation enters through
 *   G  = sum_i |dg/dz_i| * za_i,   za_i = sum_j |M_ij d_j|
 *   Gd = sum_i |dg/dz_i| * ||d||_2
 * (an error dz_i <= a * za_i + b * ||d||_2 in z moves g by at most
 * a * G + b * Gd to first order), with the true derivative of each body.
 * ====================================================================== */
#define B_OP 2.0
#define B_TR 6.0

typedef struct {
  double E, G, Gd;
} orc_bnd;

/* one body over n coordinates of z (za per coordinate, dn = ||d||_2) */
static void body_bound(int family, const double* z, const double* za, double dn, int n,
                       orc_bnd* out) {
  double E = 0.0, G = 0.0, Gn = 0.0, T = 0.0;
  if (n <= 0) return;
  double* gi = (double*)calloc((size_t)n, sizeof(double));
  switch (family) {
    case ORC_ELLIPSOID:
      for (int i = 1; i <= n; ++i) {
        double coef = (n > 1) ? pow(10.0, 6.0 * (double)(i - 1) / (double)(n - 1)) : 1.0;
        double t = coef * z[i - 1] * z[i - 1];
        gi[i - 1] = 2.0 * coef * z[i - 1];
        E += B_OP * 2.0 * t + B_TR * t; /* z*z, coef*(.), the coefficient (pow) */
        T += t;
      }
      break;
    case ORC_ROSENBROCK:
      for (int i = 0; i + 1 < n; ++i) {
        double yi = z[i] + 1.0, yn = z[i + 1] + 1.0;
        double a = yi * yi - yn, b = yi - 1.0;
        double t = 100.0 * a * a + b * b;
        gi[i] += 400.0 * a * yi + 2.0 * b;
        gi[i + 1] += -200.0 * a;
        /* yi*yi, -yn, a*a, 100*(.), yi-1, b*b, the sum */
        E += B_OP * (200.0 * fabs(a) * yi * yi + 200.0 * a * a + 200.0 * a * a +
                     2.0 * b * b + b * b + t);
        T += t;
      }
      for (int i = 0; i < n; ++i) E += B_OP * fabs(gi[i]) * fabs(z[i] + 1.0); /* y = z + 1 */
      break;
    case ORC_RASTRIGIN:
      for (int i = 0; i < n; ++i) {
        double w = ORC_TWO_PI * z[i], cz = cos(w), sz = sin(w);
        double t = z[i] * z[i] - 10.0 * cz + 10.0;
        gi[i] = 2.0 * z[i] + 10.0 * ORC_TWO_PI * sz;
        /* z*z, 2 pi z, 10*cos, z^2 - 10 cos, + 10; the cosine */
        E += B_OP * (z[i] * z[i] + 10.0 * fabs(sz * w) + 10.0 * fabs(cz) +
                     fabs(z[i] * z[i] - 10.0 * cz) + fabs(t)) +
             B_TR * 10.0 * fabs(cz);
        T += fabs(t);
      }
      break;
    case ORC_SCHWEFEL: {
      double s = schwefel_s();
      double c = s * sin(sqrt(s));
      for (int i = 0; i < n; ++i) {
        double y = z[i] + s, ay = fabs(y), t;
        if (ay <= 500.0) {
          double r = sqrt(ay), sr = sin(r), cr = cos(r), v = y * sr;
          t = c - v;
          gi[i] = -(sr + 0.5 * r * cr);
          /* y = z + s and the shift s itself, sqrt, y*sin, c - v; the sine;
           * c = s sin sqrt s (its product and its host sine, <= 1 ulp each
           * side; first order in s vanishes at the argmax) */
          E += B_OP * (2.0 * fabs(gi[i]) * ay + fabs(y * cr) * r + fabs(v) + fabs(t) +
                       3.0 * fabs(c)) +
               B_TR * fabs(v);
        } else {
          double b = (y > 0.0) ? 500.0 : -500.0, q = ay - 500.0;
          double vb = b * sin(sqrt(500.0)), pen = 1e-4 * q * q;
          t = c - vb + pen;
          gi[i] = ((y > 0.0) ? 2e-4 : -2e-4) * q;
          /* y and s, |y| - 500, q*q, 1e-4*(.), sqrt 500 and b*sin, c - vb, + pen, c; the sine */
          E += B_OP * (2.0 * fabs(gi[i]) * ay + 2e-4 * q * q + 2.0 * pen +
                       fabs(vb) * (1.0 + 0.5 * sqrt(500.0)) + fabs(c - vb) + fabs(t) +
                       3.0 * fabs(c)) +
               B_TR * fabs(vb);
        }
        T += fabs(t);
      }
      break;
    }
    case ORC_ACKLEY: {
      double sq = 0.0, sc = 0.0, asc = 0.0, arg = 0.0;
      for (int i = 0; i < n; ++i) {
        double w = ORC_TWO_PI * z[i];
        sq += z[i] * z[i];
        sc += cos(w);
        asc += fabs(cos(w));
        arg += fabs(sin(w) * w);
      }
      double r = sqrt(sq / (double)n);
      double a = exp(-0.2 * r), b = exp(sc / (double)n), e = exp(1.0);
      double g = (20.0 - 20.0 * a) + (e - b);
      for (int i = 0; i < n; ++i) {
        /* 4a z_i / (n r) is bounded by 4a / sqrt(n) (the Lipschitz constant of
         * the norm), which also covers the cone point r = 0 */
        double da = (sq > 0.0) ? 4.0 * a * fabs(z[i]) / sqrt((double)n * sq) : 4.0 * a / sqrt((double)n);
        gi[i] = da + b * ORC_TWO_PI * fabs(sin(ORC_TWO_PI * z[i])) / (double)n;
      }
      /* sum of squares (n + 1 roundings, relative), /n, sqrt, *0.2 each
       * relative on r (dg/dr = 4a; the sum's share halved by the sqrt);
       * exp and 20*a; 20 - 20a; cos arguments and values, their sum, /n, exp;
       * e = exp(1); e - b; the final add */
      E += B_OP * (4.0 * a * r * (0.5 * (double)(n + 2) + 2.0) + 20.0 * a + fabs(20.0 - 20.0 * a)) +
           B_TR * 20.0 * a;
      E += B_OP * (b * arg / (double)n + b * asc + b * fabs(sc / (double)n) + fabs(e - b) + fabs(g)) +
           B_TR * (b * asc / (double)n + b + e);
      break;
    }
    case ORC_GRIEWANK: {
      double sq = 0.0, pr = 1.0, arg = 0.0;
      for (int i = 1; i <= n; ++i) {
        double xi = z[i - 1] / sqrt((double)i);
        sq += z[i - 1] * z[i - 1];
        pr *= cos(xi);
        arg += fabs(sin(xi) * xi);
        /* |prod_{k != i} cos| <= 1 */
        gi[i - 1] = z[i - 1] / 2000.0 + fabs(sin(xi)) / sqrt((double)i);
      }
      double g = sq / 4000.0 + (1.0 - pr);
      /* z^2 sum, /4000; the cosine arguments (sqrt, division); each factor
       * and product rounding (relative on pr); 1 - pr; the final add */
      E += B_OP * ((double)(n + 2) * sq / 4000.0 + 2.0 * arg + (double)n * fabs(pr) +
                   fabs(1.0 - pr) + fabs(g)) +
           B_TR * (double)n * fabs(pr);
      break;
    }
    default:
      E = NAN;
  }
  E += B_OP * (double)n * T; /* the coordinate sum, any order */
  for (int i = 0; i < n; ++i) {
    G += fabs(gi[i]) * za[i];
    Gn += fabs(gi[i]);
  }
  free(gi);
  out->E += E;
  out->G += G;
  out->Gd += Gn * dn;
}

double orc_body(int family, const double* z, int n) {
  return body_impl(family, z, n);
}

/* ======================================================================
 * Instances: shift o ~ U[-80,80]^D, rotation M = Q of a Householder QR of a
 * seeded Gaussian D x D matrix with diag(R) > 0; hybrid permutation and
 * groups; composition components.
 * ====================================================================== */
struct orc_problem {
  int family, D, K;     /* K: hybrid groups or composition components */
  double fstar;
  double* o;            /* K_o * D  (K_o = Nc for composition, else 1) */
  double* M;            /* K_o * D * D, row-major, hybrid rows permuted */
  int* perm;            /* hybrid: D */
  int* gsize;           /* hybrid: K */
  int* gbody;           /* hybrid: K, composition: Nc */
  double* sigma;        /* composition */
  double* lambda;
  double* bias;
  int* cK;              /* composition of hybrids: groups per component (Nc) */
  int* cgsize;          /* Nc x 8 group sizes */
  int* cgbody;          /* Nc x 8 group bodies */
  int* cperm;           /* Nc x D permutations */
};

static void gen_shift(uint64_t seed, int D, int comp, double* o) {
  uint32_t w[4];
  for (int j = 0; j < D; ++j) {
    draw(seed, (uint32_t)(j >> 1), 0, (uint32_t)D, ORC_P_SHIFT, (uint32_t)comp, w);
    int pr = j & 1;
    double u = orc_u53(w[2 * pr], w[2 * pr + 1]);
    o[j] = -80.0 + 160.0 * u;
  }
}

/* Gaussian entry e = r*D + k by Box-Muller on (u1,u2) of one Philox call */
static void gen_gauss(uint64_t seed, int D, int comp, double* G) {
  uint32_t w[4];
  int64_t n = (int64_t)D * D;
  for (int64_t e = 0; e < n; ++e) {
    uint64_t pair = (uint64_t)e >> 1;
    draw(seed, (uint32_t)pair, (uint32_t)(pair >> 32), (uint32_t)D, ORC_P_ROT,
         (uint32_t)comp, w);
    double u1 = orc_u53(w[0], w[1]);
    double u2 = orc_u53(w[2], w[3]);
    double R = sqrt(-2.0 * log(1.0 - u1));
    double th = ORC_TWO_PI * u2;
    G[e] = (e & 1) ? R * sin(th) : R * cos(th);
  }
}

/* Householder QR of G (row-major D x D); writes Q (row-major) with the
 * columns sign-fixed so that diag(R) > 0.  Works on a column-major copy so
 * every reflector touches contiguous memory; each trailing column is
 * updated independently (parallel over columns, order-independent). */
static void householder_q(const double* G, int D, double* Q) {
  double* A = (double*)malloc(sizeof(double) * (size_t)D * D);  /* col-major */
  double* V = (double*)calloc((size_t)D * D, sizeof(double));  /* reflectors */
  double* beta = (double*)calloc((size_t)D, sizeof(double));
  double* rdiag = (double*)calloc((size_t)D, sizeof(double));
  for (int r = 0; r < D; ++r)
    for (int k = 0; k < D; ++k) A[(size_t)k * D + r] = G[(size_t)r * D + k];

  for (int k = 0; k < D; ++k) {
    double* a = A + (size_t)k * D;
    double nrm2 = 0.0;
    for (int r = k; r < D; ++r) nrm2 += a[r] * a[r];
    double nrm = sqrt(nrm2);
    if (k == D - 1 || nrm == 0.0) {
      rdiag[k] = a[k];
      beta[k] = 0.0;
      continue;
    }
    double alpha = (a[k] >= 0.0) ? -nrm : nrm;
    double* v = V + (size_t)k * D;
    for (int r = k; r < D; ++r) v[r] = a[r];
    v[k] -= alpha;
    double vtv = 0.0;
    for (int r = k; r < D; ++r) vtv += v[r] * v[r];
    beta[k] = (vtv > 0.0) ? 2.0 / vtv : 0.0;
    rdiag[k] = alpha;
    /* apply H_k = I - beta v v^T to the trailing columns */
#pragma omp parallel for schedule(static)
    for (int j = k + 1; j < D; ++j) {
      double* aj = A + (size_t)j * D;
      double s = 0.0;
      for (int r = k; r < D; ++r) s += v[r] * aj[r];
      s *= beta[k];
      for (int r = k; r < D; ++r) aj[r] -= s * v[r];
    }
  }
  /* Q = H_0 H_1 ... H_{D-2} applied to I (backward accumulation), column-major */
  double* Qc = A; /* reuse */
  memset(Qc, 0, sizeof(double) * (size_t)D * D);
  for (int j = 0; j < D; ++j) Qc[(size_t)j * D + j] = 1.0;
  for (int k = D - 1; k >= 0; --k) {
    if (beta[k] == 0.0) continue;
    const double* v = V + (size_t)k * D;
#pragma omp parallel for schedule(static)
    for (int j = k; j < D; ++j) {
      double* qj = Qc + (size_t)j * D;
      double s = 0.0;
      for (int r = k; r < D; ++r) s += v[r] * qj[r];
      s *= beta[k];
      for (int r = k; r < D; ++r) qj[r] -= s * v[r];
    }
  }
  /* sign fix: column k of Q times sign(R_kk) */
  for (int r = 0; r < D; ++r)
    for (int k = 0; k < D; ++k) {
      double q = Qc[(size_t)k * D + r];
      Q[(size_t)r * D + k] = (rdiag[k] < 0.0) ? -q : q;
    }
  free(A);
  free(V);
  free(beta);
  free(rdiag);
}

static void gen_rotation(uint64_t seed, int D, int comp, double* M) {
  double* G = (double*)malloc(sizeof(double) * (size_t)D * D);
  gen_gauss(seed, D, comp, G);
  householder_q(G, D, M);
  free(G);
}

/* Fisher-Yates over Philox: for i = D-1..1 swap perm[i] with perm[below(i+1)] */
static void gen_perm_salt(uint64_t seed, int D, uint32_t salt, int* perm) {
  uint32_t w[4];
  for (int i = 0; i < D; ++i) perm[i] = i;
  for (int i = D - 1; i >= 1; --i) {
    draw(seed, (uint32_t)i, 0, (uint32_t)D, ORC_P_PERM, salt, w);
    int j = (int)orc_below(w[0], (uint32_t)(i + 1));
    int t = perm[i];
    perm[i] = perm[j];
    perm[j] = t;
  }
}

static void gen_perm(uint64_t seed, int D, int* perm) { gen_perm_salt(seed, D, 0, perm); }

/* hybrid structure from the HYB draws with salt: K in 3..5 groups, fractions
 * 0.1 + (1 - 0.1 K) E_k / sum E (E ~ Exp(1)), bodies among the six, sizes
 * floor(frac D) with the last group taking the remainder */
static int gen_hybrid_groups(uint64_t seed, int D, uint32_t salt, int* gsize, int* gbody) {
  uint32_t w[4];
  draw(seed, 0, 0, (uint32_t)D, ORC_P_HYB, salt, w);
  const int K = 3 + (int)orc_below(w[0], 3);
  double E[8], sumE = 0.0;
  for (int k = 0; k < K; ++k) {
    draw(seed, (uint32_t)(1 + k), 0, (uint32_t)D, ORC_P_HYB, salt, w);
    E[k] = -log(1.0 - orc_u53(w[0], w[1]));
    gbody[k] = (int)orc_below(w[2], 6);
    sumE += E[k];
  }
  int used = 0;
  for (int k = 0; k < K; ++k) {
    const double frac = 0.1 + (1.0 - 0.1 * (double)K) * E[k] / sumE;
    if (k < K - 1) {
      gsize[k] = (int)floor(frac * (double)D);
      used += gsize[k];
    } else {
      gsize[k] = D - used;
    }
  }
  return K;
}

static orc_problem* alloc_problem(int family, int D, int K, int ncomp) {
  orc_problem* p = (orc_problem*)calloc(1, sizeof(orc_problem));
  p->family = family;
  p->D = D;
  p->K = K;
  p->fstar = 100.0;
  p->o = (double*)calloc((size_t)ncomp * D, sizeof(double));
  p->M = (double*)calloc((size_t)ncomp * D * D, sizeof(double));
  return p;
}

/* rows of M permuted: M'[t] = M[perm[t]] */
static void permute_rows(double* M, const int* perm, int D) {
  double* T = (double*)malloc(sizeof(double) * (size_t)D * D);
  for (int t = 0; t < D; ++t)
    memcpy(T + (size_t)t * D, M + (size_t)perm[t] * D, sizeof(double) * D);
  memcpy(M, T, sizeof(double) * (size_t)D * D);
  free(T);
}

static orc_problem* make_hybrid(uint64_t seed, int D, int K, const double* frac,
                                const int* bodies) {
  orc_problem* p = alloc_problem(ORC_HYBRID, D, K, 1);
  p->perm = (int*)calloc((size_t)D, sizeof(int));
  p->gsize = (int*)calloc((size_t)K, sizeof(int));
  p->gbody = (int*)calloc((size_t)K, sizeof(int));
  int used = 0;
  for (int k = 0; k < K; ++k) {
    p->gbody[k] = bodies[k];
    if (k < K - 1) {
      p->gsize[k] = (int)floor(frac[k] * (double)D);
      used += p->gsize[k];
    } else {
      p->gsize[k] = D - used;
    }
  }
  gen_shift(seed, D, 0, p->o);
  gen_rotation(seed, D, 0, p->M);
  gen_perm(seed, D, p->perm);
  permute_rows(p->M, p->perm, D);
  return p;
}

orc_problem* orc_hybrid_create(uint64_t seed, int D, int K, const double* frac,
                               const int* bodies) {
  if (D < 1 || K < 1 || K > 16) return NULL;
  return make_hybrid(seed, D, K, frac, bodies);
}

orc_problem* orc_problem_create(uint64_t seed, int family, int D) {
  if (D < 1 || family < 0 || family > ORC_COMP_HYBRID) return NULL;
  uint32_t w[4];
  if (family == ORC_COMP_HYBRID) {
    draw(seed, 0, 0, (uint32_t)D, ORC_P_COMP, 0, w);
    const int Nc = 3 + (int)orc_below(w[0], 3);
    orc_problem* p = alloc_problem(ORC_COMP_HYBRID, D, Nc, Nc);
    p->sigma = (double*)calloc((size_t)Nc, sizeof(double));
    p->lambda = (double*)calloc((size_t)Nc, sizeof(double));
    p->bias = (double*)calloc((size_t)Nc, sizeof(double));
    p->cK = (int*)calloc((size_t)Nc, sizeof(int));
    p->cgsize = (int*)calloc((size_t)Nc * 8, sizeof(int));
    p->cgbody = (int*)calloc((size_t)Nc * 8, sizeof(int));
    p->cperm = (int*)calloc((size_t)Nc * D, sizeof(int));
    for (int c = 0; c < Nc; ++c) {
      draw(seed, (uint32_t)(1 + c), 0, (uint32_t)D, ORC_P_COMP, 0, w);
      p->sigma[c] = 10.0 * (double)(1 + orc_below(w[0], 6));
      p->lambda[c] = pow(10.0, -6.0 + 6.0 * orc_u53(w[1], w[2]));
      p->bias[c] = 100.0 * (double)c;
      gen_shift(seed, D, c, p->o + (size_t)c * D);
      gen_rotation(seed, D, c, p->M + (size_t)c * D * D);
      p->cK[c] = gen_hybrid_groups(seed, D, (uint32_t)(1 + c), p->cgsize + 8 * c,
                                   p->cgbody + 8 * c);
      gen_perm_salt(seed, D, (uint32_t)(1 + c), p->cperm + (size_t)c * D);
      permute_rows(p->M + (size_t)c * D * D, p->cperm + (size_t)c * D, D);
    }
    return p;
  }
  if (family <= ORC_GRIEWANK) {
    orc_problem* p = alloc_problem(family, D, 1, 1);
    gen_shift(seed, D, 0, p->o);
    gen_rotation(seed, D, 0, p->M);
    return p;
  }
  if (family == ORC_HYBRID) {
    draw(seed, 0, 0, (uint32_t)D, ORC_P_HYB, 0, w);
    int K = 3 + (int)orc_below(w[0], 3);
    double E[8], frac[8];
    int bodies[8];
    double sumE = 0.0;
    for (int k = 0; k < K; ++k) {
      draw(seed, (uint32_t)(1 + k), 0, (uint32_t)D, ORC_P_HYB, 0, w);
      E[k] = -log(1.0 - orc_u53(w[0], w[1]));
      bodies[k] = (int)orc_below(w[2], 6);
      sumE += E[k];
    }
    for (int k = 0; k < K; ++k)
      frac[k] = 0.1 + (1.0 - 0.1 * (double)K) * E[k] / sumE;
    return make_hybrid(seed, D, K, frac, bodies);
  }
  /* composition */
  draw(seed, 0, 0, (uint32_t)D, ORC_P_COMP, 0, w);
  int Nc = 3 + (int)orc_below(w[0], 8);
  orc_problem* p = alloc_problem(ORC_COMPOSITION, D, Nc, Nc);
  p->gbody = (int*)calloc((size_t)Nc, sizeof(int));
  p->sigma = (double*)calloc((size_t)Nc, sizeof(double));
  p->lambda = (double*)calloc((size_t)Nc, sizeof(double));
  p->bias = (double*)calloc((size_t)Nc, sizeof(double));
  for (int c = 0; c < Nc; ++c) {
    draw(seed, (uint32_t)(1 + c), 0, (uint32_t)D, ORC_P_COMP, 0, w);
    p->sigma[c] = 10.0 * (double)(1 + orc_below(w[0], 6));
    p->lambda[c] = pow(10.0, -6.0 + 6.0 * orc_u53(w[1], w[2]));
    p->gbody[c] = (int)orc_below(w[3], 6);
    p->bias[c] = 100.0 * (double)c;
    gen_shift(seed, D, c, p->o + (size_t)c * D);
    gen_rotation(seed, D, c, p->M + (size_t)c * D * D);
  }
  return p;
}

void orc_problem_destroy(orc_problem* p) {
  if (!p) return;
  free(p->o);
  free(p->M);
  free(p->perm);
  free(p->gsize);
  free(p->gbody);
  free(p->sigma);
  free(p->lambda);
  free(p->bias);
  free(p->cK);
  free(p->cgsize);
  free(p->cgbody);
  free(p->cperm);
  free(p);
}

void orc_problem_info(const orc_problem* p, int info[3], double* fstar) {
  info[0] = p->family;
  info[1] = p->D;
  info[2] = p->K;
  if (fstar) *fstar = p->fstar;
}

int orc_problem_get(const orc_problem* p, int comp, double* o, double* M) {
  int nc = (p->family == ORC_COMPOSITION || p->family == ORC_COMP_HYBRID) ? p->K : 1;
  if (comp < 0 || comp >= nc) return -1;
  size_t D = (size_t)p->D;
  if (o) memcpy(o, p->o + comp * D, sizeof(double) * D);
  if (M) memcpy(M, p->M + comp * D * D, sizeof(double) * D * D);
  return 0;
}

int orc_problem_hybrid(const orc_problem* p, int* perm, int* gsize, int* gbody) {
  if (p->family != ORC_HYBRID) return -1;
  if (perm) memcpy(perm, p->perm, sizeof(int) * p->D);
  if (gsize) memcpy(gsize, p->gsize, sizeof(int) * p->K);
  if (gbody) memcpy(gbody, p->gbody, sizeof(int) * p->K);
  return 0;
}

int orc_problem_comp_hybrid(const orc_problem* p, int c, int* perm, int* gsize, int* gbody) {
  if (p->family != ORC_COMP_HYBRID || c < 0 || c >= p->K) return -1;
  if (perm) memcpy(perm, p->cperm + (size_t)c * p->D, sizeof(int) * p->D);
  if (gsize) memcpy(gsize, p->cgsize + 8 * c, sizeof(int) * p->cK[c]);
  if (gbody) memcpy(gbody, p->cgbody + 8 * c, sizeof(int) * p->cK[c]);
  return p->cK[c];
}

int orc_problem_comp(const orc_problem* p, int* body, double* sigma,
                     double* lambda, double* bias) {
  if (p->family != ORC_COMPOSITION && p->family != ORC_COMP_HYBRID) return -1;
  int n = p->K;
  if (body && p->gbody) memcpy(body, p->gbody, sizeof(int) * n);
  if (sigma) memcpy(sigma, p->sigma, sizeof(double) * n);
  if (lambda) memcpy(lambda, p->lambda, sizeof(double) * n);
  if (bias) memcpy(bias, p->bias, sizeof(double) * n);
  return 0;
}

/* ======================================================================
 * Evaluation
 * ====================================================================== */

/* z_i = sum_j M_ij (x_j - o_j), j ascending */
void orc_transform(const orc_problem* p, int comp, const double* x, double* z) {
  int D = p->D;
  const double* o = p->o + (size_t)comp * D;
  const double* M = p->M + (size_t)comp * D * D;
  double* d = (double*)malloc(sizeof(double) * D);
  for (int j = 0; j < D; ++j) d[j] = x[j] - o[j];
  for (int i = 0; i < D; ++i) {
    double acc = 0.0;
    for (int j = 0; j < D; ++j) acc += M[(size_t)i * D + j] * d[j];
    z[i] = acc;
  }
  free(d);
}

/* za_i = sum_j |M_ij (x_j - o_j)| for component comp */
static void transform_abs(const orc_problem* p, int comp, const double* x, double* za) {
  int D = p->D;
  const double* o = p->o + (size_t)comp * D;
  const double* M = p->M + (size_t)comp * D * D;
  for (int i = 0; i < D; ++i) {
    double acc = 0.0;
    for (int j = 0; j < D; ++j) acc += fabs(M[(size_t)i * D + j] * (x[j] - o[j]));
    za[i] = acc;
  }
}

static double eval_impl(const orc_problem* p, const double* x, orc_bnd* bnd) {
  int D = p->D;
  double* z = (double*)malloc(sizeof(double) * D);
  double* za = bnd ? (double*)malloc(sizeof(double) * D) : NULL;
  double g = 0.0;
  if (p->family <= ORC_HYBRID) {
    orc_transform(p, 0, x, z); /* hybrid rows already permuted: z' = P M d */
    double dn = 0.0;
    if (bnd) {
      transform_abs(p, 0, x, za);
      for (int j = 0; j < D; ++j) dn += (x[j] - p->o[j]) * (x[j] - p->o[j]);
      dn = sqrt(dn);
    }
    if (p->family <= ORC_GRIEWANK) {
      g = body_impl(p->family, z, D);
      if (bnd) body_bound(p->family, z, za, dn, D, bnd);
    } else {
      double ag = 0.0;
      int start = 0;
      for (int k = 0; k < p->K; ++k) {
        double gk = body_impl(p->gbody[k], z + start, p->gsize[k]);
        g += gk;
        ag += fabs(gk);
        if (bnd) body_bound(p->gbody[k], z + start, za + start, dn, p->gsize[k], bnd);
        start += p->gsize[k];
      }
      if (bnd) bnd->E += B_OP * (double)p->K * ag; /* the sum over groups */
    }
  } else {
    int Nc = p->K;
    double gc[16], sc[16], w[16], om[16], h[16];
    orc_bnd bc[16];
    int exact = -1;
    for (int c = 0; c < Nc; ++c) {
      const double* oc = p->o + (size_t)c * D;
      double s = 0.0;
      for (int j = 0; j < D; ++j) {
        double dj = x[j] - oc[j];
        s += dj * dj;
      }
      sc[c] = s;
      orc_transform(p, c, x, z);
      bc[c].E = bc[c].G = bc[c].Gd = 0.0;
      if (za) transform_abs(p, c, x, za);
      if (p->family == ORC_COMP_HYBRID) { /* component c is a hybrid */
        gc[c] = 0.0;
        double ag = 0.0;
        int start = 0;
        for (int k = 0; k < p->cK[c]; ++k) {
          const int b = p->cgbody[8 * c + k], n = p->cgsize[8 * c + k];
          double gk = body_impl(b, z + start, n);
          gc[c] += gk;
          ag += fabs(gk);
          if (bnd) body_bound(b, z + start, za + start, sqrt(s), n, &bc[c]);
          start += n;
        }
        bc[c].E += B_OP * (double)p->cK[c] * ag;
      } else {
        gc[c] = body_impl(p->gbody[c], z, D);
        if (bnd) body_bound(p->gbody[c], z, za, sqrt(s), D, &bc[c]);
      }
      if (s == 0.0 && exact < 0) exact = c;
    }
    double ex[16], W = 0.0;
    if (exact >= 0) {
      for (int c = 0; c < Nc; ++c) om[c] = (c == exact) ? 1.0 : 0.0;
    } else {
      for (int c = 0; c < Nc; ++c) {
        double sg = p->sigma[c];
        ex[c] = sc[c] / (2.0 * (double)D * sg * sg);
        w[c] = (1.0 / sqrt(sc[c])) * exp(-ex[c]);
        W += w[c];
      }
      for (int c = 0; c < Nc; ++c) om[c] = (W > 0.0) ? w[c] / W : 1.0 / (double)Nc;
    }
    for (int c = 0; c < Nc; ++c) {
      h[c] = p->lambda[c] * gc[c] + p->bias[c];
      g += om[c] * h[c];
    }
    if (bnd) {
      double E = 0.0, ah = 0.0;
      for (int c = 0; c < Nc; ++c) {
        double lw = om[c] * p->lambda[c];
        E += lw * bc[c].E;
        bnd->G += lw * bc[c].G;
        bnd->Gd += lw * bc[c].Gd;
        /* lambda * g_c, + bias, omega * h */
        E += B_OP * om[c] * (p->lambda[c] * fabs(gc[c]) + 2.0 * fabs(h[c]));
        ah += om[c] * fabs(h[c]);
      }
      E += B_OP * (double)Nc * ah; /* the sum over components */
      if (exact < 0 && W > 0.0) {
        /* weights: s_c (n + 2 roundings, relative), 1/sqrt, the exponent's
         * relative error times its size, exp, the product; a common relative
         * error of W cancels against the normalisation up to |g| */
        for (int c = 0; c < Nc; ++c) {
          double rs = B_OP * (double)(D + 2);
          double rw = 0.5 * rs + 2.0 * B_OP + ex[c] * (rs + 4.0 * B_OP) + B_TR + B_OP;
          E += om[c] * rw * fabs(h[c] - g);
        }
        E += B_OP * (double)(Nc + 1) * fabs(g);
      }
      bnd->E += E;
    }
  }
  free(z);
  free(za);
  return g;
}

double orc_eval(const orc_problem* p, const double* x) { return eval_impl(p, x, NULL); }

void orc_eval_bound(const orc_problem* p, const double* x, double out[3]) {
  orc_bnd b = {0.0, 0.0, 0.0};
  eval_impl(p, x, &b);
  out[0] = b.E;
  out[1] = b.G;
  out[2] = b.Gd;
}

void orc_eval_bound_batch(const orc_problem* p, const double* X, int64_t N, int64_t ld,
                          double* out) {
#pragma omp parallel for schedule(dynamic, 4)
  for (int64_t i = 0; i < N; ++i) orc_eval_bound(p, X + i * ld, out + 3 * i);
}

void orc_eval_batch(const orc_problem* p, const double* X, int64_t N, int64_t ld,
                    double* out) {
#pragma omp parallel for schedule(dynamic, 4)
  for (int64_t i = 0; i < N; ++i) out[i] = eval_impl(p, X + i * ld, NULL);
}

/* ======================================================================
 * DE and PSO operators
 * ====================================================================== */

void orc_init_population(uint64_t seed, int NP, int D, double lb, double ub,
                         double* X) {
  uint32_t w[4];
  for (int i = 0; i < NP; ++i)
    for (int j = 0; j < D; ++j) {
      draw(seed, (uint32_t)(j >> 1), (uint32_t)i, 0, ORC_P_INIT, 0, w);
      int pr = j & 1;
      double u = orc_u53(w[2 * pr], w[2 * pr + 1]);
      X[(size_t)i * D + j] = lb + (ub - lb) * u;
    }
}

/* skip-draw: value v in [0, n-m) mapped past the m excluded indices given in
 * ascending order, so the result is uniform over [0,n) minus the excluded */
static int skip_sorted(int v, const int* excl_sorted, int m) {
  for (int t = 0; t < m; ++t)
    if (v >= excl_sorted[t]) ++v;
  return v;
}

static void sort_small(int* a, int m) {
  for (int i = 1; i < m; ++i)
    for (int j = i; j > 0 && a[j - 1] > a[j]; --j) {
      int t = a[j];
      a[j] = a[j - 1];
      a[j - 1] = t;
    }
}

/* binomial crossover + midpoint-target repair of one row */
static void cross_repair(uint64_t seed, uint64_t gen, int i, int D, double CR,
                         int jrand, const double* v, const double* x, double lb,
                         double ub, double* u) {
  uint32_t w[4];
  for (int j = 0; j < D; ++j) {
    if ((j & 3) == 0) draw(seed, (uint32_t)(j >> 2), (uint32_t)i, (uint32_t)gen, ORC_P_CROSS, 0, w);
    double U = (double)w[j & 3] * (1.0 / 4294967296.0);
    double t = (U < CR || j == jrand) ? v[j] : x[j];
    if (t < lb) t = (lb + x[j]) * 0.5;
    if (t > ub) t = (ub + x[j]) * 0.5;
    u[j] = t;
  }
}

void orc_de_rand1_trials(uint64_t seed, uint64_t gen, const double* X, int NP,
                         int D, double F, double CR, double lb, double ub,
                         double* U, int32_t* part) {
  uint32_t w[4];
  double* v = (double*)malloc(sizeof(double) * D);
  for (int i = 0; i < NP; ++i) {
    draw(seed, 0, (uint32_t)i, (uint32_t)gen, ORC_P_PART, 0, w);
    int ex[3];
    int a = (int)orc_below(w[0], (uint32_t)(NP - 1));
    ex[0] = i;
    a = skip_sorted(a, ex, 1);
    ex[1] = a;
    sort_small(ex, 2);
    int b = skip_sorted((int)orc_below(w[1], (uint32_t)(NP - 2)), ex, 2);
    ex[2] = b;
    sort_small(ex, 3);
    int c = skip_sorted((int)orc_below(w[2], (uint32_t)(NP - 3)), ex, 3);
    int jr = (int)orc_below(w[3], (uint32_t)D);
    const double *xa = X + (size_t)a * D, *xb = X + (size_t)b * D, *xc = X + (size_t)c * D;
    for (int j = 0; j < D; ++j) v[j] = fma(F, xb[j] - xc[j], xa[j]);
    cross_repair(seed, gen, i, D, CR, jr, v, X + (size_t)i * D, lb, ub, U + (size_t)i * D);
    if (part) {
      part[4 * i + 0] = a;
      part[4 * i + 1] = b;
      part[4 * i + 2] = c;
      part[4 * i + 3] = jr;
    }
  }
  free(v);
}

int orc_pbest_k(double p, int NP) {
  int k = (int)ceil(p * (double)NP - 1e-9);
  if (k < 1) k = 1;
  if (k > NP) k = NP;
  return k;
}

/* stable ranking by (fitness, index); plain insertion sort keeps it
 * re-entrant for the thread pool */
void orc_rank(const double* f, int NP, int32_t* order) {
  for (int i = 0; i < NP; ++i) order[i] = i;
  for (int i = 1; i < NP; ++i) {
    int32_t cur = order[i];
    int j = i;
    while (j > 0) {
      int32_t prv = order[j - 1];
      int before = (f[cur] < f[prv]) || (f[cur] == f[prv] && cur < prv);
      if (!before) break;
      order[j] = prv;
      --j;
    }
    order[j] = cur;
  }
}

void orc_de_ctpb_trials(uint64_t seed, uint64_t gen, const double* X,
                        const double* fx, int NP, int D, double F, double CR,
                        double p, const double* A, int asize, double lb,
                        double ub, double* U, int32_t* part) {
  uint32_t w[4];
  int k = orc_pbest_k(p, NP);
  int32_t* order = (int32_t*)malloc(sizeof(int32_t) * NP);
  orc_rank(fx, NP, order);
  double* v = (double*)malloc(sizeof(double) * D);
  for (int i = 0; i < NP; ++i) {
    draw(seed, 0, (uint32_t)i, (uint32_t)gen, ORC_P_PART, 0, w);
    int pb = order[orc_below(w[0], (uint32_t)k)];
    int ex[2] = {i, 0};
    int r1 = skip_sorted((int)orc_below(w[1], (uint32_t)(NP - 1)), ex, 1);
    ex[1] = r1;
    sort_small(ex, 2);
    int r2 = skip_sorted((int)orc_below(w[2], (uint32_t)(NP + asize - 2)), ex, 2);
    int jr = (int)orc_below(w[3], (uint32_t)D);
    const double* xi = X + (size_t)i * D;
    const double* xp = X + (size_t)pb * D;
    const double* x1 = X + (size_t)r1 * D;
    const double* x2 = (r2 < NP) ? X + (size_t)r2 * D : A + (size_t)(r2 - NP) * D;
    /* v = x_i + F (x_pb - x_i) + F (x_r1 - x~_r2), as fma(F, a, fma(F, b, x_i)) */
    for (int j = 0; j < D; ++j)
      v[j] = fma(F, x1[j] - x2[j], fma(F, xp[j] - xi[j], xi[j]));
    cross_repair(seed, gen, i, D, CR, jr, v, xi, lb, ub, U + (size_t)i * D);
    if (part) {
      part[4 * i + 0] = pb;
      part[4 * i + 1] = r1;
      part[4 * i + 2] = r2;
      part[4 * i + 3] = jr;
    }
  }
  free(v);
  free(order);
}

/* ---------------------------------------------------------------- SHADE */
void orc_shade_params(uint64_t seed, uint64_t gen, int NP, int H, const double* MF,
                      const double* MCR, double* F, double* CR, int32_t* kpb) {
  uint32_t w[4];
  const double pmin = 2.0 / (double)NP;
  for (int i = 0; i < NP; ++i) {
    draw(seed, 0, (uint32_t)i, (uint32_t)gen, ORC_P_SHADE, 0, w);
    const int r = (int)orc_below(w[0], (uint32_t)H);
    const double p = pmin + (0.2 - pmin) * orc_u53(w[1], w[2]);
    int k = (int)floor(p * (double)NP + 0.5);
    if (k < 1) k = 1;
    if (k > NP) k = NP;
    kpb[i] = k;
    draw(seed, 1, (uint32_t)i, (uint32_t)gen, ORC_P_SHADE, 0, w);
    const double u1 = orc_u53(w[0], w[1]), u2 = orc_u53(w[2], w[3]);
    double cr = MCR[r] + 0.1 * (sqrt(-2.0 * log(1.0 - u1)) * cos(2.0 * ORC_PI * u2));
    if (cr < 0.0) cr = 0.0;
    if (cr > 1.0) cr = 1.0;
    CR[i] = cr;
    double f = MF[r];
    for (int t = 0; t < 64; ++t) {
      draw(seed, (uint32_t)(2 + t), (uint32_t)i, (uint32_t)gen, ORC_P_SHADE, 0, w);
      const double c = MF[r] + 0.1 * tan(ORC_PI * (orc_u53(w[0], w[1]) - 0.5));
      if (c > 0.0) {
        f = c;
        break;
      }
    }
    F[i] = f > 1.0 ? 1.0 : f;
  }
}

int orc_shade_kmax(int NP) {
  const double p = (2.0 / (double)NP > 0.2) ? 2.0 / (double)NP : 0.2;
  int k = (int)floor(p * (double)NP + 0.5);
  if (k < 1) k = 1;
  if (k > NP) k = NP;
  return k;
}

void orc_shade_trials(uint64_t seed, uint64_t gen, const double* X, const double* fx,
                      int NP, int D, const double* F, const double* CR,
                      const int32_t* kpb, double lb, double ub, double* U, int32_t* part) {
  uint32_t w[4];
  int32_t* order = (int32_t*)malloc(sizeof(int32_t) * NP);
  orc_rank(fx, NP, order);
  double* v = (double*)malloc(sizeof(double) * D);
  for (int i = 0; i < NP; ++i) {
    draw(seed, 0, (uint32_t)i, (uint32_t)gen, ORC_P_PART, 0, w);
    const int pb = order[orc_below(w[0], (uint32_t)kpb[i])];
    int ex[2] = {i, 0};
    const int r1 = skip_sorted((int)orc_below(w[1], (uint32_t)(NP - 1)), ex, 1);
    ex[1] = r1;
    sort_small(ex, 2);
    const int r2 = skip_sorted((int)orc_below(w[2], (uint32_t)(NP - 2)), ex, 2);
    const int jr = (int)orc_below(w[3], (uint32_t)D);
    const double* xi = X + (size_t)i * D;
    const double* xp = X + (size_t)pb * D;
    const double* x1 = X + (size_t)r1 * D;
    const double* x2 = X + (size_t)r2 * D;
    for (int j = 0; j < D; ++j)
      v[j] = fma(F[i], x1[j] - x2[j], fma(F[i], xp[j] - xi[j], xi[j]));
    cross_repair(seed, gen, i, D, CR[i], jr, v, xi, lb, ub, U + (size_t)i * D);
    if (part) {
      part[4 * i + 0] = pb;
      part[4 * i + 1] = r1;
      part[4 * i + 2] = r2;
      part[4 * i + 3] = jr;
    }
  }
  free(v);
  free(order);
}

int orc_shade_update(int NP, int H, const double* fx, const double* fu, const double* F,
                     const double* CR, double* MF, double* MCR, int* k) {
  double sw = 0.0, swf = 0.0, swf2 = 0.0, swcr = 0.0;
  int n = 0;
  for (int i = 0; i < NP; ++i) {
    if (!(fu[i] < fx[i])) continue;
    const double d = fx[i] - fu[i];
    sw += d;
    swf += d * F[i];
    swf2 += d * F[i] * F[i];
    swcr += d * CR[i];
    ++n;
  }
  if (n > 0 && sw > 0.0 && swf > 0.0) {
    MF[*k] = swf2 / swf;
    MCR[*k] = swcr / sw;
    *k = (*k + 1) % H;
  }
  return n;
}

int orc_de_select(uint64_t seed, uint64_t gen, double* X, double* fx,
                  const double* U, const double* fu, int NP, int D, double* A,
                  int* asize, uint8_t* acc) {
  uint32_t w[4];
  int nacc = 0;
  for (int i = 0; i < NP; ++i) {
    int a = fu[i] <= fx[i];
    if (acc) acc[i] = (uint8_t)a;
    if (!a) continue;
    ++nacc;
    if (A) {
      int slot;
      if (*asize < NP) {
        slot = (*asize)++;
      } else {
        draw(seed, 0, (uint32_t)i, (uint32_t)gen, ORC_P_ARCH, 0, w);
        slot = (int)orc_below(w[0], (uint32_t)NP);
      }
      memcpy(A + (size_t)slot * D, X + (size_t)i * D, sizeof(double) * D);
    }
    memcpy(X + (size_t)i * D, U + (size_t)i * D, sizeof(double) * D);
    fx[i] = fu[i];
  }
  return nacc;
}

void orc_pso_guides(const double* fp, int NP, int topology, int32_t* guide) {
  if (topology == 0) {
    int b = 0;
    for (int i = 1; i < NP; ++i)
      if (fp[i] < fp[b]) b = i;
    for (int i = 0; i < NP; ++i) guide[i] = b;
    return;
  }
  for (int i = 0; i < NP; ++i) {
    int nb[3] = {(i + NP - 1) % NP, i, (i + 1) % NP};
    sort_small(nb, 3);
    int b = nb[0];
    for (int t = 1; t < 3; ++t)
      if (fp[nb[t]] < fp[b]) b = nb[t];
    guide[i] = b;
  }
}

void orc_pso_move(uint64_t seed, uint64_t gen, double* X, double* V,
                  const double* P, const int32_t* guide, int NP, int D,
                  double w, double c1, double c2, double lb, double ub) {
  uint32_t r[4];
  for (int i = 0; i < NP; ++i) {
    const double* g = P + (size_t)guide[i] * D;
    for (int j = 0; j < D; ++j) {
      size_t e = (size_t)i * D + j;
      draw(seed, (uint32_t)j, (uint32_t)i, (uint32_t)gen, ORC_P_PSO, 0, r);
      double r1 = orc_u53(r[0], r[1]);
      double r2 = orc_u53(r[2], r[3]);
      double a = c1 * r1, b = c2 * r2;
      double x = X[e];
      double v = fma(w, V[e], fma(a, P[e] - x, b * (g[j] - x)));
      double xn = x + v;
      if (xn < lb) {
        xn = lb;
        v = 0.0;
      }
      if (xn > ub) {
        xn = ub;
        v = 0.0;
      }
      X[e] = xn;
      V[e] = v;
    }
  }
}

/* ---------------------------------------------------------------- CSO */
void orc_cso_generation(uint64_t seed, uint64_t gen, double* X, double* V, const double* fx,
                        int NP, int D, double phi, double lb, double ub, int32_t* pair) {
  uint32_t w[4];
  /* pairing: indices sorted by (key, index) */
  uint32_t* key = (uint32_t*)malloc(sizeof(uint32_t) * NP);
  int32_t* ord = (int32_t*)malloc(sizeof(int32_t) * NP);
  for (int i = 0; i < NP; ++i) {
    draw(seed, 0, (uint32_t)i, (uint32_t)gen, ORC_P_CSO, 0, w);
    key[i] = w[0];
    ord[i] = i;
  }
  for (int i = 1; i < NP; ++i) { /* insertion sort, stable in the index */
    int32_t cur = ord[i];
    int j = i;
    while (j > 0 && key[ord[j - 1]] > key[cur]) {
      ord[j] = ord[j - 1];
      --j;
    }
    ord[j] = cur;
  }
  /* mean position before the update */
  double* xbar = (double*)calloc((size_t)D, sizeof(double));
  for (int i = 0; i < NP; ++i)
    for (int j = 0; j < D; ++j) xbar[j] += X[(size_t)i * D + j];
  for (int j = 0; j < D; ++j) xbar[j] /= (double)NP;
  for (int k = 0; k < NP / 2; ++k) {
    const int a = ord[2 * k], b = ord[2 * k + 1];
    const int win = (fx[a] <= fx[b]) ? a : b, los = (win == a) ? b : a;
    pair[2 * k] = win;
    pair[2 * k + 1] = los;
    double* xl = X + (size_t)los * D;
    double* vl = V + (size_t)los * D;
    const double* xw = X + (size_t)win * D;
    for (int j = 0; j < D; ++j) {
      draw(seed, (uint32_t)(1 + 2 * j), (uint32_t)los, (uint32_t)gen, ORC_P_CSO, 0, w);
      const double R1 = orc_u53(w[0], w[1]), R2 = orc_u53(w[2], w[3]);
      draw(seed, (uint32_t)(2 + 2 * j), (uint32_t)los, (uint32_t)gen, ORC_P_CSO, 0, w);
      const double R3 = orc_u53(w[0], w[1]);
      const double v = fma(R1, vl[j], fma(R2, xw[j] - xl[j], (phi * R3) * (xbar[j] - xl[j])));
      double x = xl[j] + v;
      if (x < lb) x = lb;
      if (x > ub) x = ub;
      vl[j] = v;
      xl[j] = x;
    }
  }
  free(xbar);
  free(ord);
  free(key);
}

int orc_pso_update(const double* X, const double* fx, double* P, double* fp,
                   int NP, int D) {
  int n = 0;
  for (int i = 0; i < NP; ++i)
    if (fx[i] < fp[i]) {
      memcpy(P + (size_t)i * D, X + (size_t)i * D, sizeof(double) * D);
      fp[i] = fx[i];
      ++n;
    }
  return n;
}

/* ---------------------------------------------------------------- PSODE */
void orc_psode_select(const double* X, const double* Y, const double* fy, const double* X3,
                      const double* f3, int NP, int D, double* Xn, double* fn, double* V) {
  for (int i = 0; i < NP; ++i) {
    const int from_pso = fy[i] < f3[i];
    for (int j = 0; j < D; ++j) {
      const size_t e = (size_t)i * D + j;
      const double x = X[e], x3 = X3[e];
      V[e] = x3 - x;
      Xn[e] = from_pso ? Y[e] : x3;
    }
    fn[i] = from_pso ? fy[i] : f3[i];
  }
}

void orc_psode_generation(const orc_problem* p, uint64_t seed, uint64_t gen, int NP,
                          double* X, double* fx, double* V, double* P, double* fp,
                          int32_t* guide, double* MF, double* MCR, int* mk, double w, double c1,
                          double c2, double lb, double ub, double* Y, double* fy, double* U,
                          double* fu) {
  const int D = p->D;
  const size_t n = (size_t)NP * D;
  double* VY = (double*)malloc(sizeof(double) * n);
  double* X3 = (double*)malloc(sizeof(double) * n);
  double* f3 = (double*)malloc(sizeof(double) * NP);
  double* Fi = (double*)malloc(sizeof(double) * NP);
  double* CRi = (double*)malloc(sizeof(double) * NP);
  int32_t* kpb = (int32_t*)malloc(sizeof(int32_t) * NP);
  /* the PSO component moves a copy of the population */
  memcpy(Y, X, sizeof(double) * n);
  memcpy(VY, V, sizeof(double) * n);
  orc_pso_move(seed, gen, Y, VY, P, guide, NP, D, w, c1, c2, lb, ub);
  for (int i = 0; i < NP; ++i) fy[i] = orc_eval(p, Y + (size_t)i * D);
  orc_pso_update(Y, fy, P, fp, NP, D);
  orc_pso_guides(fp, NP, 1, guide);
  /* SHADE on another copy */
  orc_shade_params(seed, gen, NP, ORC_SHADE_H, MF, MCR, Fi, CRi, kpb);
  orc_shade_trials(seed, gen, X, fx, NP, D, Fi, CRi, kpb, lb, ub, U, NULL);
  for (int i = 0; i < NP; ++i) fu[i] = orc_eval(p, U + (size_t)i * D);
  orc_shade_update(NP, ORC_SHADE_H, fx, fu, Fi, CRi, MF, MCR, mk);
  memcpy(X3, X, sizeof(double) * n);
  memcpy(f3, fx, sizeof(double) * NP);
  orc_de_select(seed, gen, X3, f3, U, fu, NP, D, NULL, NULL, NULL);
  /* velocity = DE displacement, then the pairwise/3 selection */
  orc_psode_select(X, Y, fy, X3, f3, NP, D, X, fx, V);
  free(VY);
  free(X3);
  free(f3);
  free(Fi);
  free(CRi);
  free(kpb);
}

/* ======================================================================
 * Whole runs: the budget loop of Listing 4 (evaluate NP, count them, then
 * generations while fes < max_fes); only the first (budget - fes) rows of a
 * last, overshooting generation count toward best-so-far.
 * ====================================================================== */
static double min_first(const double* f, int n) {
  double b = INFINITY;
  for (int i = 0; i < n; ++i)
    if (f[i] < b) b = f[i];
  return b;
}

void orc_run(const orc_problem* p, const orc_alg* a, uint64_t seed,
             orc_result* res, int64_t* trace_fes, double* trace_best,
             int64_t trace_cap) {
  int NP = a->NP, D = p->D;
  size_t n = (size_t)NP * D;
  double* X = (double*)malloc(sizeof(double) * n);
  double* fx = (double*)malloc(sizeof(double) * NP);
  double* U = (double*)malloc(sizeof(double) * n);
  double* fu = (double*)malloc(sizeof(double) * NP);
  double* A = NULL;
  double *V = NULL, *P = NULL, *fp = NULL;
  int32_t* guide = NULL;
  int asize = 0;
  int64_t ntr = 0;

  orc_init_population(seed, NP, D, a->lb, a->ub, X);
  for (int i = 0; i < NP; ++i) fx[i] = orc_eval(p, X + (size_t)i * D);
  int64_t cnt = (a->budget < NP) ? a->budget : NP;
  int64_t fes = cnt;
  double best = min_first(fx, (int)cnt);
  if (trace_fes && ntr < trace_cap) {
    trace_fes[ntr] = fes;
    trace_best[ntr] = best;
    ++ntr;
  }
  int64_t gen = 0;
  if (a->alg == 1) A = (double*)malloc(sizeof(double) * n);
  double MF[ORC_SHADE_H], MCR[ORC_SHADE_H];
  int mk = 0;
  double *Fi = NULL, *CRi = NULL;
  int32_t* kpb = NULL;
  if (a->alg == 4 || a->alg == 6) {
    for (int h = 0; h < ORC_SHADE_H; ++h) MF[h] = MCR[h] = 0.5;
    Fi = (double*)malloc(sizeof(double) * NP);
    CRi = (double*)malloc(sizeof(double) * NP);
    kpb = (int32_t*)malloc(sizeof(int32_t) * NP);
  }
  int32_t* pair = NULL;
  if (a->alg == 5) {
    V = (double*)calloc(n, sizeof(double));
    pair = (int32_t*)malloc(sizeof(int32_t) * NP);
  }
  double *Y = NULL, *fy = NULL;
  if (a->alg == 2 || a->alg == 3 || a->alg == 6) {
    V = (double*)calloc(n, sizeof(double));
    P = (double*)malloc(sizeof(double) * n);
    fp = (double*)malloc(sizeof(double) * NP);
    guide = (int32_t*)malloc(sizeof(int32_t) * NP);
    memcpy(P, X, sizeof(double) * n);
    memcpy(fp, fx, sizeof(double) * NP);
    orc_pso_guides(fp, NP, a->alg == 2 ? 0 : 1, guide);
  }
  if (a->alg == 6) {
    Y = (double*)malloc(sizeof(double) * n);
    fy = (double*)malloc(sizeof(double) * NP);
  }
  while (fes < a->budget) {
    ++gen;
    cnt = a->budget - fes;
    if (cnt > NP) cnt = NP;
    if (a->alg == 6) {  /* PSODE: NP PSO rows, then NP DE rows */
      cnt = a->budget - fes;
      if (cnt > 2 * (int64_t)NP) cnt = 2 * (int64_t)NP;
      orc_psode_generation(p, seed, (uint64_t)gen, NP, X, fx, V, P, fp, guide, MF, MCR, &mk,
                           a->w, a->c1, a->c2, a->lb, a->ub, Y, fy, U, fu);
      double b = min_first(fy, (int)(cnt < NP ? cnt : NP));
      if (b < best) best = b;
      b = min_first(fu, (int)(cnt > NP ? cnt - NP : 0));
      if (b < best) best = b;
    } else if (a->alg == 5) {  /* CSO: NP/2 evaluations per generation */
      cnt = a->budget - fes;
      if (cnt > NP / 2) cnt = NP / 2;
      orc_cso_generation(seed, (uint64_t)gen, X, V, fx, NP, D, a->w, a->lb, a->ub, pair);
      for (int k = 0; k < NP / 2; ++k) {
        const int l = pair[2 * k + 1];
        fx[l] = orc_eval(p, X + (size_t)l * D);
        if (k < cnt && fx[l] < best) best = fx[l];
      }
    } else if (a->alg == 4) {
      orc_shade_params(seed, (uint64_t)gen, NP, ORC_SHADE_H, MF, MCR, Fi, CRi, kpb);
      orc_shade_trials(seed, (uint64_t)gen, X, fx, NP, D, Fi, CRi, kpb, a->lb, a->ub, U, NULL);
      for (int i = 0; i < NP; ++i) fu[i] = orc_eval(p, U + (size_t)i * D);
      double b = min_first(fu, (int)cnt);
      if (b < best) best = b;
      orc_shade_update(NP, ORC_SHADE_H, fx, fu, Fi, CRi, MF, MCR, &mk);
      orc_de_select(seed, (uint64_t)gen, X, fx, U, fu, NP, D, NULL, NULL, NULL);
    } else if (a->alg <= 1) {
      if (a->alg == 0)
        orc_de_rand1_trials(seed, (uint64_t)gen, X, NP, D, a->F, a->CR, a->lb, a->ub, U, NULL);
      else
        orc_de_ctpb_trials(seed, (uint64_t)gen, X, fx, NP, D, a->F, a->CR, a->p, A, asize,
                           a->lb, a->ub, U, NULL);
      for (int i = 0; i < NP; ++i) fu[i] = orc_eval(p, U + (size_t)i * D);
      double b = min_first(fu, (int)cnt);
      if (b < best) best = b;
      orc_de_select(seed, (uint64_t)gen, X, fx, U, fu, NP, D, A, a->alg == 1 ? &asize : NULL,
                    NULL);
    } else {
      orc_pso_move(seed, (uint64_t)gen, X, V, P, guide, NP, D, a->w, a->c1, a->c2, a->lb,
                   a->ub);
      for (int i = 0; i < NP; ++i) fx[i] = orc_eval(p, X + (size_t)i * D);
      double b = min_first(fx, (int)cnt);
      if (b < best) best = b;
      orc_pso_update(X, fx, P, fp, NP, D);
      orc_pso_guides(fp, NP, a->alg - 2, guide);
    }
    fes += cnt;
    if (trace_fes && ntr < trace_cap) {
      trace_fes[ntr] = fes;
      trace_best[ntr] = best;
      ++ntr;
    }
  }
  res->best = best;
  res->fes = fes;
  res->gens = gen;
  res->success = best <= 1e-8;
  free(X);
  free(fx);
  free(U);
  free(fu);
  free(A);
  free(V);
  free(P);
  free(fp);
  free(Fi);
  free(CRi);
  free(kpb);
  free(pair);
  free(guide);
  free(Y);
  free(fy);
}

/* ---- thread pool over independent tasks (Sec. 2.4: tasks distributed over
 * the threads of a pool, each running asynchronously) ---- */
typedef struct {
  const orc_problem* const* probs;
  const orc_alg* algs;
  const uint64_t* seeds;
  orc_result* res;
  int ntask;
  int next;
  pthread_mutex_t mu;
} pool_t;

static void* pool_worker(void* arg) {
  pool_t* pl = (pool_t*)arg;
  for (;;) {
    pthread_mutex_lock(&pl->mu);
    int t = pl->next++;
    pthread_mutex_unlock(&pl->mu);
    if (t >= pl->ntask) break;
    orc_run(pl->probs[t], &pl->algs[t], pl->seeds[t], &pl->res[t], NULL, NULL, 0);
  }
  return NULL;
}

void orc_run_many(const orc_problem* const* probs, const orc_alg* algs,
                  const uint64_t* seeds, int ntask, int nthreads,
                  orc_result* res) {
  pool_t pl;
  pl.probs = probs;
  pl.algs = algs;
  pl.seeds = seeds;
  pl.res = res;
  pl.ntask = ntask;
  pl.next = 0;
  pthread_mutex_init(&pl.mu, NULL);
  if (nthreads < 1) nthreads = 1;
  pthread_t* th = (pthread_t*)malloc(sizeof(pthread_t) * nthreads);
  for (int t = 0; t < nthreads; ++t) pthread_create(&th[t], NULL, pool_worker, &pl);
  for (int t = 0; t < nthreads; ++t) pthread_join(th[t], NULL);
  free(th);
  pthread_mutex_destroy(&pl.mu);
}
