/*
 * sevo_oracle.h -- plain FP64 CPU oracle for the batched EA hot path.
 *
 * TEST INFRASTRUCTURE ONLY.  This library is the slow, obviously-correct
 * statement of what the GPU path computes.  Only the test-suite, the smoke
 * check and the benchmark's CPU-baseline leg may load it; the product library
 * never links, includes or calls it, and it shares no source with the CUDA
 * path.
 *
 * What it follows (SEvoBench, arXiv 2505.17430):
 *   - problem = (suite, dimension, instance) and seeded random instances of
 *     each problem: Sec. 1 and Sec. 2.3 (Listing 2);
 *   - algorithm = callable over a fitness function with an evaluation budget,
 *     and the "evaluate NP, then do ... while (fes < max_fes)" loop: Sec. 2.2
 *     and Sec. 4 (Listing 4);
 *   - DE modules: mutation (current-to-pbest/1 "ttpb1"), binomial crossover,
 *     midpoint-target repair, external archive: Sec. 2.2 (Listing 1);
 *   - PSO modules: topology (global / ring "lbest") and update: Sec. 2.2
 *     (Listing 1);
 *   - best-so-far record: Sec. 2.4 and Sec. 3.2;
 *   - runner over (problem, run) tasks on a thread pool: Sec. 2.4 (Listing 3).
 * The paper prints no formula for any body, transform or operator; every
 * formula here is a reading of it, stated at the function that implements
 * it (body forms, Schwefel domain handling, hybrid grouping, composition
 * weighting, Philox counter layout, partner draws, archive policy, PSO
 * details, budget rule).
 *
 * Every function below is pinned by tests under tests/ (closed forms,
 * invariants, brute force, published Philox vectors, exact arithmetic for
 * the rounding bound) except one result: the final error of a full run on a
 * multimodal instance, which the paper does not print (parity unpinned).
 */
#ifndef SEVO_ORACLE_H
#define SEVO_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- families (same numbering as the public C ABI; written independently) */
enum {
  ORC_ELLIPSOID = 0, ORC_ROSENBROCK = 1, ORC_RASTRIGIN = 2, ORC_SCHWEFEL = 3,
  ORC_ACKLEY = 4, ORC_GRIEWANK = 5, ORC_HYBRID = 6, ORC_COMPOSITION = 7,
  /* composition whose components are hybrid functions (the CEC-style
   * composition of hybrid components): Nc in 3..5 components, each with the
   * composition's sigma, lambda, bias, shift and rotation, and its own hybrid
   * groups, bodies and permutation (drawn as a hybrid's, salt 1 + c) */
  ORC_COMP_HYBRID = 8
};

/* ---- Philox purposes (high byte of counter word 3) */
enum {
  ORC_P_INIT = 1, ORC_P_PART = 2, ORC_P_CROSS = 3, ORC_P_ARCH = 4, ORC_P_PSO = 5,
  ORC_P_SHADE = 6, ORC_P_CSO = 7,
  ORC_P_SHIFT = 16, ORC_P_ROT = 17, ORC_P_PERM = 18, ORC_P_HYB = 19, ORC_P_COMP = 20
};

/* Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11). */
void orc_philox(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                uint32_t k0, uint32_t k1, uint32_t out[4]);
double orc_u53(uint32_t w0, uint32_t w1);          /* [0,1), 53 bits   */
uint32_t orc_below(uint32_t w, uint32_t n);        /* [0,n), mul-high  */

/* ---- problem instances ------------------------------------------------ */
typedef struct orc_problem orc_problem;
orc_problem* orc_problem_create(uint64_t seed, int family, int D);
/* hybrid with caller-fixed group count, fractions and bodies (the
 * permutation and rotation are still drawn from the seed). */
orc_problem* orc_hybrid_create(uint64_t seed, int D, int K, const double* frac,
                               const int* bodies);
void orc_problem_destroy(orc_problem* p);
/* info[0]=family, info[1]=D, info[2]=K (hybrid) or Nc (composition) else 1 */
void orc_problem_info(const orc_problem* p, int info[3], double* fstar);
/* copy out component c's shift o (D) and rotation M (D*D row-major; for a
 * hybrid this is the permuted M' = P*M). */
int orc_problem_get(const orc_problem* p, int comp, double* o, double* M);
int orc_problem_hybrid(const orc_problem* p, int* perm, int* gsize, int* gbody);
int orc_problem_comp(const orc_problem* p, int* body, double* sigma,
                     double* lambda, double* bias);
/* composition of hybrids: component c's permutation (D), group sizes and
 * bodies (up to 8 each); returns the component's group count, -1 if none */
int orc_problem_comp_hybrid(const orc_problem* p, int c, int* perm, int* gsize, int* gbody);

/* ---- evaluation: returns the error f(x) - f* (bias-free) -------------- */
double orc_eval(const orc_problem* p, const double* x);
void orc_eval_batch(const orc_problem* p, const double* X, int64_t N, int64_t ld,
                    double* out);
/* rounding-error bound of the plain FP64 evaluation at x, used only to
 * state parity tolerances (not a definition): out[0] = E, the first-order
 * rounding magnitude of the body arithmetic of two implementations of the
 * plain forms, in units of u = 2^-53; out[1] = G = sum_i |dg/dz_i| *
 * sum_j |M_ij d_j|; out[2] = Gd = sum_i |dg/dz_i| * ||d||_2 (per component,
 * weighted by omega_c * lambda_c for compositions).  An error in z of at
 * most a * sum_j |M_ij d_j| + b * ||d||_2 per coordinate then moves g by at
 * most a * G + b * Gd to first order. */
void orc_eval_bound(const orc_problem* p, const double* x, double out[3]);
/* the same for N rows of X (leading dimension ld); out is N x 3 */
void orc_eval_bound_batch(const orc_problem* p, const double* X, int64_t N, int64_t ld,
                          double* out);
/* the bias-free body on an already-transformed vector z of length n */
double orc_body(int family, const double* z, int n);
/* z = M (x - o) for component c (hybrid: the permuted z) */
void orc_transform(const orc_problem* p, int comp, const double* x, double* z);

/* ---- algorithm steps (explicit state arrays, row-major NP x D) --------- */
/* initial population: x_ij = lb + (ub - lb) * u */
void orc_init_population(uint64_t seed, int NP, int D, double lb, double ub,
                         double* X);
/* DE/rand/1/bin trial generation + midpoint-target repair.
 * part (optional, NP*4): r1,r2,r3,jrand per row. */
void orc_de_rand1_trials(uint64_t seed, uint64_t gen, const double* X, int NP,
                         int D, double F, double CR, double lb, double ub,
                         double* U, int32_t* part);
/* pbest pool size k = max(1, ceil(p*NP)) with a 1e-9 guard */
int orc_pbest_k(double p, int NP);
/* rank: indices sorted by (fitness asc, index asc) */
void orc_rank(const double* f, int NP, int32_t* order);
/* DE/current-to-pbest/1/bin with archive A (asize rows) */
void orc_de_ctpb_trials(uint64_t seed, uint64_t gen, const double* X,
                        const double* fx, int NP, int D, double F, double CR,
                        double p, const double* A, int asize, double lb,
                        double ub, double* U, int32_t* part);
/* one-to-one selection (accept iff fu <= fx); archive (may be NULL) gets the
 * replaced parents in row order, random-slot eviction once full (capacity
 * NP).  Returns the number accepted; acc (optional) gets the flags. */
int orc_de_select(uint64_t seed, uint64_t gen, double* X, double* fx,
                  const double* U, const double* fu, int NP, int D, double* A,
                  int* asize, uint8_t* acc);
/* ---- SHADE (Sec. 2.2, Listing 1: shade_parameter with current-to-pbest/1,
 * binomial crossover, midpoint repair, no external archive; success-history
 * adaptation as in the SHADE reference [14] of the paper).  Memory of H slots
 * (M_F, M_CR), initialised to 0.5, write position k. */
#define ORC_SHADE_H 100
/* per individual i (Philox purpose SHADE, counter (sub, i, gen)):
 *   sub 0: r = below(w0, H); p = pmin + (0.2 - pmin) u53(w1, w2), pmin = 2/NP;
 *          pool k_i = floor(p NP + 1/2) clamped to [1, NP] (the top p NP
 *          members, rounded: 2 .. 0.2 NP)
 *   sub 1: CR = M_CR[r] + 0.1 sqrt(-2 ln(1 - u53(w0,w1))) cos(2 pi u53(w2,w3)),
 *          clipped to [0, 1]
 *   sub 2 + t, t < 64: F = M_F[r] + 0.1 tan(pi (u53(w0,w1) - 0.5)) until F > 0
 *          (all 64 failing: F = M_F[r]); F > 1 -> 1 */
void orc_shade_params(uint64_t seed, uint64_t gen, int NP, int H, const double* MF,
                      const double* MCR, double* F, double* CR, int32_t* kpb);
/* largest pool any individual can draw: floor(max(0.2, 2/NP) NP + 1/2) */
int orc_shade_kmax(int NP);
/* current-to-pbest/1/bin without archive with per-individual F, CR, pool */
void orc_shade_trials(uint64_t seed, uint64_t gen, const double* X, const double* fx,
                      int NP, int D, const double* F, const double* CR,
                      const int32_t* kpb, double lb, double ub, double* U, int32_t* part);
/* memory update from the strict improvements fu < fx (fx before selection),
 * weights proportional to fx - fu: M_F[k] = sum w F^2 / sum w F (Lehmer),
 * M_CR[k] = sum w CR / sum w; k = (k + 1) mod H; nothing if no improvement.
 * Sums in row order.  Returns the number of improvements. */
int orc_shade_update(int NP, int H, const double* fx, const double* fu, const double* F,
                     const double* CR, double* MF, double* MCR, int* k);

/* ---- CSO (the competitive swarm optimizer of Sec. 3.3, its reference [16]).
 * One generation of a swarm of NP (even) particles: the pairing is the
 * indices sorted by a Philox key (purpose CSO, counter (0, i, gen), word 0;
 * ties by index) taken two by two; in each pair (a, b) the lower fitness wins
 * (ties: a); the loser l learns:
 *   v_l = fma(R1, v_l, fma(R2, x_w - x_l, (phi R3) (xbar - x_l)))
 *   x_l = x_l + v_l, clamped to [lb, ub] (v_l kept)
 * with R1, R2 = u53 pairs of the draw (purpose CSO, counter (1 + 2 j, l, gen))
 * and R3 the first u53 pair of (2 + 2 j, l, gen); xbar is the swarm's mean
 * position before the update (rows summed in index order, divided by NP).
 * pair (2 NP/2 entries): winner and loser of pair k at [2k], [2k + 1].  The
 * caller evaluates the NP/2 losers. */
void orc_cso_generation(uint64_t seed, uint64_t gen, double* X, double* V, const double* fx,
                        int NP, int D, double phi, double lb, double ub, int32_t* pair);

/* PSO guide index per particle from pbest fitness: topology 0 = global,
 * 1 = ring {i-1,i,i+1} */
void orc_pso_guides(const double* fp, int NP, int topology, int32_t* guide);
/* PSO move: velocity + position + clamp */
void orc_pso_move(uint64_t seed, uint64_t gen, double* X, double* V,
                  const double* P, const int32_t* guide, int NP, int D,
                  double w, double c1, double c2, double lb, double ub);
/* pbest update (strict improvement) */
int orc_pso_update(const double* X, const double* fx, double* P, double* fp,
                   int NP, int D);

/* ---- PSODE (Sec. 4, case study 1; Listing 4's pairwise/3 hybrid of the
 * PSO and SHADE components).  The PSO component keeps personal bests P, fp
 * and ring {i-1,i,i+1} guides, made from the initial population; V starts at
 * zero.  One generation on the population X, fx:
 *   Y  = X moved by orc_pso_move with V, P and the guides (the moved velocity
 *        is dropped), fy = f(Y); personal-best update from (Y, fy) and ring
 *        guides refreshed from fp;
 *   SHADE on X, fx (orc_shade_params, _trials, f(U), _update, then
 *        orc_de_select on a copy) gives the survivors X3, f3;
 *   V  = X3 - X (the DE displacement);
 *   X  = Y where fy < f3, else X3 (a tie keeps the DE survivor).
 * Y, fy, U, fu (NP rows each) receive the generation's 2 NP evaluated rows;
 * the budget counts the PSO rows first, then the DE rows. */
/* the last two steps alone: Xn, fn, V from X, Y, fy, X3, f3 (Xn may be X,
 * fn may be f3) */
void orc_psode_select(const double* X, const double* Y, const double* fy, const double* X3,
                      const double* f3, int NP, int D, double* Xn, double* fn, double* V);
void orc_psode_generation(const orc_problem* p, uint64_t seed, uint64_t gen, int NP,
                          double* X, double* fx, double* V, double* P, double* fp,
                          int32_t* guide, double* MF, double* MCR, int* mk, double w, double c1,
                          double c2, double lb, double ub, double* Y, double* fy, double* U,
                          double* fu);

/* ---- whole runs ------------------------------------------------------- */
typedef struct {
  int alg;          /* 0 DE rand/1/bin, 1 DE ctpb/1/bin+archive, 2 PSO gbest, 3 PSO ring,
                       4 SHADE (F, CR, p unused), 5 CSO (phi in w),
                       6 PSODE (ring PSO with w, c1, c2 + SHADE; F, CR, p unused) */
  int NP;
  double F, CR, p;  /* DE */
  double w, c1, c2; /* PSO */
  double lb, ub;
  int64_t budget;
} orc_alg;

typedef struct {
  double best;      /* best-so-far error (FP64) */
  int64_t fes;      /* evaluations counted (== budget) */
  int64_t gens;     /* generations after the initial one */
  int success;      /* best <= 1e-8 */
} orc_result;

/* trace (optional): trace_fes/trace_best get one entry per generation
 * boundary (initial + each generation), at most trace_cap entries. */
void orc_run(const orc_problem* p, const orc_alg* a, uint64_t seed,
             orc_result* res, int64_t* trace_fes, double* trace_best,
             int64_t trace_cap);

/* thread-pool runner over independent (problem, alg, seed) tasks */
void orc_run_many(const orc_problem* const* probs, const orc_alg* algs,
                  const uint64_t* seeds, int ntask, int nthreads,
                  orc_result* res);

#ifdef __cplusplus
}
#endif
#endif
