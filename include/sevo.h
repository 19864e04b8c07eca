/*
 * sevo.h -- C ABI of the GB300 batched evolutionary-benchmark hot path.
 *
 * What the library computes (SEvoBench, arXiv 2505.17430):
 *   - problems are (suite, dimension, instance) triples with seeded random
 *     instances (Sec. 1; Sec. 2.3, Listing 2): here a family, a dimension D
 *     and a 64-bit seed give a shifted-rotated, hybrid or composition
 *     instance;
 *   - an algorithm is a callable over the fitness function with an
 *     evaluation budget (Sec. 2.2; Sec. 4, Listing 4): here DE
 *     (rand/1/bin, current-to-pbest/1/bin with an external archive,
 *     binomial crossover, midpoint-target repair -- Listing 1) and PSO
 *     (inertia weight, global or ring "lbest" topology -- Listing 1);
 *   - the runner takes (algorithm, suite, observer, independent runs)
 *     (Sec. 2.4, Listing 3) and records the best-so-far error
 *     (Sec. 2.4, Sec. 3.2).
 * The paper prints no formula for any body, transform or operator; each
 * function below states the reading of the paper it implements.
 *
 * Conventions for every call:
 *   - returns int32 status: SEVO_OK (0) or a negative SEVO_ERR_* code; the
 *     library never aborts, traps or exits; sevo_strerror() explains a code;
 *   - "device" pointers are CUDA global-memory pointers on the device that was
 *     current when the object was created; "host" pointers are ordinary CPU
 *     memory;
 *   - streams are caller-owned cudaStream_t passed as void* (NULL = legacy
 *     default stream); calls that only launch work are asynchronous on that
 *     stream; calls that return results to the host synchronize it;
 *   - FP64 populations are row-major N x D with a leading dimension ld >= D
 *     (in elements) and 8-byte aligned; 16-byte aligned rows (ld even) let
 *     the tensor-core path use vector loads.
 */
#ifndef SEVO_H
#define SEVO_H
#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---------------------------------------------------- */
#define SEVO_OK 0
#define SEVO_ERR_ARG -1          /* bad argument (range, NULL, alignment)  */
#define SEVO_ERR_CUDA -2         /* a CUDA runtime call failed             */
#define SEVO_ERR_OOM -3          /* device or host allocation failed       */
#define SEVO_ERR_TIMEOUT -4      /* a bounded device wait gave up          */
#define SEVO_ERR_NAN -5          /* NaN/Inf in an input population         */
#define SEVO_ERR_UNSUPPORTED -6  /* size or mode not supported             */
#define SEVO_ERR_STATE -7        /* object in the wrong state for the call */

const char* sevo_strerror(int32_t status);
/* library version, e.g. 100 for 0.1.0 */
int32_t sevo_version(void);
/* number of CUDA kernels this library has launched in the process so far
 * (launch accounting for benchmarks; graph replays count the kernels of
 * every replayed generation) */
int64_t sevo_kernel_launches(void);
/* name of the CUDA error behind the calling thread's most recent
 * SEVO_ERR_CUDA ("" if none); static storage */
const char* sevo_last_cuda_error(void);

/* ---- problem families and precision modes ----------------------------- */
enum sevo_family {
  SEVO_ELLIPSOID = 0,   /* sum 10^{6(i-1)/(n-1)} z_i^2                      */
  SEVO_ROSENBROCK = 1,  /* y=z+1: sum 100(y_i^2-y_{i+1})^2 + (y_i-1)^2        */
  SEVO_RASTRIGIN = 2,   /* sum z^2 - 10 cos(2 pi z) + 10                       */
  SEVO_SCHWEFEL = 3,    /* y=z+s: sum c - y sin sqrt|y| (+ outside penalty)   */
  SEVO_ACKLEY = 4,      /* 20 - 20 e^{-0.2 rms(z)} + e - e^{mean cos 2 pi z}  */
  SEVO_GRIEWANK = 5,    /* sum z^2/4000 + 1 - prod cos(z_i/sqrt i)            */
  SEVO_HYBRID = 6,      /* permuted z split into 3..5 groups, a body each     */
  SEVO_COMPOSITION = 7,  /* 3..10 shifted-rotated components, distance weights */
  /* composition whose 3..5 components are hybrid functions (the CEC-style
   * composition of hybrid components): each component has the composition's
   * sigma, lambda, bias, shift and rotation and its own hybrid groups, bodies
   * and permutation (drawn as a hybrid's with salt 1 + c) */
  SEVO_COMP_HYBRID = 8
};

enum sevo_prec {
  SEVO_FP64 = 0,     /* plain FP64 path: DFMA rotation, FP64 bodies           */
  SEVO_TF32 = 1,     /* tcgen05 TF32 rotation GEMM, FP32 bodies, FP64 refine   */
  SEVO_BF16X3 = 2,   /* tcgen05 split-BF16 (hi*hi + hi*lo + lo*hi), FP64 refine */
  SEVO_FP32 = 3      /* CUDA-core FP32 rotation, FP32 bodies, FP64 refine      */
};

/* rows whose mixed-precision error is below this are re-evaluated in FP64 */
#define SEVO_REFINE_THRESHOLD 1e-4
/* a run succeeds when its best-so-far FP64 error is at most this */
#define SEVO_SUCCESS_THRESHOLD 1e-8
#define SEVO_MAX_D 5000
#define SEVO_MAX_GROUPS 8
#define SEVO_MAX_COMPONENTS 10

/* ---- problems -------------------------------------------------------- */
typedef struct sevo_problem sevo_problem; /* opaque, library-owned */

/* Create a seeded random instance of `family` in dimension D (2..5000)
 * (Sec. 1: random instances per problem; Sec. 2.3).  The instance is built
 * on the host; its device copy is made on first device use, on the device
 * current then (later use from another device returns SEVO_ERR_STATE).
 *   shift o ~ U[-80,80]^D; rotation M = Q of the QR (diag R > 0) of a D x D
 *   standard-normal matrix (Box-Muller over Philox4x32-10); hybrid: K in
 *   {3,4,5} groups, fractions 0.1 + (1-0.1K) E_k / sum E (E ~ Exp(1)), a
 *   Fisher-Yates permutation P folded into M' = P M, a body per group;
 *   composition: Nc in [3,10] components with their own o_c, M_c, body,
 *   sigma_c in {10..60}, lambda_c = 10^{U[-6,0]}, bias_c = 100 c.
 *   f* = 100 for every instance.  Host cost O(D^3) (QR); device memory
 *   ~ 16 D^2 bytes per rotation.
 * out: receives a handle owned by the caller until sevo_problem_destroy. */
int32_t sevo_problem_create(uint64_t seed, int32_t family, int32_t D, sevo_problem** out);

/* Hybrid with caller-fixed groups: K (1..8) fractions frac[k] (group k gets
 * floor(frac[k] D) coordinates, the last one the remainder) and bodies[k]
 * (SEVO_ELLIPSOID..SEVO_GRIEWANK).  Permutation and rotation are still drawn
 * from the seed (same o and M as the single-family instance of that seed). */
int32_t sevo_hybrid_create(uint64_t seed, int32_t D, int32_t K, const double* frac,
                           const int32_t* bodies, sevo_problem** out);

int32_t sevo_problem_destroy(sevo_problem* p);

/* family, D, K (hybrid groups) or Nc (components) else 1, and f* (host) */
int32_t sevo_problem_info(const sevo_problem* p, int32_t* family, int32_t* D,
                          int32_t* ncomp, double* fstar);

/* Copy instance data to host buffers (any may be NULL): component `comp`'s
 * shift o (D) and rotation M (D*D row-major, hybrid: permuted M'); hybrid
 * perm (D), gsize and gbody (K); composition body, sigma, lambda, bias (Nc);
 * composition of hybrids: component `comp`'s perm (D), gsize and gbody (its
 * groups, at most 8) and sigma, lambda, bias (Nc). */
int32_t sevo_problem_export(const sevo_problem* p, int32_t comp, double* o, double* M,
                            int32_t* perm, int32_t* gsize, int32_t* gbody, double* sigma,
                            double* lambda, double* bias);

/* ---- batched fitness evaluation (the hot path) ------------------------ */
/* Evaluate N individuals: out[i] = f(pop_i) - f*, FP64 (Sec. 2.3 problem
 * module; best-so-far error of Sec. 2.4 is this value).
 *   pop: device, N x D row-major FP64, leading dimension ld >= D;
 *   out: device, N doubles; prec: enum sevo_prec.
 * Mixed modes (TF32, BF16X3, FP32) compute z = M (x - o) with the shift in
 * FP64, the product in reduced precision with FP32 accumulation and the
 * bodies in FP32; every row whose result is below SEVO_REFINE_THRESHOLD is
 * recomputed on the FP64 path before the call's work completes.
 * Scratch memory comes from a per-problem, per-device pool the library
 * allocates on first use (rows x D x 4 bytes for large D).
 * Errors: SEVO_ERR_ARG for bad sizes/pointers, SEVO_ERR_UNSUPPORTED for a
 * mode/size combination not built.  Asynchronous on `stream`. */
int32_t sevo_evaluate(const sevo_problem* p, const double* pop, int64_t N, int32_t D,
                      int64_t ld, double* out, int32_t prec, void* stream);

/* Same as sevo_evaluate, and also returns (host, after synchronizing the
 * stream) how many rows were refined in FP64 and how many rows held NaN/Inf
 * (those rows get NaN in out and the call returns SEVO_ERR_NAN). */
int32_t sevo_evaluate_sync(const sevo_problem* p, const double* pop, int64_t N, int32_t D,
                           int64_t ld, double* out, int32_t prec, void* stream,
                           int64_t* refined, int64_t* nonfinite);

/* Evaluation that allocates nothing (the paper has no counterpart: this is a
 * library-usage variant of sevo_evaluate, not a step of the method).
 * Some callers cannot allocate device memory at the point of the call --
 * for example a host program whose memory manager has already reserved the
 * GPU's memory in its own pool, or a latency-bound loop that must not pay
 * for (or synchronize on) an allocation.  This entry point takes the same
 * arguments as sevo_evaluate and does the same work, but its scratch (the
 * FP64-refinement row list, the counters and the composition staging) lives
 * in one fixed device array of SEVO_NOALLOC_SCRATCH_BYTES owned by the
 * library; it calls no cudaMalloc/cudaFree and no allocating routine.
 *   - N must be at most SEVO_NOALLOC_MAX_ROWS, else SEVO_ERR_UNSUPPORTED;
 *     in SEVO_TF32 / SEVO_BF16X3 at D > 128 the converted operand and the
 *     per-slice records share the array too, so the limit is lower: with
 *     a(x) = x rounded up to a multiple of 256, kpad = 64 ceil(D / 64) and
 *     nsub = 4 ceil(D / 128), a call needs a(4N) + 512 + a(4 N kpad) +
 *     a(104 N nsub) (+ a(160 N) for compositions) bytes, and N beyond what
 *     fits in SEVO_NOALLOC_SCRATCH_BYTES returns SEVO_ERR_UNSUPPORTED
 *     (D = 1000: 423 rows; D = 5000: 85 rows);
 *   - the problem must already have its device copy on the current device
 *     (any earlier sevo_evaluate / sevo_state_create call with it makes it),
 *     else SEVO_ERR_STATE -- making that copy would allocate;
 *   - every call looks up the array's device address in the current
 *     context (cudaGetSymbolAddress, which allocates nothing and is legal
 *     during stream capture once the library's module is loaded: make one
 *     call of any kind on the device before capturing); after a device reset
 *     every library object (problems, states) is invalid and must be made
 *     again, as for any CUDA allocation;
 *   - every call shares the one array and the array keeps the last call's
 *     contents (the counters are cleared on the stream by each call): calls
 *     whose work overlaps on the GPU (different streams, or different host
 *     threads without ordering) race on it and must be serialized.
 * The device array is held by every GPU that loads the library until the
 * process exits. */
#define SEVO_NOALLOC_MAX_ROWS 16384
#define SEVO_NOALLOC_SCRATCH_BYTES (3u << 20)
int32_t sevo_evaluate_noalloc(const sevo_problem* p, const double* pop, int64_t N, int32_t D,
                              int64_t ld, double* out, int32_t prec, void* stream);

/* ---- algorithms and runs ---------------------------------------------- */
enum sevo_alg {
  SEVO_DE_RAND1 = 0,     /* DE/rand/1/bin                                  */
  SEVO_DE_CTPB = 1,      /* DE/current-to-pbest/1/bin + external archive   */
  SEVO_PSO_GBEST = 2,    /* inertia-weight PSO, global topology            */
  SEVO_PSO_RING = 3,     /* inertia-weight PSO, ring {i-1,i,i+1} topology  */
  /* SHADE (Sec. 2.2, Listing 1's shade_parameter with current-to-pbest/1,
   * binomial crossover and midpoint repair, no external archive): every
   * generation each individual draws its own F (Cauchy around a memory slot's
   * M_F, scale 0.1, redrawn while <= 0, capped at 1), CR (normal around
   * M_CR, sd 0.1, clipped to [0, 1]) and pbest pool (the top round(p NP),
   * p ~ U[2/NP, 0.2]); after selection the strict improvements update one
   * slot (weighted Lehmer mean of F, weighted mean of CR, weights fx - fu).
   * The F, CR and p fields of sevo_alg_params are not used. */
  SEVO_DE_SHADE = 4,
  /* CSO, the competitive swarm optimizer of Sec. 3.3 (its reference [16]):
   * each generation the swarm (NP even) is paired at random (indices sorted
   * by a Philox key); in each pair the loser learns from the winner and from
   * the swarm's mean position, v = R1 v + R2 (x_w - x_l) + phi R3 (xbar - x_l),
   * x = x + v clamped to the bounds, and only the NP/2 losers are evaluated.
   * phi is the `w` field of sevo_alg_params; driven by sevo_pso_step. */
  SEVO_CSO = 5,
  /* PSODE, Sec. 4's first case study (Listing 4: the pairwise/3 hybrid of
   * a PSO and SHADE iterated on copies of one population).  The PSO
   * component is the inertia-weight PSO with ring {i-1,i,i+1} topology
   * (w, c1, c2) and keeps its own personal bests P, fp and guides, made from
   * the initial population; V starts at zero.  One generation (2 NP
   * evaluations, the PSO rows counted first):
   *   Y = X + v, v = w V + c1 r1 (P - X) + c2 r2 (P_guide - X), clamped to
   *       [lb, ub] (the same draws as SEVO_PSO_RING); fy = f(Y); personal
   *       bests from (Y, fy) (strict improvement), guides refreshed;
   *   SHADE on X, fx exactly as SEVO_DE_SHADE: survivors X3, f3 and the
   *       memory update;
   *   V = X3 - X (the DE displacement);
   *   X = Y where fy < f3, else X3 (a tie keeps the DE survivor).
   * The F, CR and p fields are not used.  NP >= 4.  Driven by
   * sevo_state_step only; sevo_state_get's U and fu then hold 2 NP rows
   * per run (the PSO offspring Y, then the DE trials), part the DE partner
   * draws, and sevo_state_get_shade / _set_shade reach the SHADE memory. */
  SEVO_PSODE = 6
};
#define SEVO_SHADE_H 100   /* success-history memory slots per run */

typedef struct {
  int32_t alg;        /* enum sevo_alg                                   */
  int32_t NP;         /* population size (DE >= 4, PSO >= 2)              */
  double F, CR, p;    /* DE scale, crossover rate, pbest fraction         */
  double w, c1, c2;   /* PSO inertia and acceleration coefficients        */
  double lb, ub;      /* box bounds of every coordinate                   */
  int64_t budget;     /* evaluation budget (Listing 4's max_fes)          */
  int32_t prec;       /* enum sevo_prec used for every evaluation         */
} sevo_alg_params;

typedef struct sevo_state sevo_state; /* opaque, library-owned */

/* Allocate one run's device state for problem p, draw the initial
 * population x_ij = lb + (ub-lb) u (Philox, generation 0), evaluate it and
 * count NP evaluations (Listing 4's initial evaluate + add_fes).  The state
 * keeps a pointer to p, which must outlive it. */
int32_t sevo_state_create(const sevo_problem* p, const sevo_alg_params* a, uint64_t seed,
                          void* stream, sevo_state** out);
int32_t sevo_state_destroy(sevo_state* s);
/* Restart every run of the state from a fresh initial population drawn with
 * seeds[0..R) (R = the runs given at creation): the state becomes what
 * sevo_state_create / _create_batch would have made with these seeds and
 * the same problems and parameters (population, fitness, archive emptied,
 * velocities zeroed, personal bests, guides, best-so-far, evaluation and
 * generation counts), without reallocating.  A restart strategy for the
 * caller's outer loop; the paper's algorithms themselves never restart.
 * Enqueued on the state's stream. */
int32_t sevo_state_restart(sevo_state* s, const uint64_t* seeds);

/* Batched state: R independent runs of the same algorithm in one state,
 * run r on problems[r] (all of one dimension D) with Philox key seeds[r].
 * Every step advances all R runs with one launch per kernel; state arrays
 * in sevo_state_get/set/save become R*NP rows (run-major).  R = 1 is
 * exactly sevo_state_create. */
int32_t sevo_state_create_batch(const sevo_problem* const* problems, int32_t R,
                                const sevo_alg_params* a, const uint64_t* seeds, void* stream,
                                sevo_state** out);
/* per-run best-so-far errors (host, R values); synchronizes */
int32_t sevo_state_best(const sevo_state* s, double* best);

/* One DE generation (DE algorithms only): trials from the Philox stream at
 * counter `philox_counter` (mutation, binomial crossover, midpoint-target
 * repair -- Listing 1), their evaluation, one-to-one selection f(u) <= f(x)
 * and, for current-to-pbest, archive insertion of replaced parents.
 * Counts min(NP, budget - fes) evaluations toward best-so-far.
 * SEVO_ERR_STATE if the budget is already spent or the algorithm is not one
 * of SEVO_DE_RAND1, SEVO_DE_CTPB, SEVO_DE_SHADE. */
int32_t sevo_de_step(sevo_state* s, uint64_t philox_counter);

/* One generation of any algorithm (sevo_de_step for DE kinds,
 * sevo_pso_step for PSO kinds and CSO, the PSODE generation above for
 * SEVO_PSODE); counts min(per-generation evaluations, budget - fes).
 * SEVO_ERR_STATE if the budget is already spent. */
int32_t sevo_state_step(sevo_state* s, uint64_t philox_counter);

/* One generation of each of n states (1 <= n <= SEVO_STEP_MANY_MAX), all at
 * counter `philox_counter`, with the same results as sevo_state_step on each
 * in turn: the runner's independent tasks advanced together (Sec. 2.4,
 * Listing 3, whose thread pool runs (problem, run) tasks side by side).
 * When every state is a batched DE, PSO or CSO state (not PSODE, not a
 * run-per-CTA state) of one dimension and precision, each state's
 * operators run on its own stream, then the rows of all states are
 * evaluated in one pass on states[0]'s stream (for D <= 128 in the
 * tensor-core modes one persistent fused launch over every state's rows),
 * then each state's selection runs on its own stream after that pass;
 * otherwise the states step one after another.  The first joint call with
 * a given states[0] allocates that state's joint scratch (grown, never
 * shrunk, freed with the state); make it before any stream capture.  Every
 * state must be on the current device (else SEVO_ERR_STATE), appear once
 * (else SEVO_ERR_ARG) and have budget left (else SEVO_ERR_STATE, checked
 * before anything is launched). */
#define SEVO_STEP_MANY_MAX 16
int32_t sevo_state_step_many(sevo_state* const* states, int32_t n, uint64_t philox_counter);

/* One PSO generation (SEVO_PSO_GBEST, SEVO_PSO_RING and SEVO_CSO only;
 * SEVO_ERR_STATE otherwise or once the budget is spent): velocity and
 * position update with per-coordinate r1, r2 from the Philox stream at
 * `philox_counter`, clamp to [lb,ub] (velocity zeroed where clamped),
 * evaluation, strict pbest update and guide (gbest or ring lbest) refresh;
 * CSO runs the generation described at SEVO_CSO. */
int32_t sevo_pso_step(sevo_state* s, uint64_t philox_counter);

/* Synchronize the state's stream and read the run's bookkeeping (host).
 * Returns SEVO_ERR_TIMEOUT if a bounded device wait gave up in any
 * evaluation since the last call (the results are then unreliable). */
int32_t sevo_state_result(const sevo_state* s, double* best, int64_t* fes, int64_t* gens,
                          int64_t* refined);

/* Host copies of the state arrays (any pointer may be NULL):
 * X, fx (current population and fitness), A (archive rows, asize of them),
 * V, P, fp (PSO velocity, pbest, pbest fitness), U, fu, part (last
 * generation's trial vectors, their fitness and the per-row draws:
 * DE r1,r2,r3,jrand or pbest,r1,r2,jrand; PSO: guide in part[4i]; CSO:
 * the pairing in part[4i]).  Arrays are NP x D row-major (ld = D); for
 * SEVO_PSODE, U and fu are 2 NP rows per run (PSO offspring, then DE
 * trials).  Synchronizes. */
int32_t sevo_state_get(const sevo_state* s, double* X, double* fx, double* A, int32_t* asize,
                       double* V, double* P, double* fp, double* U, double* fu, int32_t* part);
/* SHADE and PSODE runs only (SEVO_ERR_ARG otherwise).  get: the memory (M_F, M_CR: R x
 * SEVO_SHADE_H, slot-major per run; k: R write positions) and the last
 * generation's per-row F, CR and pbest pool sizes (R x NP); any pointer may be
 * NULL; synchronizes.  set: overwrite the memory (NULL = leave as is). */
int32_t sevo_state_get_shade(const sevo_state* s, double* MF, double* MCR, int32_t* k, double* F,
                             double* CR, int32_t* kpb);
int32_t sevo_state_set_shade(sevo_state* s, const double* MF, const double* MCR,
                             const int32_t* k);
/* Overwrite the state arrays from host copies (NULL = leave as is); fes is
 * set to `fes` (>= 0) and guides are recomputed for PSO. */
int32_t sevo_state_set(sevo_state* s, const double* X, const double* fx, const double* A,
                       int32_t asize, const double* V, const double* P, const double* fp,
                       int64_t fes);
/* The same two transfers without waiting: enqueued on the state's stream
 * (after any work already there) and returning at once.  The caller owns the
 * host arrays until the stream has passed this point (set: unchanged; get:
 * not yet valid) -- synchronize the stream (or an event recorded after the
 * call) first.  Page-locked (pinned) host arrays let the copies overlap other
 * work; pageable ones are staged.  sevo_state_get_async has no asize or part
 * outputs. */
int32_t sevo_state_set_async(sevo_state* s, const double* X, const double* fx, const double* A,
                             int32_t asize, const double* V, const double* P, const double* fp,
                             int64_t fes);
int32_t sevo_state_get_async(const sevo_state* s, double* X, double* fx, double* A, double* V,
                             double* P, double* fp, double* U, double* fu);
/* Serialize the whole state (arrays + counters) into buf; *size in: buffer
 * capacity, out: bytes needed/written.  buf == NULL queries the size.
 * Because every draw is counter-based, load + the same counters resumes the
 * run bit-for-bit. */
int32_t sevo_state_save(const sevo_state* s, void* buf, size_t* size);
int32_t sevo_state_load(sevo_state* s, const void* buf, size_t size);

/* ---- experiment grid (Sec. 2.4, Listing 3: evo_bench over runs) -------- */
typedef struct {
  int32_t problem;    /* index into sevo_grid.problems */
  int32_t alg;        /* index into sevo_grid.algs     */
  uint64_t seed;      /* run seed (Philox key)         */
} sevo_task;

typedef struct {
  int32_t nproblems;
  const sevo_problem* const* problems;
  int32_t nalgs;
  const sevo_alg_params* algs;
  int32_t ntasks;
  const sevo_task* tasks;
  int32_t gens_per_graph;  /* generations captured per CUDA graph (0 = auto) */
} sevo_grid;

typedef struct {          /* caller-allocated host arrays, ntasks entries each */
  double* best;           /* best-so-far error (FP64)                          */
  int64_t* fes;           /* evaluations counted (== budget)                   */
  int64_t* gens;          /* generations after the initial one                 */
  int32_t* success;       /* best <= SEVO_SUCCESS_THRESHOLD                     */
  double wall_ms;         /* device wall time of the whole grid                */
  int64_t evals;          /* total evaluations performed                        */
} sevo_grid_result;

/* Run every task to its budget (Sec. 2.4, Listing 3: the runner over
 * (problem, run) tasks).  Tasks with the same algorithm entry and D form a
 * bucket that advances together: one batched launch per kernel per
 * generation over all their runs, generations captured into CUDA graphs.
 * The buckets run side by side, each on its own stream that starts after
 * the work already queued on `stream` (NULL: the legacy default stream);
 * the call returns when all of them are done and `stream` is ordered after
 * them.  Results equal the single-run state API's for the same (problem,
 * alg, seed).  wall_ms is the device time from the start of the first
 * bucket to the end of the last.  Synchronous; every bucket's state is
 * allocated at once (device memory ~ the sum over buckets). */
int32_t sevo_run_grid(const sevo_grid* grid, sevo_grid_result* res, void* stream);

/* ---- execution policy (library infrastructure; the paper has no counterpart)
 * Process-wide switches, read when a state or a grid bucket is created
 * (SEVO_POLICY_REFINE: at each sevo_evaluate / sevo_evaluate_sync call). */
enum sevo_policy {
  /* 1: runs with D <= 32 and NP <= 512 advance in one CTA per run, whole
   * generations per launch, evaluated by CUDA cores (FP64, or FP32 with the
   * operand rounding of the requested mode and FP64 refinement); 0 (default):
   * such runs use the batched kernels like every other run (faster on this
   * part for run grids: one SM's FP64 rate bounds a run-per-CTA generation) */
  SEVO_POLICY_SMALL_RUNS = 0,
  /* 1 (default): sevo_evaluate / sevo_evaluate_sync re-evaluate in FP64 the
   * mixed-precision rows below SEVO_REFINE_THRESHOLD; 0: they return the
   * mixed values as computed (the rows are still counted in `refined`), to
   * measure the mixed arithmetic's own error.  States, grids and
   * sevo_evaluate_noalloc always refine. */
  SEVO_POLICY_REFINE = 1,
  /* for testing the failure path: > 0 makes every CTA of the fused
   * tensor-core evaluation (TF32 / BF16X3, D <= 128) first wait on a
   * barrier that nothing completes, bounded by this many clock cycles
   * (1 .. SEVO_TEST_WAIT_MAX), before it issues any TMEM allocation, TMA
   * copy or MMA; the wait gives up, the CTA leaves with nothing in flight
   * and the call reports SEVO_ERR_TIMEOUT like a real timeout.  0 (default):
   * off. */
  SEVO_POLICY_TEST_WAIT = 2,
  /* 1: in SEVO_TF32 / SEVO_BF16X3 at D <= 128 the DE trials (rand/1,
   * current-to-pbest, SHADE) and the PSO move (global and ring) are formed
   * by the producer warps of the fused tensor-core evaluation, which write
   * them and feed them to the MMA in one pass; 0 (default): each operator
   * runs as a kernel of its own before the evaluation (faster on GB300,
   * whose operator kernels hide their random row loads with far more warps
   * than the fused kernel's producers have).  The results are the same bits
   * either way (the same operator code); read when a generation is
   * launched. */
  SEVO_POLICY_FUSE_OPS = 3,
  /* 1 (default): launch choices that only change speed (today the N-tile
   * width, 64, 128 or 256 columns, of the large-D rotation GEMM) are
   * measured with CUDA events the first time a (D, row count rounded up to
   * a power of two, precision) is evaluated outside stream capture, and
   * cached in memory and in a file ($SEVO_TUNE_FILE, else
   * $XDG_CACHE_HOME/sevo/tune-<gpu>.txt, else $HOME/.cache/sevo/
   * tune-<gpu>.txt); that first call synchronizes its stream.  A cached
   * width other than 64, 128 or 256 is ignored and measured again.  Every
   * width gives the same result bits.  0: a fixed rule (whole waves of jobs times
   * their cost) instead.  2: forget the cached choices and read the file
   * again (the value then reads back as 1). */
  SEVO_POLICY_AUTOTUNE = 4
};
#define SEVO_TEST_WAIT_MAX 100000000
/* SEVO_ERR_ARG for an unknown key or value */
int32_t sevo_set_policy(int32_t key, int64_t value);
/* current value, or -1 for an unknown key */
int64_t sevo_get_policy(int32_t key);

/* ---- kernel tracing (library infrastructure; the paper has no counterpart)
 * While tracing is on, every kernel this library launches on a stream that is
 * not being captured into a graph is bracketed by two CUDA events recorded on
 * that same stream, so the device time of each launch is measured where it
 * ran.  Launches made during graph capture (sevo_run_grid) are not traced.
 * Kinds are fixed; sevo_trace_name gives each one's name. */
enum sevo_trace_kind {
  SEVO_TK_EVAL_TC_FUSED = 0, /* tensor-core evaluation, D <= 128 (fused)     */
  SEVO_TK_EVAL_CC,           /* CUDA-core evaluation (FP64 or FP32 path)      */
  SEVO_TK_REFINE,            /* FP64 re-evaluation of listed rows             */
  SEVO_TK_COMPOSE,           /* composition weighting of component values     */
  SEVO_TK_CONVERT,           /* D > 128: x - o to TF32 / BF16 operand         */
  SEVO_TK_GEMM_BIG,          /* D > 128: rotation GEMM + fused bodies         */
  SEVO_TK_COMBINE,           /* D > 128: merge of column-slice records        */
  SEVO_TK_INIT,              /* initial population                             */
  SEVO_TK_DE_TRIAL,          /* DE mutation + crossover + repair               */
  SEVO_TK_DE_RANK,           /* p-best ranking for current-to-pbest           */
  SEVO_TK_DE_SELECT,         /* DE selection decisions + archive slots        */
  SEVO_TK_DE_APPLY,          /* DE row copies (population, archive)           */
  SEVO_TK_PSO_MOVE,          /* PSO velocity + position update                */
  SEVO_TK_PSO_UPDATE,        /* PSO personal/neighbourhood best               */
  SEVO_TK_PSO_COPY,          /* PSO personal-best row copies                  */
  SEVO_TK_CONTROL,           /* generation counters, fills                     */
  SEVO_TK_SMALL_RUN,         /* run-per-CTA generations of small runs          */
  SEVO_TRACE_KINDS
};
/* on = 1 or 2: clear the accumulators and start tracing (2 also keeps the
 * per-launch timeline below); on = 0: stop (the accumulated figures stay
 * readable); SEVO_ERR_ARG for any other value.  Host-side; cheap when off. */
int32_t sevo_trace_enable(int32_t on);
/* Wait for every traced launch to finish and add its event-measured time to
 * the per-kind totals; counts and ms are caller arrays of SEVO_TRACE_KINDS
 * entries (either may be NULL). */
int32_t sevo_trace_read(int64_t* counts, double* ms);
/* static name of a kind ("" if out of range) */
const char* sevo_trace_name(int32_t kind);
/* The timeline of tracing mode 2: every traced launch finished so far (at
 * most 2^20) as its kind, a stream id (0, 1, ... in order of the streams'
 * first traced launch), and its start and end in ms from the start of the
 * first launch traced since sevo_trace_enable (event resolution, about half
 * a microsecond; a launch on another stream may start before it, giving a
 * negative time), sorted by start.  Waits for every traced launch.  Writes
 * the first min(cap, total) entries into the caller's arrays (each of cap
 * entries; may be NULL when cap is 0) and returns the total count, or
 * SEVO_ERR_ARG / SEVO_ERR_CUDA (negative). */
int64_t sevo_trace_timeline(int64_t cap, int32_t* kinds, int32_t* streams, double* t0,
                            double* t1);

#ifdef __cplusplus
}
#endif
#endif
