// kernels.cuh -- launcher prototypes shared by the library's translation units.
#pragma once
#include <algorithm>
#include <type_traits>

#include "sevo_internal.cuh"

// side outputs of an evaluation pass
struct EvalAux {
  int32_t* refine_list;   // rows whose mixed-precision error < threshold
  int32_t* refine_count;  // number of entries in refine_list
  uint32_t* nonfinite;    // rows whose result is NaN/Inf
};

#define SV_MAX_SEG 64

// Per-generation control block, device-resident so that generations captured
// in a CUDA graph read their Philox counter and evaluation count at run time.
struct GenCtl {
  unsigned long long gen;  // Philox counter of the current generation
  int count;               // rows of this generation that count toward the budget
  int pad;
};

// A generation's counter and count handed to its first kernel as a launch
// argument (on = 1), which publishes them to the control block: no separate
// launch to set the block.  on = 0: the kernel reads the block.
struct CtlSet {
  unsigned long long gen;
  int count;
  int on;
};

// An operator the fused tensor-core evaluation applies in its producer warps
// in place of loading the rows it evaluates: DE trials (rand/1,
// current-to-pbest with archive, SHADE) written to U, or the PSO move
// written in place to X and V; the generation's counter from cs (published
// to ctl by the launch) or, when cs.on == 0, from ctl.
struct GenOp {
  int alg;  // SEVO_DE_RAND1, SEVO_DE_CTPB, SEVO_DE_SHADE, SEVO_PSO_GBEST or SEVO_PSO_RING
  int NP, D, ld, pk;
  double F, lb, ub, w, c1, c2;
  unsigned long long cr_thr;
  const double* X;  // DE: the population
  double* U;        // DE: the trials;  PSO: the population (moved in place)
  const double* A;
  const int32_t* asize;
  const int32_t* order;
  int32_t* part;
  const uint64_t* seeds;
  const double* Fi;
  const double* CRi;
  const int32_t* kpb;
  double* V;
  const double* P;
  const int32_t* guide;
  GenCtl* ctl;
  CtlSet cs;
};

// a run of rows [row0, row0 + nrows) of X evaluated on one problem; X, out,
// err and refined may name the segment's own population, results, device
// error word and refined-row counter (null: the evaluation call's)
struct TcSegment {
  const sevo_problem* p;
  int64_t row0;
  int64_t nrows;
  const double* X = nullptr;
  double* out = nullptr;
  uint32_t* err = nullptr;
  unsigned long long* refined = nullptr;
  const GenOp* op = nullptr;  // rows made by this operator (fused tensor-core path only)
  // the rows' TF32 operand (d = x - o), written by the operator that made
  // them, as a tensor map over the batch's operand buffer (null: convert here)
  const CUtensorMap* amap = nullptr;
};

// tensor map over an operand buffer (rows x D floats, pitch a multiple of 4)
// as the fused evaluation's loader wants it; false if it cannot be built
bool sv_make_operand_map(CUtensorMap* m, const float* A, int D, int64_t rows, int pitch);

// per-segment refinement sub-lists: segment s lists its rows (row indices of
// its own X / out) in list[list_off[s] ...] with count[s] entries
struct RefineTable {
  int nseg;
  const ProblemDev* P[SV_MAX_SEG];
  int64_t list_off[SV_MAX_SEG];
  const double* X[SV_MAX_SEG];  // the segment's rows (null: the launch's X)
  double* out[SV_MAX_SEG];      // the segment's results (null: the launch's out)
  unsigned long long* total[SV_MAX_SEG];  // running count of refined rows (null: none)
};

// SM count of the current device (cached per device)
int sv_num_sms();
// Run a one-time setup step (kernel attributes, which are per device) on the
// current device: `step` runs until it first succeeds on each device; `slot`
// names the step (0 .. SV_ONCE_SLOTS - 1).  Safe to call from several host
// threads (the step may then run more than once; it must be idempotent).
constexpr int SV_ONCE_SLOTS = 8;
enum : int { SV_ONCE_FUSED_SMEM = 0, SV_ONCE_BIG_SMEM = 1 };
cudaError_t sv_once_per_device(int slot, cudaError_t (*step)());

// CUDA-core evaluation of one segment: prec SEVO_FP64 (plain path) or SEVO_FP32
cudaError_t sv_eval_cc(const ProblemDev* Pd, int prec, const double* X, int64_t ld, int64_t row0,
                       int64_t N, double* out, EvalAux aux, cudaStream_t st);
// FP64 re-evaluation of every listed row, all segments in one launch
cudaError_t sv_eval_refine(const RefineTable& T, const double* X, int64_t ld, int64_t max_rows,
                           const int32_t* list, const int32_t* counts, double* out,
                           cudaStream_t st);
// tcgen05 evaluation (TF32 or BF16X3) of segments sharing one D (<= 128);
// refine lists per segment at list_off[s] with counters counts[s]
// (every segment names its X, out and error word; rows of all segments share ld)
cudaError_t sv_eval_tc_segments(const TcSegment* segs, int nseg, int prec, int64_t ld,
                                int32_t* list, const int64_t* list_off, int32_t* counts,
                                uint32_t* nonfinite, void* scratch, size_t scratch_bytes,
                                cudaStream_t st);
// composition scratch of the fused tensor-core pass for `rows` rows
size_t sv_eval_tc_scratch_bytes(bool any_comp, int prec, int64_t rows);
// tensor-core evaluation of one segment with D > 128 (convert, GEMM, combine)
cudaError_t sv_eval_tc_big(const TcSegment& seg, int prec, const double* X, int64_t ld,
                           double* out, int32_t* list, int64_t list_off, int32_t* count,
                           uint32_t* nonfinite, void* scratch, size_t scratch_bytes,
                           uint32_t* dev_err, cudaStream_t st);
size_t sv_eval_big_scratch_bytes(int D, bool any_comp, int prec, int64_t rows);
// encode the TMA descriptors of a freshly uploaded problem
int32_t sv_build_tmaps(sevo_problem* p);

// scratch of one evaluation pass over segments with `rows` rows in total
struct EvalScratch {
  int32_t* list;      // rows (refine sub-lists)
  int32_t* counters;  // [0, SV_MAX_SEG) refine counts, [SV_MAX_SEG] nonfinite,
                      // [SV_MAX_SEG + 1] device error bits
  void* tc;           // tensor-core composition staging
  size_t tc_bytes;
  uint32_t* err;      // persistent device error bits (null: use the counters' word)
  unsigned long long* refined;  // running count of refined rows (null: none)
  bool skip_refine;   // list the rows but keep their mixed values (measurement)
};
#define SV_COUNTERS_BYTES ((SV_MAX_SEG + 4) * 4)
size_t sv_eval_scratch_bytes(int D, bool any_comp, int prec, int64_t rows);
// SEVO_POLICY_REFINE's current value (1: refine, the default)
int sv_policy_refine();
// SEVO_POLICY_TEST_WAIT's current value (0: off, the default)
long long sv_policy_test_wait();
// SEVO_POLICY_FUSE_OPS's current value (0: off, the default)
int sv_policy_fuse_ops();
// measured launch choices (tune.cu): SEVO_POLICY_AUTOTUNE's value (1: on,
// the default); a cached choice for (kind, D, rows, prec), 0 if none; a new
// measured choice with its candidates' times
enum : int { SV_TUNE_BIG_NTILE = 0 };
int sv_policy_autotune();
int32_t sv_tune_set_policy(int64_t value);
int sv_tune_lookup(int kind, int D, int64_t rows, int prec);
void sv_tune_store(int kind, int D, int64_t rows, int prec, int choice, const float* ms,
                   const int* cand, int n);
void sv_eval_scratch_carve(void* base, int D, bool any_comp, int prec, int64_t rows,
                           EvalScratch* s);
// evaluate segments (same D) into out with refinement; resets counters first
cudaError_t sv_eval_segments(const TcSegment* segs, int nseg, int prec, const double* X,
                             int64_t ld, double* out, const EvalScratch& s, cudaStream_t st);
