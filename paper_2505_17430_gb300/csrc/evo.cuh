// evo.cuh -- batched DE/PSO run state shared by the state API (one run) and
// the grid runner (many runs advancing together).
#pragma once
#include <vector>

#include "kernels.cuh"

struct Batch {
  int alg, D, NP, R, ld;  // R runs of NP rows each, row stride ld (even)
  int per_gen;            // evaluations counted per generation (CSO: NP / 2)
  double F, CR, p, w, c1, c2, lb, ub;
  unsigned long long cr_thr;  // crossover test: word < cr_thr  <=>  word * 2^-32 < CR
  int pbest_k;
  int64_t budget;
  int prec;
  // per-run problem pointers (host) and segments of runs sharing a problem
  std::vector<const sevo_problem*> run_prob;
  std::vector<int> seg_begin;  // first run of each segment (runs sorted by problem)
  // device arrays (one allocation)
  void* block;
  size_t block_bytes;
  double *X, *fx, *U, *fu, *A, *V, *P, *fp, *best;
  int32_t *asize, *guide, *part, *order, *action;
  double* xbar;                  // CSO: the swarm's mean position per run (R x ld)
  double *MF, *MCR, *Fi, *CRi;  // SHADE memory (R x SEVO_SHADE_H) and per-row F, CR
  int32_t *mk, *kpb;            // SHADE write positions (R) and per-row pbest pools
  double *Y, *fy;               // PSODE: the PSO offspring and its fitness
  uint64_t* seeds;
  GenCtl* ctl;
  uint32_t* err;  // device error bits accumulated over every evaluation
  unsigned long long* refined;  // rows re-evaluated in FP64, all generations
  const ProblemDev** rp;        // per-run problem descriptors (device)
  bool small;                   // generations run by the run-per-CTA kernel
  // evaluation scratch (refine list + counters + tensor-core staging)
  void* eval_block;
  size_t eval_bytes;
  bool any_comp;
  cudaStream_t stream;
  CtlSet pending{0ull, 0, 0};   // set by sv_ctl_defer, taken by the next generation's first kernel
  GenOp gop;                    // this generation's operator, when the evaluation applies it
  // the p-best order was ranked from the current fitness by the last
  // selection (current-to-pbest); cleared whenever the host changes fx
  bool rank_fresh = false;
  // the operators' TF32 operand of the rows they make (d = x - o, R*NP rows
  // of apitch floats) and its tensor map, for the fused tensor-core
  // evaluation (TF32, D <= 128, single-component problems); null otherwise
  float* Ad = nullptr;
  int apitch = 0;
  CUtensorMap amap;
  // o of every run's problem as its float hi/lo split, R x apitch each (hi
  // rows, then lo rows), zero past D: read by the operators that write Ad
  float* Osp = nullptr;
};

int32_t sv_batch_alloc(Batch* b, const std::vector<const sevo_problem*>& probs,
                       const std::vector<uint64_t>& seeds, const sevo_alg_params* a,
                       cudaStream_t st);
void sv_batch_free(Batch* b);
// draw the initial population (generation 0), evaluate it, set pbest/guides
cudaError_t sv_batch_init(Batch* b);
// one generation; gen/count read from b->ctl (set by the caller's launch)
cudaError_t sv_batch_generation(Batch* b);
// A generation split at its one evaluation, so that a caller can evaluate
// the rows of several batches in one pass: pre_eval launches the operators
// that make the rows to evaluate (rpr rows per run of M, results into f),
// post_eval the selection that reads the results.  Not for run-per-CTA
// batches or PSODE (two evaluations per generation): sv_batch_splittable.
struct EvalReq {
  const double* M;
  double* f;
  int rpr;
  const GenOp* op;  // the operator the evaluation applies first (fused path), or null
  const CUtensorMap* amap = nullptr;  // the rows' operand, written by their operator
};
bool sv_batch_splittable(const Batch* b);
cudaError_t sv_batch_pre_eval(Batch* b, EvalReq* q);
cudaError_t sv_batch_post_eval(Batch* b);
// the evaluation segments of one batch's request (each naming the batch's
// rows, results, error word and refined counter)
void sv_batch_segments(const Batch* b, const EvalReq& q, std::vector<TcSegment>* segs);
// small batches (b->small): generations gen0 + 1 .. gen0 + gens in run-per-CTA
// launches; leaves ctl at generation gen0 + gens
cudaError_t sv_batch_run_small(Batch* b, unsigned long long gen0, int64_t gens);
cudaError_t sv_ctl_set(Batch* b, unsigned long long gen, int count);
// the next generation's first kernel sets the control block (no launch of
// its own); for batches stepped by sv_batch_generation, not run-per-CTA ones
void sv_ctl_defer(Batch* b, unsigned long long gen, int count);
cudaError_t sv_ctl_advance(Batch* b);  // gen += 1, count from gen and budget
int sv_pbest_k(double p, int NP);
cudaError_t sv_batch_guides(Batch* b);
// read and clear the batch's device error bits (synchronizes its stream)
int32_t sv_batch_status(Batch* b);
#define SV_MAX_NP 4096

// algorithm kinds
inline bool sv_is_de(int alg) {
  return alg == SEVO_DE_RAND1 || alg == SEVO_DE_CTPB || alg == SEVO_DE_SHADE;
}
inline bool sv_is_pso(int alg) {
  return alg == SEVO_PSO_GBEST || alg == SEVO_PSO_RING || alg == SEVO_CSO;
}
// SHADE parameter adaptation (SHADE itself and PSODE's DE component)
inline bool sv_has_shade(int alg) { return alg == SEVO_DE_SHADE || alg == SEVO_PSODE; }
// personal bests and guides (PSO kinds except CSO, and PSODE's PSO component)
inline bool sv_has_pbest(int alg) {
  return alg == SEVO_PSO_GBEST || alg == SEVO_PSO_RING || alg == SEVO_PSODE;
}
inline int sv_topology(int alg) { return (alg == SEVO_PSO_RING || alg == SEVO_PSODE) ? 1 : 0; }
