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

int sv_num_sms();

// CUDA-core evaluation: prec SEVO_FP64 (plain path) or SEVO_FP32
cudaError_t sv_eval_cc(const ProblemDev* Pd, int prec, const double* X, int64_t ld, int64_t N,
                       double* out, EvalAux aux, cudaStream_t st);
// FP64 re-evaluation of the rows listed in list[0 .. *count)
cudaError_t sv_eval_refine(const ProblemDev* Pd, const double* X, int64_t ld, int64_t Nmax,
                           const int32_t* list, const int32_t* count, double* out,
                           cudaStream_t st);
// tcgen05 evaluation (TF32 or BF16X3); scratch_a: N x kpad x 4 bytes (used
// when the A operand is staged through memory), may be null for D <= 256
cudaError_t sv_eval_tc(const sevo_problem* p, int prec, const double* X, int64_t ld, int64_t N,
                       double* out, EvalAux aux, void* scratch, size_t scratch_bytes,
                       uint32_t* dev_err, cudaStream_t st);
size_t sv_eval_tc_scratch_bytes(const sevo_problem* p, int prec, int64_t N);

// full mixed/FP64 evaluation of N rows with refinement, using the given
// scratch (refine list of N int32 + counters); returns a CUDA error
struct EvalScratch {
  int32_t* list;      // N
  int32_t* counters;  // [0] refine count, [1] nonfinite count, [2] device error bits
  void* tc;           // tensor-core staging
  size_t tc_bytes;
};
size_t sv_eval_scratch_bytes(const sevo_problem* p, int prec, int64_t N);
void sv_eval_scratch_carve(void* base, const sevo_problem* p, int prec, int64_t N, EvalScratch* s);
cudaError_t sv_eval_full(const sevo_problem* p, int prec, const double* X, int64_t ld, int64_t N,
                         double* out, const EvalScratch& s, bool reset_counters, cudaStream_t st);
