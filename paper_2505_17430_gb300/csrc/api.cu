// api.cu -- sevo_evaluate: the batched fitness evaluation entry points.
//
// Mixed modes run one reduced-precision pass over all rows (tcgen05 GEMM or
// CUDA-core FP32), which lists every row whose error is below the
// refinement threshold; the FP64 pass then recomputes exactly those rows
// (the refinement rule of the mixed-precision design: FP64 is kept for the
// shift, the final error near the success threshold and the best-so-far).
#include "kernels.cuh"

static size_t al256(size_t b) { return (b + 255) & ~(size_t)255; }

size_t sv_eval_scratch_bytes(const sevo_problem* p, int prec, int64_t N) {
  size_t b = al256((size_t)N * 4) + al256(16);
  if (prec == SEVO_TF32 || prec == SEVO_BF16X3) b += al256(sv_eval_tc_scratch_bytes(p, prec, N));
  return b;
}

void sv_eval_scratch_carve(void* base, const sevo_problem* p, int prec, int64_t N,
                           EvalScratch* s) {
  char* c = (char*)base;
  s->list = (int32_t*)c;
  c += al256((size_t)N * 4);
  s->counters = (int32_t*)c;
  c += al256(16);
  s->tc = nullptr;
  s->tc_bytes = 0;
  if (prec == SEVO_TF32 || prec == SEVO_BF16X3) {
    s->tc_bytes = sv_eval_tc_scratch_bytes(p, prec, N);
    s->tc = s->tc_bytes ? (void*)c : nullptr;
  }
}

cudaError_t sv_eval_full(const sevo_problem* p, int prec, const double* X, int64_t ld, int64_t N,
                         double* out, const EvalScratch& s, bool reset_counters,
                         cudaStream_t st) {
  cudaError_t e;
  if (reset_counters) {
    e = cudaMemsetAsync(s.counters, 0, 16, st);
    if (e != cudaSuccess) return e;
  }
  EvalAux aux{s.list, s.counters + 0, (uint32_t*)(s.counters + 1)};
  if (prec == SEVO_FP64) {
    aux.refine_list = nullptr;
    return sv_eval_cc(p->desc_d, SEVO_FP64, X, ld, N, out, aux, st);
  }
  if (prec == SEVO_FP32) {
    e = sv_eval_cc(p->desc_d, SEVO_FP32, X, ld, N, out, aux, st);
  } else {
    e = sv_eval_tc(p, prec, X, ld, N, out, aux, s.tc, s.tc_bytes, (uint32_t*)(s.counters + 2), st);
  }
  if (e != cudaSuccess) return e;
  return sv_eval_refine(p->desc_d, X, ld, N, s.list, s.counters + 0, out, st);
}

static int32_t check_eval_args(const sevo_problem* p, const double* pop, int64_t N, int32_t D,
                               int64_t ld, const double* out, int32_t prec) {
  if (!p || !pop || !out || N < 0 || D != p->D || ld < D) return SEVO_ERR_ARG;
  if (prec < SEVO_FP64 || prec > SEVO_FP32) return SEVO_ERR_ARG;
  if (N > (int64_t)INT32_MAX) return SEVO_ERR_UNSUPPORTED;
  if ((prec == SEVO_TF32 || prec == SEVO_BF16X3) && (((uintptr_t)pop & 15) || (ld & 1)))
    return SEVO_ERR_ARG;
  if (((uintptr_t)pop & 7) || ((uintptr_t)out & 7)) return SEVO_ERR_ARG;
  return sv_problem_ready(p);
}

static int32_t evaluate_impl(const sevo_problem* p, const double* pop, int64_t N, int32_t D,
                             int64_t ld, double* out, int32_t prec, void* stream,
                             int64_t* refined, int64_t* nonfinite, bool sync) {
  int32_t st = check_eval_args(p, pop, N, D, ld, out, prec);
  if (st != SEVO_OK) return st;
  if (N == 0) {
    if (refined) *refined = 0;
    if (nonfinite) *nonfinite = 0;
    return SEVO_OK;
  }
  cudaStream_t s = (cudaStream_t)stream;
  size_t bytes = sv_eval_scratch_bytes(p, prec, N);
  void* base = nullptr;
  SV_CUDA(cudaMallocAsync(&base, bytes, s));
  EvalScratch sc;
  sv_eval_scratch_carve(base, p, prec, N, &sc);
  cudaError_t e = sv_eval_full(p, prec, pop, ld, N, out, sc, true, s);
  int32_t host_c[4] = {0, 0, 0, 0};
  if (e == cudaSuccess && sync) e = cudaMemcpyAsync(host_c, sc.counters, 16, cudaMemcpyDeviceToHost, s);
  cudaFreeAsync(base, s);
  if (e != cudaSuccess) {
    sv_set_last_cuda_error(e);
    return SEVO_ERR_CUDA;
  }
  if (sync) {
    SV_CUDA(cudaStreamSynchronize(s));
    if (refined) *refined = host_c[0];
    if (nonfinite) *nonfinite = (uint32_t)host_c[1];
    if (host_c[2] & SV_DEVERR_TIMEOUT) return SEVO_ERR_TIMEOUT;
    if (host_c[1]) return SEVO_ERR_NAN;
  }
  return SEVO_OK;
}

extern "C" int32_t sevo_evaluate(const sevo_problem* p, const double* pop, int64_t N, int32_t D,
                                 int64_t ld, double* out, int32_t prec, void* stream) {
  return evaluate_impl(p, pop, N, D, ld, out, prec, stream, nullptr, nullptr, false);
}

extern "C" int32_t sevo_evaluate_sync(const sevo_problem* p, const double* pop, int64_t N,
                                      int32_t D, int64_t ld, double* out, int32_t prec,
                                      void* stream, int64_t* refined, int64_t* nonfinite) {
  return evaluate_impl(p, pop, N, D, ld, out, prec, stream, refined, nonfinite, true);
}
