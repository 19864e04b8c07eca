// api.cu -- sevo_evaluate: the batched fitness evaluation entry points.
//
// Mixed modes run one reduced-precision pass over all rows (tcgen05 GEMM or
// CUDA-core FP32), which lists every row whose error is below the
// refinement threshold; the FP64 pass then recomputes exactly those rows
// (the refinement rule of the mixed-precision design: FP64 is kept for the
// shift, the final error near the success threshold and the best-so-far).
#include "kernels.cuh"

static size_t al256(size_t b) { return (b + 255) & ~(size_t)255; }

static size_t tc_bytes(int D, bool any_comp, int prec, int64_t rows) {
  if (prec != SEVO_TF32 && prec != SEVO_BF16X3) return 0;
  return D > 128 ? sv_eval_big_scratch_bytes(D, any_comp, prec, rows)
                 : sv_eval_tc_scratch_bytes(any_comp, prec, rows);
}

size_t sv_eval_scratch_bytes(int D, bool any_comp, int prec, int64_t rows) {
  return al256((size_t)rows * 4) + al256(SV_COUNTERS_BYTES) + al256(tc_bytes(D, any_comp, prec, rows));
}

void sv_eval_scratch_carve(void* base, int D, bool any_comp, int prec, int64_t rows,
                           EvalScratch* s) {
  char* c = (char*)base;
  s->list = (int32_t*)c;
  c += al256((size_t)rows * 4);
  s->counters = (int32_t*)c;
  c += al256(SV_COUNTERS_BYTES);
  s->tc_bytes = tc_bytes(D, any_comp, prec, rows);
  s->tc = s->tc_bytes ? (void*)c : nullptr;
  s->err = nullptr;
  s->refined = nullptr;
  s->skip_refine = false;
}

// one pass: mixed evaluation of every segment, then one FP64 re-evaluation
// launch over the rows each segment listed (segments are processed in
// groups of SV_MAX_SEG)
cudaError_t sv_eval_segments(const TcSegment* segs, int nseg, int prec, const double* X,
                             int64_t ld, double* out, const EvalScratch& s, cudaStream_t st) {
  cudaError_t e;
  for (int base = 0; base < nseg; base += SV_MAX_SEG) {
    const int n = std::min(SV_MAX_SEG, nseg - base);
    // each segment's own rows, results, error word and refined counter,
    // else the call's
    TcSegment sg[SV_MAX_SEG];
    e = cudaMemsetAsync(s.counters, 0, SV_COUNTERS_BYTES, st);
    if (e != cudaSuccess) return e;
    uint32_t* nonfinite = (uint32_t*)(s.counters + SV_MAX_SEG);
    uint32_t* dev_err = s.err ? s.err : (uint32_t*)(s.counters + SV_MAX_SEG + 1);
    int64_t off[SV_MAX_SEG];
    int64_t tot = 0;
    for (int k = 0; k < n; ++k) {
      sg[k] = segs[base + k];
      if (!sg[k].X) sg[k].X = X;
      if (!sg[k].out) sg[k].out = out;
      if (!sg[k].err) sg[k].err = dev_err;
      if (!sg[k].refined) sg[k].refined = s.refined;
      off[k] = tot;
      tot += sg[k].nrows;
    }
    if (prec == SEVO_FP64) {
      for (int k = 0; k < n; ++k) {
        EvalAux aux{nullptr, nullptr, nonfinite};
        e = sv_eval_cc(sg[k].p->desc_d, SEVO_FP64, sg[k].X, ld, sg[k].row0, sg[k].nrows,
                       sg[k].out, aux, st);
        if (e != cudaSuccess) return e;
      }
      continue;
    }
    if (prec == SEVO_FP32) {
      for (int k = 0; k < n; ++k) {
        EvalAux aux{s.list + off[k], s.counters + k, nonfinite};
        e = sv_eval_cc(sg[k].p->desc_d, SEVO_FP32, sg[k].X, ld, sg[k].row0, sg[k].nrows,
                       sg[k].out, aux, st);
        if (e != cudaSuccess) return e;
      }
    } else if (sg[0].p->D <= 128) {
      e = sv_eval_tc_segments(sg, n, prec, ld, s.list, off, s.counters, nonfinite, s.tc,
                              s.tc_bytes, st);
      if (e != cudaSuccess) return e;
    } else {
      for (int k = 0; k < n; ++k) {
        e = sv_eval_tc_big(sg[k], prec, sg[k].X, ld, sg[k].out, s.list, off[k], s.counters + k,
                           nonfinite, s.tc, s.tc_bytes, sg[k].err, st);
        if (e != cudaSuccess) return e;
      }
    }
    if (s.skip_refine) continue;
    RefineTable RT;
    RT.nseg = n;
    for (int k = 0; k < n; ++k) {
      RT.P[k] = sg[k].p->desc_d;
      RT.list_off[k] = off[k];
      RT.X[k] = sg[k].X;
      RT.out[k] = sg[k].out;
      RT.total[k] = sg[k].refined;
    }
    e = sv_eval_refine(RT, X, ld, tot, s.list, s.counters, out, st);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

static int32_t check_eval_args(const sevo_problem* p, const double* pop, int64_t N, int32_t D,
                               int64_t ld, const double* out, int32_t prec) {
  if (!p || !pop || !out || N < 0 || D != p->D || ld < D) return SEVO_ERR_ARG;
  if (prec < SEVO_FP64 || prec > SEVO_FP32) return SEVO_ERR_ARG;
  if (N > (int64_t)INT32_MAX) return SEVO_ERR_UNSUPPORTED;
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
  const bool comp = sv_weighted_family(p->family);
  size_t bytes = sv_eval_scratch_bytes(p->D, comp, prec, N);
  void* base = nullptr;
  SV_CUDA(cudaMallocAsync(&base, bytes, s));
  EvalScratch sc;
  sv_eval_scratch_carve(base, p->D, comp, prec, N, &sc);
  sc.skip_refine = sv_policy_refine() == 0;
  TcSegment seg{p, 0, N};
  cudaError_t e = sv_eval_segments(&seg, 1, prec, pop, ld, out, sc, s);
  int32_t host_c[SV_MAX_SEG + 4] = {0};
  if (e == cudaSuccess && sync)
    e = cudaMemcpyAsync(host_c, sc.counters, SV_COUNTERS_BYTES, cudaMemcpyDeviceToHost, s);
  cudaFreeAsync(base, s);
  if (e != cudaSuccess) {
    sv_set_last_cuda_error(e);
    return SEVO_ERR_CUDA;
  }
  if (sync) {
    SV_CUDA(cudaStreamSynchronize(s));
    if (refined) *refined = host_c[0];
    if (nonfinite) *nonfinite = (uint32_t)host_c[SV_MAX_SEG];
    if (host_c[SV_MAX_SEG + 1] & SV_DEVERR_TIMEOUT) return SEVO_ERR_TIMEOUT;
    if (host_c[SV_MAX_SEG]) return SEVO_ERR_NAN;
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
