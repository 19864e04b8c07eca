// state.cu -- single-run state API (sevo_state_*, sevo_de_step,
// sevo_pso_step): one run is a batch of one, driven generation by
// generation with the caller's Philox counters (Listing 4's loop body).
#include <cstring>
#include <vector>

#include "evo.cuh"

struct sevo_state {
  Batch b;
  const sevo_problem* prob;
  sevo_alg_params params;
  uint64_t seed;
  int64_t fes, gens;
  int device;
  // sevo_state_step_many: this state's event (its operators done, or, on
  // the state leading a group, the joint evaluation done) and, on a leading
  // state, the joint evaluation's scratch (kept for the next group step)
  cudaEvent_t ev = nullptr;
  void* joint = nullptr;
  size_t joint_bytes = 0;
};

static bool is_de(int alg) { return sv_is_de(alg); }

static int32_t check_params(const sevo_problem* p, const sevo_alg_params* a) {
  if (!p || !a) return SEVO_ERR_ARG;
  if (a->alg < SEVO_DE_RAND1 || a->alg > SEVO_PSODE) return SEVO_ERR_ARG;
  if (a->alg == SEVO_CSO && (a->NP < 2 || (a->NP & 1))) return SEVO_ERR_ARG;
  if (a->prec < SEVO_FP64 || a->prec > SEVO_FP32) return SEVO_ERR_ARG;
  if (a->NP > SV_MAX_NP || a->budget < 1) return SEVO_ERR_ARG;
  if ((is_de(a->alg) || a->alg == SEVO_PSODE) && a->NP < 4) return SEVO_ERR_ARG;
  if (a->NP < 2) return SEVO_ERR_ARG;
  if (!(a->lb < a->ub) || !(a->CR >= 0.0 && a->CR <= 1.0)) return SEVO_ERR_ARG;
  if (a->alg == SEVO_DE_CTPB && !(a->p > 0.0 && a->p <= 1.0)) return SEVO_ERR_ARG;
  return SEVO_OK;
}

static int32_t create_impl(const sevo_problem* const* probs, int32_t R, const sevo_alg_params* a,
                           const uint64_t* seeds, void* stream, sevo_state** out) {
  if (!out || !probs || !seeds || R < 1) return SEVO_ERR_ARG;
  *out = nullptr;
  for (int r = 0; r < R; ++r) {
    int32_t st = check_params(probs[r], a);
    if (st != SEVO_OK) return st;
    if (probs[r]->D != probs[0]->D) return SEVO_ERR_ARG;
    if ((st = sv_problem_ready(probs[r])) != SEVO_OK) return st;
  }
  if ((int64_t)R * a->NP > (int64_t)INT32_MAX / 4) return SEVO_ERR_UNSUPPORTED;
  sevo_state* s = new (std::nothrow) sevo_state();
  if (!s) return SEVO_ERR_OOM;
  s->prob = probs[0];
  s->params = *a;
  s->seed = seeds[0];
  s->b.block = nullptr;
  s->b.eval_block = nullptr;
  std::vector<const sevo_problem*> pv(probs, probs + R);
  std::vector<uint64_t> sv(seeds, seeds + R);
  int32_t st = sv_batch_alloc(&s->b, pv, sv, a, (cudaStream_t)stream);
  if (st != SEVO_OK) {
    sv_batch_free(&s->b);
    delete s;
    return st;
  }
  cudaError_t e = sv_batch_init(&s->b);
  if (e != cudaSuccess) {
    sv_set_last_cuda_error(e);
    sv_batch_free(&s->b);
    delete s;
    return SEVO_ERR_CUDA;
  }
  s->fes = std::min<int64_t>(a->budget, a->NP);
  s->gens = 0;
  if (cudaGetDevice(&s->device) != cudaSuccess) s->device = -1;
  *out = s;
  return SEVO_OK;
}

extern "C" int32_t sevo_state_create(const sevo_problem* p, const sevo_alg_params* a,
                                     uint64_t seed, void* stream, sevo_state** out) {
  if (!p) return SEVO_ERR_ARG;
  return create_impl(&p, 1, a, &seed, stream, out);
}

extern "C" int32_t sevo_state_restart(sevo_state* s, const uint64_t* seeds) {
  if (!s || !seeds) return SEVO_ERR_ARG;
  Batch& b = s->b;
  const int64_t rows = (int64_t)b.R * b.NP;
  cudaError_t e = cudaMemcpyAsync(b.seeds, seeds, (size_t)b.R * 8, cudaMemcpyHostToDevice, b.stream);
  if (e == cudaSuccess && b.asize) e = cudaMemsetAsync(b.asize, 0, (size_t)b.R * 4, b.stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(b.refined, 0, 8, b.stream);
  if (e == cudaSuccess && b.V)
    e = cudaMemsetAsync(b.V, 0, (size_t)rows * b.ld * 8, b.stream);
  if (e == cudaSuccess) e = sv_batch_init(&b);
  if (e != cudaSuccess) {
    sv_set_last_cuda_error(e);
    return SEVO_ERR_CUDA;
  }
  s->seed = seeds[0];
  s->fes = std::min<int64_t>(s->params.budget, s->params.NP);
  s->gens = 0;
  return SEVO_OK;
}

extern "C" int32_t sevo_state_create_batch(const sevo_problem* const* problems, int32_t R,
                                           const sevo_alg_params* a, const uint64_t* seeds,
                                           void* stream, sevo_state** out) {
  return create_impl(problems, R, a, seeds, stream, out);
}

extern "C" int32_t sevo_state_best(const sevo_state* s, double* best) {
  if (!s || !best) return SEVO_ERR_ARG;
  SV_CUDA(cudaMemcpyAsync(best, s->b.best, (size_t)s->b.R * 8, cudaMemcpyDeviceToHost,
                          s->b.stream));
  SV_CUDA(cudaStreamSynchronize(s->b.stream));
  return sv_batch_status(const_cast<Batch*>(&s->b));
}

extern "C" int32_t sevo_state_destroy(sevo_state* s) {
  if (!s) return SEVO_ERR_ARG;
  cudaStreamSynchronize(s->b.stream);
  if (s->ev) cudaEventDestroy(s->ev);
  if (s->joint) cudaFree(s->joint);
  sv_batch_free(&s->b);
  delete s;
  return SEVO_OK;
}

enum StepKind { STEP_DE, STEP_PSO, STEP_ANY };

static int32_t step(sevo_state* s, uint64_t counter, StepKind kind) {
  if (!s) return SEVO_ERR_ARG;
  if (kind == STEP_DE && !is_de(s->params.alg)) return SEVO_ERR_STATE;
  if (kind == STEP_PSO && !sv_is_pso(s->params.alg)) return SEVO_ERR_STATE;
  if (s->fes >= s->params.budget) return SEVO_ERR_STATE;
  const int count = (int)std::min<int64_t>(s->b.per_gen, s->params.budget - s->fes);
  cudaError_t e = cudaSuccess;
  if (s->b.small)
    e = sv_ctl_set(&s->b, (unsigned long long)counter, count);
  else
    sv_ctl_defer(&s->b, (unsigned long long)counter, count);
  if (e == cudaSuccess) e = sv_batch_generation(&s->b);
  if (e != cudaSuccess) {
    sv_set_last_cuda_error(e);
    return SEVO_ERR_CUDA;
  }
  s->fes += count;
  s->gens += 1;
  return SEVO_OK;
}

extern "C" int32_t sevo_de_step(sevo_state* s, uint64_t philox_counter) {
  return step(s, philox_counter, STEP_DE);
}

extern "C" int32_t sevo_state_step(sevo_state* s, uint64_t philox_counter) {
  return step(s, philox_counter, STEP_ANY);
}

extern "C" int32_t sevo_pso_step(sevo_state* s, uint64_t philox_counter) {
  return step(s, philox_counter, STEP_PSO);
}

static cudaError_t state_event(sevo_state* s) {
  if (s->ev) return cudaSuccess;
  return cudaEventCreateWithFlags(&s->ev, cudaEventDisableTiming);
}

// One generation of each state with every state's rows evaluated in one
// pass: each state's operators on its own stream, then one evaluation of
// all their rows on the first state's stream (the fused tensor-core kernel
// then walks all of them in one persistent launch), then each state's
// selection on its own stream.  Same results as sevo_state_step on each.
static int32_t step_many(sevo_state* const* st, int32_t n, uint64_t counter) {
  sevo_state* lead = st[0];
  const Batch& b0 = lead->b;
  std::vector<int> counts(n);
  int64_t rows = 0;
  bool any_comp = false;
  cudaError_t e = cudaSuccess;
  for (int i = 0; i < n; ++i) {
    Batch& b = st[i]->b;
    counts[i] = (int)std::min<int64_t>(b.per_gen, st[i]->params.budget - st[i]->fes);
    rows += (int64_t)b.R * b.NP;
    any_comp = any_comp || b.any_comp;
  }
  // joint scratch on the leading state (stream-ordered after its earlier use)
  const size_t need = sv_eval_scratch_bytes(b0.D, any_comp, b0.prec, rows);
  if (lead->joint_bytes < need) {
    if (lead->joint) {
      if ((e = cudaStreamSynchronize(b0.stream)) != cudaSuccess) return SEVO_ERR_CUDA;
      cudaFree(lead->joint);
      lead->joint = nullptr;
      lead->joint_bytes = 0;
    }
    if (cudaMalloc(&lead->joint, need) != cudaSuccess) return SEVO_ERR_OOM;
    lead->joint_bytes = need;
  }
  for (int i = 0; i < n; ++i)
    if ((e = state_event(st[i])) != cudaSuccess) break;
  std::vector<TcSegment> segs;
  for (int i = 0; i < n && e == cudaSuccess; ++i) {
    Batch& b = st[i]->b;
    EvalReq q;
    sv_ctl_defer(&b, (unsigned long long)counter, counts[i]);
    e = sv_batch_pre_eval(&b, &q);
    if (e == cudaSuccess) sv_batch_segments(&b, q, &segs);
    if (e == cudaSuccess && i > 0) {
      e = cudaEventRecord(st[i]->ev, b.stream);
      if (e == cudaSuccess) e = cudaStreamWaitEvent(b0.stream, st[i]->ev, 0);
    }
  }
  if (e == cudaSuccess) {
    EvalScratch sc;
    sv_eval_scratch_carve(lead->joint, b0.D, any_comp, b0.prec, rows, &sc);
    e = sv_eval_segments(segs.data(), (int)segs.size(), b0.prec, segs[0].X, b0.ld, segs[0].out,
                         sc, b0.stream);
  }
  if (e == cudaSuccess && n > 1) e = cudaEventRecord(lead->ev, b0.stream);
  for (int i = 0; i < n && e == cudaSuccess; ++i) {
    Batch& b = st[i]->b;
    if (i > 0) e = cudaStreamWaitEvent(b.stream, lead->ev, 0);
    if (e == cudaSuccess) e = sv_batch_post_eval(&b);
  }
  if (e != cudaSuccess) {
    sv_set_last_cuda_error(e);
    return SEVO_ERR_CUDA;
  }
  for (int i = 0; i < n; ++i) {
    st[i]->fes += counts[i];
    st[i]->gens += 1;
  }
  return SEVO_OK;
}

extern "C" int32_t sevo_state_step_many(sevo_state* const* states, int32_t n,
                                        uint64_t philox_counter) {
  if (!states || n < 1 || n > SEVO_STEP_MANY_MAX) return SEVO_ERR_ARG;
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) return SEVO_ERR_CUDA;
  bool joint = true;
  for (int i = 0; i < n; ++i) {
    const sevo_state* s = states[i];
    if (!s) return SEVO_ERR_ARG;
    for (int k = 0; k < i; ++k)
      if (states[k] == s) return SEVO_ERR_ARG;
    if (s->device != dev) return SEVO_ERR_STATE;
    if (s->fes >= s->params.budget) return SEVO_ERR_STATE;
    joint = joint && sv_batch_splittable(&s->b) && s->b.D == states[0]->b.D &&
            s->b.prec == states[0]->b.prec && s->b.ld == states[0]->b.ld;
  }
  if (joint && n > 1) return step_many(states, n, philox_counter);
  // nothing to share (one state, or states whose generations cannot share
  // an evaluation): one generation each
  for (int i = 0; i < n; ++i) {
    const int32_t r = step(states[i], philox_counter, STEP_ANY);
    if (r != SEVO_OK) return r;
  }
  return SEVO_OK;
}

extern "C" int32_t sevo_state_result(const sevo_state* s, double* best, int64_t* fes,
                                     int64_t* gens, int64_t* refined) {
  if (!s) return SEVO_ERR_ARG;
  double b = 0.0;
  SV_CUDA(cudaMemcpyAsync(&b, s->b.best, 8, cudaMemcpyDeviceToHost, s->b.stream));
  SV_CUDA(cudaStreamSynchronize(s->b.stream));
  const int32_t dev = sv_batch_status(const_cast<Batch*>(&s->b));
  if (dev != SEVO_OK) return dev;
  if (best) *best = b;
  if (fes) *fes = s->fes;
  if (gens) *gens = s->gens;
  if (refined) {
    unsigned long long n = 0;
    SV_CUDA(cudaMemcpyAsync(&n, s->b.refined, 8, cudaMemcpyDeviceToHost, s->b.stream));
    SV_CUDA(cudaStreamSynchronize(s->b.stream));
    *refined = (int64_t)n;
  }
  return SEVO_OK;
}

// copy a row-major NP x D host matrix to/from the ld-strided device matrix
// host rows are dense (D doubles); device rows have pitch ld (D rounded up to
// even): one plain copy when they coincide, a pitched copy otherwise
static cudaError_t put(double* dst, const double* src, const Batch& b) {
  const size_t rows = (size_t)b.R * b.NP;
  if (b.ld == b.D)
    return cudaMemcpyAsync(dst, src, rows * b.D * 8, cudaMemcpyHostToDevice, b.stream);
  return cudaMemcpy2DAsync(dst, (size_t)b.ld * 8, src, (size_t)b.D * 8, (size_t)b.D * 8, rows,
                           cudaMemcpyHostToDevice, b.stream);
}
static cudaError_t get(double* dst, const double* src, const Batch& b) {
  const size_t rows = (size_t)b.R * b.NP;
  if (b.ld == b.D)
    return cudaMemcpyAsync(dst, src, rows * b.D * 8, cudaMemcpyDeviceToHost, b.stream);
  return cudaMemcpy2DAsync(dst, (size_t)b.D * 8, src, (size_t)b.ld * 8, (size_t)b.D * 8, rows,
                           cudaMemcpyDeviceToHost, b.stream);
}

// the generation's evaluated rows: U, fu, or for PSODE per run the NP PSO
// offspring (Y, fy) followed by the NP DE trials (U, fu)
static cudaError_t get_evaluated(double* U, double* fu, const Batch& b) {
  if (!b.Y) {
    cudaError_t e = cudaSuccess;
    if (U && b.U) e = get(U, b.U, b);
    if (e == cudaSuccess && fu && b.fu)
      e = cudaMemcpyAsync(fu, b.fu, (size_t)b.R * b.NP * 8, cudaMemcpyDeviceToHost, b.stream);
    return e;
  }
  const size_t np = (size_t)b.NP;
  for (int r = 0; r < b.R; ++r) {
    for (int half = 0; half < 2; ++half) {
      const double* M = half ? b.U : b.Y;
      const double* f = half ? b.fu : b.fy;
      const size_t hrow = (2 * (size_t)r + half) * np;  // first host row
      cudaError_t e = cudaSuccess;
      if (U)
        e = cudaMemcpy2DAsync(U + hrow * b.D, (size_t)b.D * 8, M + (size_t)r * np * b.ld,
                              (size_t)b.ld * 8, (size_t)b.D * 8, np, cudaMemcpyDeviceToHost,
                              b.stream);
      if (e == cudaSuccess && fu)
        e = cudaMemcpyAsync(fu + hrow, f + (size_t)r * np, np * 8, cudaMemcpyDeviceToHost,
                            b.stream);
      if (e != cudaSuccess) return e;
    }
  }
  return cudaSuccess;
}

extern "C" int32_t sevo_state_get(const sevo_state* s, double* X, double* fx, double* A,
                                  int32_t* asize, double* V, double* P, double* fp, double* U,
                                  double* fu, int32_t* part) {
  if (!s) return SEVO_ERR_ARG;
  const Batch& b = s->b;
  const size_t rows = (size_t)b.R * b.NP, vb = rows * 8;
  if (X) SV_CUDA(get(X, b.X, b));
  if (fx) SV_CUDA(cudaMemcpyAsync(fx, b.fx, vb, cudaMemcpyDeviceToHost, b.stream));
  if (A && b.A) SV_CUDA(get(A, b.A, b));
  int32_t as = 0;  // run 0's archive size
  if (b.asize) SV_CUDA(cudaMemcpyAsync(&as, b.asize, 4, cudaMemcpyDeviceToHost, b.stream));
  if (V && b.V) SV_CUDA(get(V, b.V, b));
  if (P && b.P) SV_CUDA(get(P, b.P, b));
  if (fp && b.fp) SV_CUDA(cudaMemcpyAsync(fp, b.fp, vb, cudaMemcpyDeviceToHost, b.stream));
  SV_CUDA(get_evaluated(U, fu, b));
  if (part) {
    if (s->params.alg == SEVO_CSO) {  // the pairing: part[4i] = pair entry i
      std::vector<int32_t> g(rows);
      SV_CUDA(cudaMemcpyAsync(g.data(), b.order, rows * 4, cudaMemcpyDeviceToHost, b.stream));
      SV_CUDA(cudaStreamSynchronize(b.stream));
      for (size_t i = 0; i < rows; ++i) {
        part[4 * i] = g[i];
        part[4 * i + 1] = part[4 * i + 2] = part[4 * i + 3] = 0;
      }
    } else if (is_de(s->params.alg) || s->params.alg == SEVO_PSODE) {
      SV_CUDA(cudaMemcpyAsync(part, b.part, rows * 16, cudaMemcpyDeviceToHost, b.stream));
    } else {
      std::vector<int32_t> g(rows);
      SV_CUDA(cudaMemcpyAsync(g.data(), b.guide, rows * 4, cudaMemcpyDeviceToHost, b.stream));
      SV_CUDA(cudaStreamSynchronize(b.stream));
      for (size_t i = 0; i < rows; ++i) {
        part[4 * i] = g[i];
        part[4 * i + 1] = part[4 * i + 2] = part[4 * i + 3] = 0;
      }
    }
  }
  SV_CUDA(cudaStreamSynchronize(b.stream));
  if (asize) *asize = as;
  return SEVO_OK;
}

static int32_t set_impl(sevo_state* s, const double* X, const double* fx, const double* A,
                        int32_t asize, const double* V, const double* P, const double* fp,
                        int64_t fes, bool wait) {
  if (!s) return SEVO_ERR_ARG;
  Batch& b = s->b;
  const size_t vb = (size_t)b.R * b.NP * 8;
  if (asize < 0 || asize > b.NP || (A && b.R != 1)) return SEVO_ERR_ARG;
  b.rank_fresh = false;  // the p-best order is ranked again from the new fitness
  if (X) SV_CUDA(put(b.X, X, b));
  if (fx) SV_CUDA(cudaMemcpyAsync(b.fx, fx, vb, cudaMemcpyHostToDevice, b.stream));
  if (A && b.A) SV_CUDA(put(b.A, A, b));
  // (a copy from pageable host memory returns once the source has been read)
  if (b.asize && A) SV_CUDA(cudaMemcpyAsync(b.asize, &asize, 4, cudaMemcpyHostToDevice, b.stream));
  if (V && b.V) SV_CUDA(put(b.V, V, b));
  if (P && b.P) SV_CUDA(put(b.P, P, b));
  if (fp && b.fp) SV_CUDA(cudaMemcpyAsync(b.fp, fp, vb, cudaMemcpyHostToDevice, b.stream));
  if (sv_has_pbest(s->params.alg) && fp && b.fp) {  // guides from the new pbest fitness
    cudaError_t e = sv_batch_guides(&b);
    if (e != cudaSuccess) {
      sv_set_last_cuda_error(e);
      return SEVO_ERR_CUDA;
    }
  }
  if (fes >= 0) s->fes = fes;
  if (wait) SV_CUDA(cudaStreamSynchronize(b.stream));
  return SEVO_OK;
}

extern "C" int32_t sevo_state_set(sevo_state* s, const double* X, const double* fx,
                                  const double* A, int32_t asize, const double* V,
                                  const double* P, const double* fp, int64_t fes) {
  return set_impl(s, X, fx, A, asize, V, P, fp, fes, true);
}

extern "C" int32_t sevo_state_set_async(sevo_state* s, const double* X, const double* fx,
                                        const double* A, int32_t asize, const double* V,
                                        const double* P, const double* fp, int64_t fes) {
  return set_impl(s, X, fx, A, asize, V, P, fp, fes, false);
}

extern "C" int32_t sevo_state_get_async(const sevo_state* s, double* X, double* fx, double* A,
                                        double* V, double* P, double* fp, double* U,
                                        double* fu) {
  if (!s) return SEVO_ERR_ARG;
  const Batch& b = s->b;
  const size_t vb = (size_t)b.R * b.NP * 8;
  if (X) SV_CUDA(get(X, b.X, b));
  if (fx) SV_CUDA(cudaMemcpyAsync(fx, b.fx, vb, cudaMemcpyDeviceToHost, b.stream));
  if (A && b.A) SV_CUDA(get(A, b.A, b));
  if (V && b.V) SV_CUDA(get(V, b.V, b));
  if (P && b.P) SV_CUDA(get(P, b.P, b));
  if (fp && b.fp) SV_CUDA(cudaMemcpyAsync(fp, b.fp, vb, cudaMemcpyDeviceToHost, b.stream));
  SV_CUDA(get_evaluated(U, fu, b));
  return SEVO_OK;
}

extern "C" int32_t sevo_state_get_shade(const sevo_state* s, double* MF, double* MCR, int32_t* k,
                                        double* F, double* CR, int32_t* kpb) {
  if (!s || !sv_has_shade(s->params.alg)) return SEVO_ERR_ARG;
  const Batch& b = s->b;
  const size_t hm = (size_t)b.R * SEVO_SHADE_H * 8, rows = (size_t)b.R * b.NP;
  if (MF) SV_CUDA(cudaMemcpyAsync(MF, b.MF, hm, cudaMemcpyDeviceToHost, b.stream));
  if (MCR) SV_CUDA(cudaMemcpyAsync(MCR, b.MCR, hm, cudaMemcpyDeviceToHost, b.stream));
  if (k) SV_CUDA(cudaMemcpyAsync(k, b.mk, (size_t)b.R * 4, cudaMemcpyDeviceToHost, b.stream));
  if (F) SV_CUDA(cudaMemcpyAsync(F, b.Fi, rows * 8, cudaMemcpyDeviceToHost, b.stream));
  if (CR) SV_CUDA(cudaMemcpyAsync(CR, b.CRi, rows * 8, cudaMemcpyDeviceToHost, b.stream));
  if (kpb) SV_CUDA(cudaMemcpyAsync(kpb, b.kpb, rows * 4, cudaMemcpyDeviceToHost, b.stream));
  SV_CUDA(cudaStreamSynchronize(b.stream));
  return SEVO_OK;
}

extern "C" int32_t sevo_state_set_shade(sevo_state* s, const double* MF, const double* MCR,
                                        const int32_t* k) {
  if (!s || !sv_has_shade(s->params.alg)) return SEVO_ERR_ARG;
  const Batch& b = s->b;
  if (k)
    for (int r = 0; r < b.R; ++r)
      if (k[r] < 0 || k[r] >= SEVO_SHADE_H) return SEVO_ERR_ARG;
  const size_t hm = (size_t)b.R * SEVO_SHADE_H * 8;
  if (MF) SV_CUDA(cudaMemcpyAsync(b.MF, MF, hm, cudaMemcpyHostToDevice, b.stream));
  if (MCR) SV_CUDA(cudaMemcpyAsync(b.MCR, MCR, hm, cudaMemcpyHostToDevice, b.stream));
  if (k) SV_CUDA(cudaMemcpyAsync(b.mk, k, (size_t)b.R * 4, cudaMemcpyHostToDevice, b.stream));
  SV_CUDA(cudaStreamSynchronize(b.stream));
  return SEVO_OK;
}

// ---- save / load: header + arrays, every array the run's next generation
// reads (counter-based draws make a resumed run bit-identical)
struct SaveHeader {
  uint32_t magic, version;
  int32_t alg, NP, D, asize;
  uint64_t seed;
  int64_t fes, gens;
  double best;
};
static const uint32_t kMagic = 0x53455642u;  // "SEVB"

static size_t save_bytes(const sevo_state* s) {
  const size_t m = (size_t)s->b.R * s->b.NP * s->b.D * 8, v = (size_t)s->b.R * s->b.NP * 8;
  size_t n = sizeof(SaveHeader) + m + v;  // X, fx
  if (s->params.alg == SEVO_DE_CTPB) n += m;              // A
  if (s->params.alg == SEVO_CSO) n += m;                   // V
  else if (sv_has_pbest(s->params.alg)) n += 2 * m + v;   // V, P, fp
  if (sv_has_shade(s->params.alg)) n += 2 * SEVO_SHADE_H * 8 + 8;  // M_F, M_CR, k
  return n;
}

// offset of the SHADE memory in a saved state: after X, fx and, for PSODE,
// the PSO component's V, P, fp
static size_t shade_offset(const sevo_state* s, size_t m, size_t v) {
  return m + v + (s->params.alg == SEVO_PSODE ? 2 * m + v : 0);
}

extern "C" int32_t sevo_state_save(const sevo_state* s, void* buf, size_t* size) {
  if (!s || !size || s->b.R != 1) return s && s->b.R != 1 ? SEVO_ERR_UNSUPPORTED : SEVO_ERR_ARG;
  const size_t need = save_bytes(s);
  if (!buf) {
    *size = need;
    return SEVO_OK;
  }
  if (*size < need) {
    *size = need;
    return SEVO_ERR_ARG;
  }
  const Batch& b = s->b;
  const size_t m = (size_t)b.NP * b.D * 8, v = (size_t)b.NP * 8;
  SaveHeader h{kMagic, 1u, s->params.alg, b.NP, b.D, 0, s->seed, s->fes, s->gens, 0.0};
  char* c = (char*)buf + sizeof(SaveHeader);
  int32_t as = 0;
  int32_t st = sevo_state_get(s, (double*)c, (double*)(c + m),
                              s->params.alg == SEVO_DE_CTPB ? (double*)(c + m + v) : nullptr, &as,
                              is_de(s->params.alg) ? nullptr : (double*)(c + m + v),
                              is_de(s->params.alg) ? nullptr : (double*)(c + 2 * m + v),
                              is_de(s->params.alg) ? nullptr : (double*)(c + 3 * m + v), nullptr,
                              nullptr, nullptr);
  if (st != SEVO_OK) return st;
  if (sv_has_shade(s->params.alg)) {  // memory after the population arrays
    char* q = c + shade_offset(s, m, v);
    int32_t k = 0;
    st = sevo_state_get_shade(s, (double*)q, (double*)(q + SEVO_SHADE_H * 8), &k, nullptr,
                              nullptr, nullptr);
    if (st != SEVO_OK) return st;
    std::memcpy(q + 2 * SEVO_SHADE_H * 8, &k, 4);
  }
  h.asize = as;
  SV_CUDA(cudaMemcpy(&h.best, b.best, 8, cudaMemcpyDeviceToHost));
  std::memcpy(buf, &h, sizeof(h));
  *size = need;
  return SEVO_OK;
}

extern "C" int32_t sevo_state_load(sevo_state* s, const void* buf, size_t size) {
  if (!s || !buf || size < sizeof(SaveHeader)) return SEVO_ERR_ARG;
  if (s->b.R != 1) return SEVO_ERR_UNSUPPORTED;
  SaveHeader h;
  std::memcpy(&h, buf, sizeof(h));
  if (h.magic != kMagic || h.version != 1u || h.alg != s->params.alg || h.NP != s->b.NP ||
      h.D != s->b.D || size < save_bytes(s))
    return SEVO_ERR_ARG;
  const size_t m = (size_t)s->b.NP * s->b.D * 8, v = (size_t)s->b.NP * 8;
  const char* c = (const char*)buf + sizeof(SaveHeader);
  const bool de = is_de(s->params.alg);
  int32_t st = sevo_state_set(s, (const double*)c, (const double*)(c + m),
                              s->params.alg == SEVO_DE_CTPB ? (const double*)(c + m + v) : nullptr,
                              h.asize, de ? nullptr : (const double*)(c + m + v),
                              de ? nullptr : (const double*)(c + 2 * m + v),
                              de ? nullptr : (const double*)(c + 3 * m + v), h.fes);
  if (st != SEVO_OK) return st;
  if (sv_has_shade(s->params.alg)) {
    const char* q = c + shade_offset(s, m, v);
    int32_t k = 0;
    std::memcpy(&k, q + 2 * SEVO_SHADE_H * 8, 4);
    st = sevo_state_set_shade(s, (const double*)q, (const double*)(q + SEVO_SHADE_H * 8), &k);
    if (st != SEVO_OK) return st;
  }
  SV_CUDA(cudaMemcpy(s->b.best, &h.best, 8, cudaMemcpyHostToDevice));
  SV_CUDA(cudaMemcpy(s->b.seeds, &h.seed, 8, cudaMemcpyHostToDevice));
  s->gens = h.gens;
  s->seed = h.seed;
  return SEVO_OK;
}
