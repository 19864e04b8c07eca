// noalloc.cu -- sevo_evaluate_noalloc: sevo_evaluate with its scratch in one
// fixed device array instead of a stream-ordered allocation, for callers
// that cannot allocate device memory at the point of the call.
#include "kernels.cuh"

// one array per device that loads the library (held until process exit)
static __device__ __align__(256) unsigned char g_noalloc_scratch[SEVO_NOALLOC_SCRATCH_BYTES];

namespace {
// the array's device address in the current context, looked up on every
// call (host code cannot use the symbol itself; the lookup allocates nothing,
// and an address kept from an earlier context would be stale after a device
// reset)
int32_t scratch_address(void** out) {
  void* p = nullptr;
  const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
  if (e != cudaSuccess || !p) {
    sv_set_last_cuda_error(e);
    return SEVO_ERR_CUDA;
  }
  *out = p;
  return SEVO_OK;
}
}  // namespace

extern "C" int32_t sevo_evaluate_noalloc(const sevo_problem* p, const double* pop, int64_t N,
                                         int32_t D, int64_t ld, double* out, int32_t prec,
                                         void* stream) {
  if (!p || !pop || !out || N < 0 || D != p->D || ld < D) return SEVO_ERR_ARG;
  if (prec < SEVO_FP64 || prec > SEVO_FP32) return SEVO_ERR_ARG;
  if (((uintptr_t)pop & 7) || ((uintptr_t)out & 7)) return SEVO_ERR_ARG;
  if (N > SEVO_NOALLOC_MAX_ROWS) return SEVO_ERR_UNSUPPORTED;
  // the problem's device copy must already exist here: making it allocates
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) return SEVO_ERR_CUDA;
  // checked under the upload lock: another thread may be making the copy
  if (sv_problem_has_device_copy(p, dev) != SEVO_OK) return SEVO_ERR_STATE;
  if (N == 0) return SEVO_OK;
  const bool comp = sv_weighted_family(p->family);
  if (sv_eval_scratch_bytes(p->D, comp, prec, N) > SEVO_NOALLOC_SCRATCH_BYTES)
    return SEVO_ERR_UNSUPPORTED;
  void* base = nullptr;
  int32_t st = scratch_address(&base);
  if (st != SEVO_OK) return st;
  EvalScratch sc;
  sv_eval_scratch_carve(base, p->D, comp, prec, N, &sc);
  TcSegment seg{p, 0, N};
  cudaError_t e = sv_eval_segments(&seg, 1, prec, pop, ld, out, sc, (cudaStream_t)stream);
  if (e != cudaSuccess) {
    sv_set_last_cuda_error(e);
    return SEVO_ERR_CUDA;
  }
  return SEVO_OK;
}
