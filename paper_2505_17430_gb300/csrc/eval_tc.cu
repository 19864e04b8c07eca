// eval_tc.cu -- placeholder until the tcgen05 kernel lands.
#include "kernels.cuh"
size_t sv_eval_tc_scratch_bytes(const sevo_problem*, int, int64_t) { return 0; }
cudaError_t sv_eval_tc(const sevo_problem*, int, const double*, int64_t, int64_t, double*, EvalAux,
                       void*, size_t, uint32_t*, cudaStream_t) {
  return cudaErrorNotSupported;
}
