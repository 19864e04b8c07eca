// evo.cu -- placeholder for the DE/PSO generation kernels.
#include "kernels.cuh"
extern "C" {
int32_t sevo_state_create(const sevo_problem*, const sevo_alg_params*, uint64_t, void*, sevo_state**) { return SEVO_ERR_UNSUPPORTED; }
int32_t sevo_state_destroy(sevo_state*) { return SEVO_ERR_UNSUPPORTED; }
int32_t sevo_de_step(sevo_state*, uint64_t) { return SEVO_ERR_UNSUPPORTED; }
int32_t sevo_pso_step(sevo_state*, uint64_t) { return SEVO_ERR_UNSUPPORTED; }
int32_t sevo_state_result(const sevo_state*, double*, int64_t*, int64_t*, int64_t*) { return SEVO_ERR_UNSUPPORTED; }
int32_t sevo_state_get(const sevo_state*, double*, double*, double*, int32_t*, double*, double*, double*, double*, double*, int32_t*) { return SEVO_ERR_UNSUPPORTED; }
int32_t sevo_state_set(sevo_state*, const double*, const double*, const double*, int32_t, const double*, const double*, const double*, int64_t) { return SEVO_ERR_UNSUPPORTED; }
int32_t sevo_state_save(const sevo_state*, void*, size_t*) { return SEVO_ERR_UNSUPPORTED; }
int32_t sevo_state_load(sevo_state*, const void*, size_t) { return SEVO_ERR_UNSUPPORTED; }
int32_t sevo_run_grid(const sevo_grid*, sevo_grid_result*, void*) { return SEVO_ERR_UNSUPPORTED; }
}
