// grid.cu -- sevo_run_grid: the experiment grid (Sec. 2.4, Listing 3: the
// runner over (problem, run) tasks).  The paper spreads tasks over a CPU
// thread pool; here tasks with the same (algorithm, dimension) advance
// together as one batch -- one launch per kernel per generation over all of
// their runs -- and the generation sequence is captured once into a CUDA
// graph that is replayed until the shared budget is spent.
#include <algorithm>
#include <map>
#include <vector>

#include "evo.cuh"

namespace {

struct GraphExec {
  cudaGraphExec_t exec = nullptr;
  ~GraphExec() {
    if (exec) cudaGraphExecDestroy(exec);
  }
};

// capture `gens` generations of batch b on its stream into an executable graph;
// *nkern receives the number of kernels in the graph (launch accounting
// counts them at every replay, not at capture)
cudaError_t capture(Batch* b, int gens, GraphExec* out, int64_t* nkern) {
  const int64_t before = sevo_kernel_launches();
  cudaError_t e = cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeRelaxed);
  if (e != cudaSuccess) return e;
  cudaError_t body = cudaSuccess;
  for (int g = 0; g < gens && body == cudaSuccess; ++g) {
    body = sv_ctl_advance(b);
    if (body == cudaSuccess) body = sv_batch_generation(b);
  }
  cudaGraph_t graph = nullptr;
  e = cudaStreamEndCapture(b->stream, &graph);
  *nkern = sevo_kernel_launches() - before;
  sv_note_launch(-*nkern);
  if (body != cudaSuccess) {
    if (graph) cudaGraphDestroy(graph);
    return body;
  }
  if (e != cudaSuccess) return e;
  e = cudaGraphInstantiate(&out->exec, graph, 0);
  cudaGraphDestroy(graph);
  return e;
}

}  // namespace

extern "C" int32_t sevo_run_grid(const sevo_grid* grid, sevo_grid_result* res, void* stream) {
  (void)stream;
  if (!grid || !res || grid->ntasks < 0 || (grid->ntasks > 0 && !grid->tasks) ||
      grid->nproblems < 1 || !grid->problems || grid->nalgs < 1 || !grid->algs)
    return SEVO_ERR_ARG;
  if (!res->best || !res->fes || !res->gens || !res->success) return SEVO_ERR_ARG;
  for (int t = 0; t < grid->ntasks; ++t) {
    const sevo_task& k = grid->tasks[t];
    if (k.problem < 0 || k.problem >= grid->nproblems || k.alg < 0 || k.alg >= grid->nalgs ||
        !grid->problems[k.problem])
      return SEVO_ERR_ARG;
  }
  for (int a = 0; a < grid->nalgs; ++a) {
    const sevo_alg_params& p = grid->algs[a];
    const bool de = sv_is_de(p.alg) || p.alg == SEVO_PSODE;  // NP >= 4
    if (p.alg == SEVO_CSO && (p.NP < 2 || (p.NP & 1))) return SEVO_ERR_ARG;
    if (p.alg < 0 || p.alg > SEVO_PSODE || p.NP > SV_MAX_NP || p.budget < 1 ||
        (de && p.NP < 4) || (!de && p.NP < 2) || !(p.lb < p.ub) || p.prec < 0 || p.prec > 3)
      return SEVO_ERR_ARG;
  }
  for (int q = 0; q < grid->nproblems; ++q) {
    int32_t st = sv_problem_ready(grid->problems[q]);
    if (st != SEVO_OK) return st;
  }
  // buckets: (alg index, D) -> task indices sorted by problem
  std::map<std::pair<int, int>, std::vector<int>> buckets;
  for (int t = 0; t < grid->ntasks; ++t) {
    const sevo_task& k = grid->tasks[t];
    buckets[{k.alg, grid->problems[k.problem]->D}].push_back(t);
  }
  cudaStream_t st;
  SV_CUDA(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  cudaEventRecord(e0, st);
  int32_t status = SEVO_OK;
  int64_t evals = 0;
  for (auto& kv : buckets) {
    std::vector<int>& tasks = kv.second;
    std::stable_sort(tasks.begin(), tasks.end(), [&](int x, int y) {
      return grid->tasks[x].problem < grid->tasks[y].problem;
    });
    const sevo_alg_params& a = grid->algs[kv.first.first];
    std::vector<const sevo_problem*> probs;
    std::vector<uint64_t> seeds;
    for (int t : tasks) {
      probs.push_back(grid->problems[grid->tasks[t].problem]);
      seeds.push_back(grid->tasks[t].seed);
    }
    Batch b{};
    status = sv_batch_alloc(&b, probs, seeds, &a, st);
    if (status != SEVO_OK) {
      sv_batch_free(&b);
      break;
    }
    cudaError_t e = sv_batch_init(&b);
    const int64_t NP = a.NP;
    const int64_t PG = b.per_gen;  // evaluations counted per generation
    const int64_t gens = (a.budget > NP) ? (a.budget - NP + PG - 1) / PG : 0;
    int G = grid->gens_per_graph > 0 ? grid->gens_per_graph : 32;
    if (G > gens) G = (int)std::max<int64_t>(gens, 1);
    int64_t done = 0;
    if (e == cudaSuccess && b.small) {  // run-per-CTA launches, no graph needed
      e = sv_batch_run_small(&b, 0ull, gens);
      done = gens;
    }
    if (e == cudaSuccess && !b.small && gens >= G && G > 0) {
      GraphExec ge;
      int64_t nk = 0;
      e = capture(&b, G, &ge, &nk);
      for (; e == cudaSuccess && done + G <= gens; done += G) {
        e = cudaGraphLaunch(ge.exec, st);
        sv_note_launch(nk);
      }
    }
    for (; e == cudaSuccess && done < gens; ++done) {
      e = sv_ctl_advance(&b);
      if (e == cudaSuccess) e = sv_batch_generation(&b);
    }
    std::vector<double> best(b.R);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(best.data(), b.best, (size_t)b.R * 8, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    const int32_t dev = (e == cudaSuccess) ? sv_batch_status(&b) : SEVO_OK;
    sv_batch_free(&b);
    if (dev != SEVO_OK) {
      status = dev;
      break;
    }
    if (e != cudaSuccess) {
      sv_set_last_cuda_error(e);
      status = (e == cudaErrorMemoryAllocation) ? SEVO_ERR_OOM : SEVO_ERR_CUDA;
      break;
    }
    const int64_t fes = std::min<int64_t>(a.budget, NP + gens * PG);
    for (size_t q = 0; q < tasks.size(); ++q) {
      const int t = tasks[q];
      res->best[t] = best[q];
      res->fes[t] = std::min<int64_t>(fes, a.budget);
      res->gens[t] = gens;
      res->success[t] = best[q] <= SEVO_SUCCESS_THRESHOLD;
    }
    evals += (int64_t)tasks.size() * (NP + gens * PG);
  }
  cudaEventRecord(e1, st);
  cudaEventSynchronize(e1);
  float ms = 0.f;
  cudaEventElapsedTime(&ms, e0, e1);
  res->wall_ms = ms;
  res->evals = evals;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaStreamDestroy(st);
  return status;
}
