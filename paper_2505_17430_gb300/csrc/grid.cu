// grid.cu -- sevo_run_grid: the experiment grid (Sec. 2.4, Listing 3: the
// runner over (problem, run) tasks).  The paper spreads tasks over a CPU
// thread pool; here tasks with the same (algorithm, dimension) advance
// together as one batch -- one launch per kernel per generation over all of
// their runs -- whose generation sequence is captured once into a CUDA graph
// that is replayed until the shared budget is spent, and the batches run
// side by side, each on its own stream forked from the caller's (small-D
// batches alone would leave most of the GPU idle).
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

namespace {

struct Bucket {
  Bucket() = default;
  Bucket(const Bucket&) = delete;
  Bucket& operator=(const Bucket&) = delete;
  int alg_index = 0;
  std::vector<int> tasks;
  Batch b{};
  bool allocated = false;
  cudaStream_t st = nullptr;
  GraphExec ge;
  int64_t nk = 0;  // kernels per replay
  int G = 0;       // generations per replay
  int64_t gens = 0, done = 0;
  cudaError_t e = cudaSuccess;
  std::vector<double> best;
};

void free_bucket(Bucket& k) {
  if (k.allocated) sv_batch_free(&k.b);
  k.allocated = false;
  if (k.ge.exec) {
    cudaGraphExecDestroy(k.ge.exec);
    k.ge.exec = nullptr;
  }
  if (k.st) cudaStreamDestroy(k.st);
  k.st = nullptr;
}

}  // namespace

extern "C" int32_t sevo_run_grid(const sevo_grid* grid, sevo_grid_result* res, void* stream) {
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
  std::map<std::pair<int, int>, std::vector<int>> groups;
  for (int t = 0; t < grid->ntasks; ++t) {
    const sevo_task& k = grid->tasks[t];
    groups[{k.alg, grid->problems[k.problem]->D}].push_back(t);
  }
  std::vector<Bucket> bk(groups.size());
  {
    size_t i = 0;
    for (auto& kv : groups) {
      bk[i].alg_index = kv.first.first;
      bk[i].tasks = kv.second;
      std::stable_sort(bk[i].tasks.begin(), bk[i].tasks.end(), [&](int x, int y) {
        return grid->tasks[x].problem < grid->tasks[y].problem;
      });
      ++i;
    }
  }
  // the caller's stream brackets the whole grid: every bucket's stream
  // starts after e0 on it, and e1 on it follows every bucket's last work
  cudaStream_t caller = (cudaStream_t)stream;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  int32_t status = SEVO_OK;
  cudaError_t ce = cudaEventCreate(&e0);
  if (ce == cudaSuccess) ce = cudaEventCreate(&e1);
  if (ce == cudaSuccess) ce = cudaEventRecord(e0, caller);
  for (auto& k : bk) {
    if (ce != cudaSuccess || status != SEVO_OK) break;
    if ((ce = cudaStreamCreateWithFlags(&k.st, cudaStreamNonBlocking)) != cudaSuccess) break;
    if ((ce = cudaStreamWaitEvent(k.st, e0, 0)) != cudaSuccess) break;
    const sevo_alg_params& a = grid->algs[k.alg_index];
    std::vector<const sevo_problem*> probs;
    std::vector<uint64_t> seeds;
    for (int t : k.tasks) {
      probs.push_back(grid->problems[grid->tasks[t].problem]);
      seeds.push_back(grid->tasks[t].seed);
    }
    status = sv_batch_alloc(&k.b, probs, seeds, &a, k.st);
    k.allocated = true;
    if (status != SEVO_OK) break;
    k.e = sv_batch_init(&k.b);
    const int64_t NP = a.NP, PG = k.b.per_gen;  // evaluations counted per generation
    k.gens = (a.budget > NP) ? (a.budget - NP + PG - 1) / PG : 0;
    k.G = grid->gens_per_graph > 0 ? grid->gens_per_graph : 32;
    if (k.G > k.gens) k.G = (int)std::max<int64_t>(k.gens, 1);
    if (k.e == cudaSuccess && k.b.small) {  // run-per-CTA launches, no graph needed
      k.e = sv_batch_run_small(&k.b, 0ull, k.gens);
      k.done = k.gens;
    }
    if (k.e == cudaSuccess && !k.b.small && k.gens >= k.G && k.G > 0)
      k.e = capture(&k.b, k.G, &k.ge, &k.nk);
  }
  // replays, round robin over the buckets so that every stream has work
  // queued while the others run
  for (bool more = (ce == cudaSuccess && status == SEVO_OK); more;) {
    more = false;
    for (auto& k : bk) {
      if (k.e != cudaSuccess || !k.ge.exec || k.done + k.G > k.gens) continue;
      k.e = cudaGraphLaunch(k.ge.exec, k.st);
      sv_note_launch(k.nk);
      k.done += k.G;
      more = more || (k.done + k.G <= k.gens);
    }
  }
  int64_t evals = 0;
  for (auto& k : bk) {
    if (ce != cudaSuccess || status != SEVO_OK || !k.allocated) break;
    for (; k.e == cudaSuccess && k.done < k.gens; ++k.done) {
      k.e = sv_ctl_advance(&k.b);
      if (k.e == cudaSuccess) k.e = sv_batch_generation(&k.b);
    }
    k.best.assign(k.b.R, 0.0);
    if (k.e == cudaSuccess)
      k.e = cudaMemcpyAsync(k.best.data(), k.b.best, (size_t)k.b.R * 8, cudaMemcpyDeviceToHost,
                            k.st);
    cudaEvent_t done = nullptr;
    if (k.e == cudaSuccess) k.e = cudaEventCreateWithFlags(&done, cudaEventDisableTiming);
    if (k.e == cudaSuccess) k.e = cudaEventRecord(done, k.st);
    if (k.e == cudaSuccess) k.e = cudaStreamWaitEvent(caller, done, 0);
    if (done) cudaEventDestroy(done);
  }
  if (ce == cudaSuccess) ce = cudaEventRecord(e1, caller);
  if (ce == cudaSuccess) ce = cudaEventSynchronize(e1);
  for (auto& k : bk) {
    if (!k.allocated || status != SEVO_OK) break;
    const int32_t dev = (k.e == cudaSuccess && ce == cudaSuccess) ? sv_batch_status(&k.b)
                                                                   : SEVO_OK;
    if (dev != SEVO_OK) {
      status = dev;
      break;
    }
    if (k.e != cudaSuccess) {
      sv_set_last_cuda_error(k.e);
      status = (k.e == cudaErrorMemoryAllocation) ? SEVO_ERR_OOM : SEVO_ERR_CUDA;
      break;
    }
    const sevo_alg_params& a = grid->algs[k.alg_index];
    const int64_t NP = a.NP, PG = k.b.per_gen;
    const int64_t fes = std::min<int64_t>(a.budget, NP + k.gens * PG);
    for (size_t q = 0; q < k.tasks.size(); ++q) {
      const int t = k.tasks[q];
      res->best[t] = k.best[q];
      res->fes[t] = fes;
      res->gens[t] = k.gens;
      res->success[t] = k.best[q] <= SEVO_SUCCESS_THRESHOLD;
    }
    evals += (int64_t)k.tasks.size() * (NP + k.gens * PG);
  }
  if (ce != cudaSuccess && status == SEVO_OK) {
    sv_set_last_cuda_error(ce);
    status = SEVO_ERR_CUDA;
  }
  float ms = 0.f;
  if (ce == cudaSuccess) cudaEventElapsedTime(&ms, e0, e1);
  res->wall_ms = ms;
  res->evals = evals;
  // a failure part way: let whatever was queued finish before freeing
  for (auto& k : bk)
    if (k.st) cudaStreamSynchronize(k.st);
  for (auto& k : bk) free_bucket(k);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  return status;
}
