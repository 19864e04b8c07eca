// trace.cu -- per-kernel device timing with CUDA events on the launching
// stream (sevo_trace_*), and the launch accounting that every launch site
// reports through sv_trace_end.
#include <algorithm>
#include <atomic>
#include <mutex>
#include <vector>

#include "sevo_internal.cuh"

namespace {

struct Pending {
  cudaEvent_t a, b;
  int kind, dev, stream;
};

struct Span {
  int kind, stream;
  double t0, t1;
};

std::mutex g_mu;
std::atomic<bool> g_on{false};
std::vector<Pending> g_open;     // indexed by token
std::vector<int> g_free_tokens;  // reusable slots of g_open
std::vector<std::pair<int, cudaEvent_t>> g_pool;  // (device, event) ready for reuse
int64_t g_count[SEVO_TRACE_KINDS];
double g_ms[SEVO_TRACE_KINDS];
// timeline (tracing mode 2): every drained launch as (kind, stream, start,
// end) in ms from the start event of the first launch traced since enable
bool g_keep = false;
cudaEvent_t g_origin = nullptr;
int g_origin_dev = -1;
std::vector<Span> g_spans;
std::vector<cudaStream_t> g_streams;  // stream ids: order of first appearance
constexpr size_t kMaxSpans = size_t(1) << 20;

const char* const k_names[SEVO_TRACE_KINDS] = {
    "eval_tc_fused", "eval_cc", "refine", "compose", "convert", "gemm_big", "combine", "init",
    "de_trial", "de_rank", "de_select", "de_apply", "pso_move", "pso_update", "pso_copy",
    "control", "small_run"};

cudaEvent_t take_event(int dev) {
  for (size_t i = 0; i < g_pool.size(); ++i) {
    if (g_pool[i].first == dev) {
      cudaEvent_t e = g_pool[i].second;
      g_pool[i] = g_pool.back();
      g_pool.pop_back();
      return e;
    }
  }
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
  return e;
}

// fold finished records into the totals (g_mu held); returns the first error
cudaError_t drain_locked() {
  cudaError_t first = cudaSuccess;
  for (size_t t = 0; t < g_open.size(); ++t) {
    Pending& p = g_open[t];
    if (!p.a) continue;
    cudaError_t e = cudaEventSynchronize(p.b);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, p.a, p.b);
    if (e == cudaSuccess) {
      g_count[p.kind] += 1;
      g_ms[p.kind] += ms;
      float s0 = 0.f;
      if (g_keep && g_origin && p.dev == g_origin_dev && g_spans.size() < kMaxSpans &&
          (p.a == g_origin || cudaEventElapsedTime(&s0, g_origin, p.a) == cudaSuccess))
        g_spans.push_back({p.kind, p.stream, (double)s0, (double)s0 + ms});
    } else if (first == cudaSuccess) {
      first = e;
    }
    if (p.a == g_origin) {
      p.a = nullptr;  // kept as the origin until tracing restarts
      g_pool.push_back({p.dev, p.b});
      p.b = nullptr;
      g_free_tokens.push_back((int)t);
      continue;
    }
    g_pool.push_back({p.dev, p.a});
    g_pool.push_back({p.dev, p.b});
    p.a = p.b = nullptr;
    g_free_tokens.push_back((int)t);
  }
  return first;
}

}  // namespace

int sv_trace_begin(int kind, cudaStream_t st) {
  if (!g_on.load(std::memory_order_relaxed)) return -1;
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(st, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) {
    cudaGetLastError();
    return -1;
  }
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return -1;
  std::lock_guard<std::mutex> lk(g_mu);
  if (g_open.size() - g_free_tokens.size() > 65536) drain_locked();  // bound the backlog
  int sid = -1;
  if (g_keep) {
    for (size_t i = 0; i < g_streams.size() && sid < 0; ++i)
      if (g_streams[i] == st) sid = (int)i;
    if (sid < 0) {
      sid = (int)g_streams.size();
      g_streams.push_back(st);
    }
  }
  Pending p{take_event(dev), take_event(dev), kind, dev, sid};
  if (!p.a || !p.b || cudaEventRecord(p.a, st) != cudaSuccess) {
    if (p.a) g_pool.push_back({dev, p.a});
    if (p.b) g_pool.push_back({dev, p.b});
    return -1;
  }
  if (g_keep && !g_origin) {
    g_origin = p.a;
    g_origin_dev = dev;
  }
  int tok;
  if (!g_free_tokens.empty()) {
    tok = g_free_tokens.back();
    g_free_tokens.pop_back();
    g_open[tok] = p;
  } else {
    tok = (int)g_open.size();
    g_open.push_back(p);
  }
  return tok;
}

void sv_trace_end(int token, cudaStream_t st) {
  sv_note_launch();
  if (token < 0) return;
  std::lock_guard<std::mutex> lk(g_mu);
  if (token >= (int)g_open.size() || !g_open[token].b) return;
  if (cudaEventRecord(g_open[token].b, st) != cudaSuccess) {
    // unusable record: return its events and slot
    Pending& p = g_open[token];
    g_pool.push_back({p.dev, p.a});
    g_pool.push_back({p.dev, p.b});
    p.a = p.b = nullptr;
    g_free_tokens.push_back(token);
  }
}

extern "C" int32_t sevo_trace_enable(int32_t on) {
  if (on < 0 || on > 2) return SEVO_ERR_ARG;
  std::lock_guard<std::mutex> lk(g_mu);
  if (on) {
    drain_locked();
    for (int k = 0; k < SEVO_TRACE_KINDS; ++k) {
      g_count[k] = 0;
      g_ms[k] = 0.0;
    }
    if (g_origin) g_pool.push_back({g_origin_dev, g_origin});
    g_origin = nullptr;
    g_origin_dev = -1;
    g_spans.clear();
    g_streams.clear();
    g_keep = on == 2;
  }
  g_on.store(on != 0);
  return SEVO_OK;
}

extern "C" int64_t sevo_trace_timeline(int64_t cap, int32_t* kinds, int32_t* streams, double* t0,
                                       double* t1) {
  if (cap < 0 || (cap > 0 && (!kinds || !streams || !t0 || !t1))) return SEVO_ERR_ARG;
  std::lock_guard<std::mutex> lk(g_mu);
  if (drain_locked() != cudaSuccess) return SEVO_ERR_CUDA;
  std::vector<Span> v(g_spans);
  std::stable_sort(v.begin(), v.end(), [](const Span& x, const Span& y) { return x.t0 < y.t0; });
  for (int64_t i = 0; i < cap && i < (int64_t)v.size(); ++i) {
    kinds[i] = v[i].kind;
    streams[i] = v[i].stream;
    t0[i] = v[i].t0;
    t1[i] = v[i].t1;
  }
  return (int64_t)v.size();
}

extern "C" int32_t sevo_trace_read(int64_t* counts, double* ms) {
  std::lock_guard<std::mutex> lk(g_mu);
  const cudaError_t e = drain_locked();
  for (int k = 0; k < SEVO_TRACE_KINDS; ++k) {
    if (counts) counts[k] = g_count[k];
    if (ms) ms[k] = g_ms[k];
  }
  return e == cudaSuccess ? SEVO_OK : SEVO_ERR_CUDA;
}

extern "C" const char* sevo_trace_name(int32_t kind) {
  return (kind >= 0 && kind < SEVO_TRACE_KINDS) ? k_names[kind] : "";
}
