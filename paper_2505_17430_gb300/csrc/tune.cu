// tune.cu -- measured launch choices (autotuning), cached per GPU model.
//
// A choice (today: the N-tile width of the large-D rotation GEMM) is keyed
// by (kind, D, row bucket, precision); the row bucket is the row count
// rounded up to a power of two.  A miss is measured by the caller with CUDA
// events on its own data (every candidate gives the same result bits, only
// the time differs) and stored here: in memory for the process and as one
// text line in a cache file,
//   <kind> <D> <row bucket> <prec> <choice> <ms of each candidate...>
// whose path is $SEVO_TUNE_FILE, else $XDG_CACHE_HOME/sevo/tune-<gpu>.txt,
// else $HOME/.cache/sevo/tune-<gpu>.txt (<gpu> = the device name with
// spaces replaced).  The file is read on first use and after
// sevo_set_policy(SEVO_POLICY_AUTOTUNE, 2); a file that cannot be read or
// written leaves the cache in memory only.
#include <sys/stat.h>

#include <atomic>
#include <cerrno>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <tuple>

#include "kernels.cuh"

namespace {

using Key = std::tuple<int, int, int64_t, int>;  // kind, D, row bucket, prec

std::mutex g_mu;
std::map<Key, int> g_table;
bool g_loaded = false;
std::string g_path;
std::atomic<int> g_policy{1};

int64_t bucket(int64_t rows) {
  int64_t b = 1;
  while (b < rows) b <<= 1;
  return b;
}

std::string gpu_tag() {
  int dev = 0;
  cudaDeviceProp prop;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaGetDeviceProperties(&prop, dev) != cudaSuccess)
    return "unknown";
  std::string s(prop.name);
  for (char& ch : s)
    if (ch == ' ' || ch == '/') ch = '_';
  return s;
}

void mkdirs(const std::string& dir) {
  for (size_t i = 1; i <= dir.size(); ++i)
    if (i == dir.size() || dir[i] == '/') mkdir(dir.substr(0, i).c_str(), 0755);
}

std::string cache_path() {
  if (const char* f = std::getenv("SEVO_TUNE_FILE")) return f;
  std::string dir;
  if (const char* x = std::getenv("XDG_CACHE_HOME"))
    dir = std::string(x) + "/sevo";
  else if (const char* h = std::getenv("HOME"))
    dir = std::string(h) + "/.cache/sevo";
  else
    return "";
  mkdirs(dir);
  return dir + "/tune-" + gpu_tag() + ".txt";
}

// (under g_mu)
void load() {
  g_table.clear();
  g_path = cache_path();
  g_loaded = true;
  if (g_path.empty()) return;
  FILE* f = std::fopen(g_path.c_str(), "r");
  if (!f) return;
  char line[512];
  while (std::fgets(line, sizeof line, f)) {
    int kind, D, prec, choice;
    long long rb;
    if (std::sscanf(line, "%d %d %lld %d %d", &kind, &D, &rb, &prec, &choice) == 5)
      g_table[Key{kind, D, (int64_t)rb, prec}] = choice;
  }
  std::fclose(f);
}

}  // namespace

int sv_policy_autotune() { return g_policy.load(); }

int32_t sv_tune_set_policy(int64_t value) {
  if (value < 0 || value > 2) return SEVO_ERR_ARG;
  if (value == 2) {
    std::lock_guard<std::mutex> lk(g_mu);
    g_loaded = false;  // forget, and read the file again on next use
    g_table.clear();
    value = 1;
  }
  g_policy.store((int)value);
  return SEVO_OK;
}

int sv_tune_lookup(int kind, int D, int64_t rows, int prec) {
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_loaded) load();
  auto it = g_table.find(Key{kind, D, bucket(rows), prec});
  return it == g_table.end() ? 0 : it->second;
}

void sv_tune_store(int kind, int D, int64_t rows, int prec, int choice, const float* ms,
                   const int* cand, int n) {
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_loaded) load();
  const int64_t rb = bucket(rows);
  g_table[Key{kind, D, rb, prec}] = choice;
  if (g_path.empty()) return;
  FILE* f = std::fopen(g_path.c_str(), "a");
  if (!f) return;
  std::fprintf(f, "%d %d %lld %d %d", kind, D, (long long)rb, prec, choice);
  for (int i = 0; i < n; ++i) std::fprintf(f, " %d:%.4f", cand[i], ms[i]);
  std::fprintf(f, "\n");
  std::fclose(f);
}
