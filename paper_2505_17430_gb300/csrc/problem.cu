// problem.cu -- seeded instance generation on the host and upload of the
// device descriptor (Sec. 1 and Sec. 2.3: each problem yields seeded random
// instances).  The instance definitions (shift, rotation, hybrid grouping,
// composition parameters) are the library's readings of the paper, stated in
// include/sevo.h at sevo_problem_create.
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <thread>
#include <vector>

#include "kernels.cuh"

static thread_local cudaError_t g_last_cuda = cudaSuccess;
void sv_set_last_cuda_error(cudaError_t e) { g_last_cuda = e; }
extern "C" const char* sevo_last_cuda_error(void) {
  return g_last_cuda == cudaSuccess ? "" : cudaGetErrorString(g_last_cuda);
}

extern "C" const char* sevo_strerror(int32_t s) {
  switch (s) {
    case SEVO_OK: return "ok";
    case SEVO_ERR_ARG: return "invalid argument";
    case SEVO_ERR_CUDA: return "CUDA runtime error";
    case SEVO_ERR_OOM: return "out of memory";
    case SEVO_ERR_TIMEOUT: return "a bounded device wait timed out";
    case SEVO_ERR_NAN: return "non-finite value in the input population";
    case SEVO_ERR_UNSUPPORTED: return "size or mode not supported";
    case SEVO_ERR_STATE: return "object in the wrong state for this call";
    default: return "unknown status";
  }
}

extern "C" int32_t sevo_version(void) { return 100; }

#include <atomic>
static std::atomic<int64_t> g_launches{0};
void sv_note_launch(int64_t n) { g_launches.fetch_add(n, std::memory_order_relaxed); }
extern "C" int64_t sevo_kernel_launches(void) { return g_launches.load(); }

// ---------------------------------------------------------------- helpers
namespace {

int n_workers() {
  unsigned h = std::thread::hardware_concurrency();
  return h == 0 ? 1 : (int)(h > 64 ? 64 : h);
}

// run f(lo, hi) over [0, n) split into contiguous blocks on worker threads
template <class F>
void parallel_blocks(int64_t n, int64_t min_block, F&& f) {
  int nw = n_workers();
  int64_t nb = (n + min_block - 1) / min_block;
  if (nb > nw) nb = nw;
  if (nb <= 1) {
    f((int64_t)0, n);
    return;
  }
  std::vector<std::thread> th;
  int64_t step = (n + nb - 1) / nb;
  for (int64_t b = 1; b < nb; ++b) {
    int64_t lo = b * step, hi = std::min(n, lo + step);
    if (lo < hi) th.emplace_back([&f, lo, hi] { f(lo, hi); });
  }
  f((int64_t)0, std::min(n, step));
  for (auto& t : th) t.join();
}

void gen_shift(uint64_t seed, int D, int comp, double* o) {
  for (int j = 0; j < D; ++j) {
    uint4 w = sv_draw(seed, (uint32_t)(j >> 1), 0u, (uint32_t)D, SV_P_SHIFT, (uint32_t)comp);
    double u = (j & 1) ? sv_u53(w.z, w.w) : sv_u53(w.x, w.y);
    o[j] = -80.0 + 160.0 * u;
  }
}

// standard normal entries by Box-Muller; entry e uses the pair call e>>1
void gen_gauss_colmajor(uint64_t seed, int D, int comp, double* Acol) {
  const int64_t n = (int64_t)D * D;
  parallel_blocks(n / 2 + 1, 4096, [&](int64_t lo, int64_t hi) {
    for (int64_t pr = lo; pr < hi; ++pr) {
      uint4 w = sv_draw(seed, (uint32_t)pr, (uint32_t)((uint64_t)pr >> 32), (uint32_t)D,
                        SV_P_ROT, (uint32_t)comp);
      double u1 = sv_u53(w.x, w.y), u2 = sv_u53(w.z, w.w);
      double R = std::sqrt(-2.0 * std::log(1.0 - u1));
      double th = 6.28318530717958647692 * u2;
      for (int t = 0; t < 2; ++t) {
        int64_t e = 2 * pr + t;
        if (e >= n) break;
        int64_t r = e / D, k = e % D;  // G[r][k]
        Acol[k * D + r] = t ? R * std::sin(th) : R * std::cos(th);
      }
    }
  });
}

// Q of the QR with positive diagonal of R, by classical Gram-Schmidt with one
// re-orthogonalisation pass per column ("twice is enough"); the diagonal of
// R is the norm of the projected column, hence positive.  In/out column-major.
void qr_q_cgs2(double* A, int D, double* Qcol) {
  std::vector<double> r((size_t)D);
  for (int k = 0; k < D; ++k) {
    double* a = A + (size_t)k * D;
    for (int pass = 0; pass < 2; ++pass) {
      if (k == 0) break;
      parallel_blocks(k, 64, [&](int64_t lo, int64_t hi) {
        for (int64_t j = lo; j < hi; ++j) {
          const double* q = Qcol + (size_t)j * D;
          double s = 0.0;
          for (int i = 0; i < D; ++i) s += q[i] * a[i];
          r[j] = s;
        }
      });
      parallel_blocks(D, 256, [&](int64_t lo, int64_t hi) {
        for (int j = 0; j < k; ++j) {
          const double* q = Qcol + (size_t)j * D;
          const double rj = r[j];
          for (int64_t i = lo; i < hi; ++i) a[i] -= rj * q[i];
        }
      });
    }
    double nrm = 0.0;
    for (int i = 0; i < D; ++i) nrm += a[i] * a[i];
    nrm = std::sqrt(nrm);
    double* q = Qcol + (size_t)k * D;
    for (int i = 0; i < D; ++i) q[i] = a[i] / nrm;
  }
}

// M (row-major) = Q; Qcol[k*D + r] = Q[r][k]
void gen_rotation(uint64_t seed, int D, int comp, double* M) {
  std::vector<double> A((size_t)D * D), Qc((size_t)D * D);
  gen_gauss_colmajor(seed, D, comp, A.data());
  qr_q_cgs2(A.data(), D, Qc.data());
  for (int r = 0; r < D; ++r)
    for (int k = 0; k < D; ++k) M[(size_t)r * D + k] = Qc[(size_t)k * D + r];
}

void gen_perm(uint64_t seed, int D, int32_t* perm, uint32_t salt = 0) {
  for (int i = 0; i < D; ++i) perm[i] = i;
  for (int i = D - 1; i >= 1; --i) {
    uint4 w = sv_draw(seed, (uint32_t)i, 0u, (uint32_t)D, SV_P_PERM, salt);
    int j = (int)sv_below(w.x, (uint32_t)(i + 1));
    int32_t t = perm[i];
    perm[i] = perm[j];
    perm[j] = t;
  }
}

// Schwefel: s = argmax_{t in [0,500]} t sin sqrt t; with u = sqrt t the
// stationarity condition is tan u = -u/2; Newton on sin u + (u/2) cos u.
double schwefel_shift() {
  double u = 20.5;
  for (int it = 0; it < 100; ++it) {
    double f = std::sin(u) + 0.5 * u * std::cos(u);
    double df = 1.5 * std::cos(u) - 0.5 * u * std::sin(u);
    double du = f / df;
    u -= du;
    if (std::fabs(du) < 1e-16 * u) break;
  }
  return u * u;
}

// round-to-nearest (ties away) to TF32: keep 10 explicit mantissa bits
float to_tf32(float x) {
  uint32_t u;
  std::memcpy(&u, &x, 4);
  if ((u & 0x7F800000u) == 0x7F800000u) return x;
  u = (u + 0x1000u) & 0xFFFFE000u;
  float y;
  std::memcpy(&y, &u, 4);
  return y;
}

int round_up(int x, int m) { return (x + m - 1) / m * m; }

}  // namespace

// ---------------------------------------------------------------- upload
static int32_t upload(sevo_problem* p) {
  const int D = p->D, nc = p->ncomp;
  ProblemDev& h = p->host_desc;
  std::memset(&h, 0, sizeof(h));
  h.family = p->family;
  h.D = D;
  h.ncomp = nc;
  h.weighted = (p->family == SEVO_COMPOSITION || p->family == SEVO_COMP_HYBRID) ? 1 : 0;
  h.kpad = round_up(D, 64);
  h.npad = (D <= 128) ? round_up(D, 16) : round_up(D, 128);
  h.fstar = p->fstar;
  h.sch_s = schwefel_shift();
  h.sch_c = h.sch_s * std::sin(std::sqrt(h.sch_s));
  {
    double B = std::sqrt(h.sch_s);
    h.sch_s32 = (float)h.sch_s;
    h.sch_B32 = (float)B;
    h.sch_sinB32 = (float)std::sin(B);
    h.sch_cosB32 = (float)std::cos(B);
    h.sch_h032 = (float)(std::sin(B) + 0.5 * B * std::cos(B));
    h.sch_c32 = (float)h.sch_c;
  }
  // groups of every component
  for (int c = 0; c < nc; ++c) {
    int ng = 1;
    const int32_t *gs = nullptr, *gb = nullptr;
    int32_t one_size = D, one_body = p->family;
    if (p->family == SEVO_HYBRID) {
      ng = p->ngroups;
      gs = p->gsize;
      gb = p->gbody;
    } else if (p->family == SEVO_COMP_HYBRID) {
      ng = p->cK[c];
      gs = p->cgsize[c];
      gb = p->cgbody[c];
    } else {
      if (p->family == SEVO_COMPOSITION) one_body = p->cbody[c];
      gs = &one_size;
      gb = &one_body;
    }
    h.ngc[c] = ng;
    h.gstart[c][0] = 0;
    for (int g = 0; g < ng; ++g) {
      h.gstart[c][g + 1] = h.gstart[c][g] + gs[g];
      h.gbody[c][g] = gb[g];
    }
  }
  for (int c = 0; c < nc; ++c) {
    h.sigma[c] = p->sigma[c];
    h.lambda[c] = p->lambda[c];
    h.bias[c] = p->bias[c];
  }
  // per-component byte layout
  const size_t DD = (size_t)D * D, NK = (size_t)h.npad * h.kpad;
  auto al = [](size_t b) { return (b + 255) & ~(size_t)255; };
  const size_t per = al(D * 8) + al(DD * 8) + al(DD * 4) + al(NK * 4) + 2 * al(NK * 2) +
                     al(D * 8) + al(D * 4) + al(D * 4) + 2 * al(D * 4);
  // six TMA descriptors per component slot: fp32, bf16 hi and lo, each with
  // full-height and 64-row boxes
  constexpr size_t kMaps = 6 * SV_MAXC;
  p->dev_bytes = per * nc + al(kMaps * sizeof(CUtensorMap)) + al(sizeof(ProblemDev));
  SV_CUDA(cudaMalloc(&p->dev_block, p->dev_bytes));
  std::vector<unsigned char> blob(p->dev_bytes, 0);
  char* base = (char*)p->dev_block;
  size_t off = 0;
  bool overflow = false;
  // placement in the block; a request past its size is refused (offset 0,
  // reported below) rather than written out of bounds
  auto take = [&](size_t b) {
    if (off + al(b) > p->dev_bytes) {
      overflow = true;
      return (size_t)0;
    }
    size_t o = off;
    off += al(b);
    return o;
  };
  for (int c = 0; c < nc; ++c) {
    const double* o = p->o_h + (size_t)c * D;
    const double* M = p->M_h + (size_t)c * DD;
    size_t oo = take(D * 8), omt = take(DD * 8), omt32 = take(DD * 4), om32 = take(NK * 4),
           ohi = take(NK * 2), olo = take(NK * 2), oa64 = take(D * 8), oa32 = take(D * 4),
           ogid = take(D * 4), ooh = take(D * 4), ool = take(D * 4);
    float* oh = (float*)&blob[ooh];
    float* ol = (float*)&blob[ool];
    for (int j = 0; j < D; ++j) sv_split_hi_lo(o[j], oh[j], ol[j]);
    std::memcpy(&blob[oo], o, D * 8);
    double* mt = (double*)&blob[omt];
    float* mt32 = (float*)&blob[omt32];
    float* m32 = (float*)&blob[om32];
    __nv_bfloat16* mhi = (__nv_bfloat16*)&blob[ohi];
    __nv_bfloat16* mlo = (__nv_bfloat16*)&blob[olo];
    for (int i = 0; i < D; ++i)
      for (int j = 0; j < D; ++j) {
        double v = M[(size_t)i * D + j];
        mt[(size_t)j * D + i] = v;
        mt32[(size_t)j * D + i] = (float)v;
        m32[(size_t)i * h.kpad + j] = to_tf32((float)v);
        float hi = __bfloat162float(__float2bfloat16_rn((float)v));
        mhi[(size_t)i * h.kpad + j] = __float2bfloat16_rn((float)v);
        mlo[(size_t)i * h.kpad + j] = __float2bfloat16_rn((float)(v - (double)hi));
      }
    // zero padding of bf16 (blob is zero-filled; bf16 zero is all-zero bits)
    double* a64 = (double*)&blob[oa64];
    float* a32 = (float*)&blob[oa32];
    int32_t* gid = (int32_t*)&blob[ogid];
    for (int g = 0; g < h.ngc[c]; ++g) {
      int b = h.gbody[c][g];
      int s = h.gstart[c][g], e = h.gstart[c][g + 1], n = e - s;
      for (int i = s; i < e; ++i) {
        int pos = i - s + 1;  // 1-based position in the group
        double v = 0.0;
        if (b == SEVO_ELLIPSOID)
          v = (n > 1) ? std::pow(10.0, 6.0 * (double)(pos - 1) / (double)(n - 1)) : 1.0;
        else if (b == SEVO_GRIEWANK)
          v = std::sqrt((double)pos);
        a64[i] = v;
        a32[i] = (float)v;
        gid[i] = g;
      }
    }
    h.o[c] = (const double*)(base + oo);
    h.MT64[c] = (const double*)(base + omt);
    h.MT32[c] = (const float*)(base + omt32);
    h.M32[c] = (const float*)(base + om32);
    h.Mhi[c] = (const __nv_bfloat16*)(base + ohi);
    h.Mlo[c] = (const __nv_bfloat16*)(base + olo);
    h.aux64[c] = (const double*)(base + oa64);
    h.aux32[c] = (const float*)(base + oa32);
    h.gid[c] = (const int32_t*)(base + ogid);
    h.oh32[c] = (const float*)(base + ooh);
    h.ol32[c] = (const float*)(base + ool);
  }
  size_t otm = take(kMaps * sizeof(CUtensorMap));
  for (int c = 0; c < nc; ++c) {
    const CUtensorMap* m = (const CUtensorMap*)(base + otm);
    h.tmap32[c] = m + c;
    h.tmaphi[c] = m + SV_MAXC + c;
    h.tmaplo[c] = m + 2 * SV_MAXC + c;
    h.tmap32h[c] = m + 3 * SV_MAXC + c;
    h.tmaphih[c] = m + 4 * SV_MAXC + c;
    h.tmaploh[c] = m + 5 * SV_MAXC + c;
  }
  size_t od = take(sizeof(ProblemDev));
  if (overflow) return SEVO_ERR_STATE;  // layout and size out of step: nothing is published
  // the descriptors encode device addresses, so they are built after the
  // operand pointers are known and copied into the block with the rest
  int32_t st = sv_build_tmaps(p);
  if (st != SEVO_OK) return st;
  for (int c = 0; c < nc; ++c) {
    std::memcpy(&blob[otm + c * sizeof(CUtensorMap)], &p->tmap_f32[c], sizeof(CUtensorMap));
    std::memcpy(&blob[otm + (SV_MAXC + c) * sizeof(CUtensorMap)], &p->tmap_hi[c], sizeof(CUtensorMap));
    std::memcpy(&blob[otm + (2 * SV_MAXC + c) * sizeof(CUtensorMap)], &p->tmap_lo[c],
                sizeof(CUtensorMap));
    std::memcpy(&blob[otm + (3 * SV_MAXC + c) * sizeof(CUtensorMap)], &p->tmap_f32h[c],
                sizeof(CUtensorMap));
    std::memcpy(&blob[otm + (4 * SV_MAXC + c) * sizeof(CUtensorMap)], &p->tmap_hih[c],
                sizeof(CUtensorMap));
    std::memcpy(&blob[otm + (5 * SV_MAXC + c) * sizeof(CUtensorMap)], &p->tmap_loh[c],
                sizeof(CUtensorMap));
  }
  std::memcpy(&blob[od], &h, sizeof(ProblemDev));
  SV_CUDA(cudaMemcpy(p->dev_block, blob.data(), p->dev_bytes, cudaMemcpyHostToDevice));
  // published only once the block holds the descriptor
  p->desc_d = (ProblemDev*)(base + od);
  return SEVO_OK;
}

static sevo_problem* alloc_problem(int family, int D, int ncomp) {
  sevo_problem* p = (sevo_problem*)std::calloc(1, sizeof(sevo_problem));
  if (!p) return nullptr;
  p->family = family;
  p->D = D;
  p->ncomp = ncomp;
  p->ngroups = 1;
  p->fstar = 100.0;
  p->o_h = (double*)std::calloc((size_t)ncomp * D, sizeof(double));
  p->M_h = (double*)std::calloc((size_t)ncomp * D * D, sizeof(double));
  if (!p->o_h || !p->M_h) {
    std::free(p->o_h);
    std::free(p->M_h);
    std::free(p);
    return nullptr;
  }
  return p;
}

static void free_problem(sevo_problem* p) {
  if (!p) return;
  if (p->dev_block) cudaFree(p->dev_block);
  std::free(p->o_h);
  std::free(p->M_h);
  std::free(p->perm_h);
  std::free(p);
}

// Instance data is generated on the host at creation; the device copy is
// made on first device use, on the device current at that time.
static std::mutex g_upload_mu;

int32_t sv_problem_ready(const sevo_problem* cp) {
  sevo_problem* p = const_cast<sevo_problem*>(cp);
  std::lock_guard<std::mutex> lk(g_upload_mu);
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) return SEVO_ERR_CUDA;
  if (p->desc_d) return (dev == p->device) ? SEVO_OK : SEVO_ERR_STATE;
  p->device = dev;
  int32_t st = upload(p);
  if (st != SEVO_OK && p->dev_block) {
    cudaFree(p->dev_block);
    p->dev_block = nullptr;
    p->desc_d = nullptr;
  }
  return st;
}

int32_t sv_problem_has_device_copy(const sevo_problem* p, int dev) {
  std::lock_guard<std::mutex> lk(g_upload_mu);
  return (p->desc_d && p->device == dev) ? SEVO_OK : SEVO_ERR_STATE;
}

static int32_t finish(sevo_problem* p, sevo_problem** out) {
  p->device = -1;
  *out = p;
  return SEVO_OK;
}

static int32_t make_hybrid(uint64_t seed, int D, int K, const double* frac, const int32_t* bodies,
                           sevo_problem** out) {
  sevo_problem* p = alloc_problem(SEVO_HYBRID, D, 1);
  if (!p) return SEVO_ERR_OOM;
  p->ngroups = K;
  p->perm_h = (int32_t*)std::calloc((size_t)D, sizeof(int32_t));
  if (!p->perm_h) {
    free_problem(p);
    return SEVO_ERR_OOM;
  }
  int used = 0;
  for (int k = 0; k < K; ++k) {
    p->gbody[k] = bodies[k];
    if (k < K - 1) {
      p->gsize[k] = (int32_t)std::floor(frac[k] * (double)D);
      used += p->gsize[k];
    } else {
      p->gsize[k] = D - used;
    }
    if (p->gsize[k] < 0) {
      free_problem(p);
      return SEVO_ERR_ARG;
    }
  }
  gen_shift(seed, D, 0, p->o_h);
  std::vector<double> M((size_t)D * D);
  gen_rotation(seed, D, 0, M.data());
  gen_perm(seed, D, p->perm_h);
  for (int t = 0; t < D; ++t)
    std::memcpy(p->M_h + (size_t)t * D, M.data() + (size_t)p->perm_h[t] * D, sizeof(double) * D);
  return finish(p, out);
}

extern "C" int32_t sevo_hybrid_create(uint64_t seed, int32_t D, int32_t K, const double* frac,
                                      const int32_t* bodies, sevo_problem** out) {
  if (!out || !frac || !bodies || D < 2 || D > SEVO_MAX_D || K < 1 || K > SV_MAXG)
    return SEVO_ERR_ARG;
  for (int k = 0; k < K; ++k)
    if (bodies[k] < 0 || bodies[k] > SEVO_GRIEWANK || !(frac[k] >= 0.0) || frac[k] > 1.0)
      return SEVO_ERR_ARG;
  return make_hybrid(seed, D, K, frac, bodies, out);
}

// hybrid groups drawn with salt (as for the hybrid family, whose salt is 0):
// K in 3..5, fractions 0.1 + (1 - 0.1 K) E_k / sum E (E ~ Exp(1)), bodies
// among the six, sizes floor(frac D) with the last group the remainder
static int hybrid_groups(uint64_t seed, int D, uint32_t salt, int32_t* gsize, int32_t* gbody) {
  uint4 w = sv_draw(seed, 0u, 0u, (uint32_t)D, SV_P_HYB, salt);
  const int K = 3 + (int)sv_below(w.x, 3u);
  double E[8], sumE = 0.0;
  for (int k = 0; k < K; ++k) {
    uint4 v = sv_draw(seed, (uint32_t)(1 + k), 0u, (uint32_t)D, SV_P_HYB, salt);
    E[k] = -std::log(1.0 - sv_u53(v.x, v.y));
    gbody[k] = (int32_t)sv_below(v.z, 6u);
    sumE += E[k];
  }
  int used = 0;
  for (int k = 0; k < K; ++k) {
    const double frac = 0.1 + (1.0 - 0.1 * (double)K) * E[k] / sumE;
    if (k < K - 1) {
      gsize[k] = (int32_t)std::floor(frac * (double)D);
      used += gsize[k];
    } else {
      gsize[k] = D - used;
    }
  }
  return K;
}

extern "C" int32_t sevo_problem_create(uint64_t seed, int32_t family, int32_t D,
                                       sevo_problem** out) {
  if (!out || D < 2 || D > SEVO_MAX_D || family < 0 || family > SEVO_COMP_HYBRID)
    return SEVO_ERR_ARG;
  *out = nullptr;
  if (family == SEVO_COMP_HYBRID) {
    uint4 w = sv_draw(seed, 0u, 0u, (uint32_t)D, SV_P_COMP);
    const int Nc = 3 + (int)sv_below(w.x, 3u);
    sevo_problem* p = alloc_problem(SEVO_COMP_HYBRID, D, Nc);
    if (!p) return SEVO_ERR_OOM;
    p->perm_h = (int32_t*)std::calloc((size_t)Nc * D, sizeof(int32_t));
    if (!p->perm_h) {
      free_problem(p);
      return SEVO_ERR_OOM;
    }
    std::vector<double> M((size_t)D * D);
    for (int c = 0; c < Nc; ++c) {
      uint4 v = sv_draw(seed, (uint32_t)(1 + c), 0u, (uint32_t)D, SV_P_COMP);
      p->sigma[c] = 10.0 * (double)(1 + sv_below(v.x, 6u));
      p->lambda[c] = std::pow(10.0, -6.0 + 6.0 * sv_u53(v.y, v.z));
      p->bias[c] = 100.0 * (double)c;
      gen_shift(seed, D, c, p->o_h + (size_t)c * D);
      gen_rotation(seed, D, c, M.data());
      p->cK[c] = hybrid_groups(seed, D, (uint32_t)(1 + c), p->cgsize[c], p->cgbody[c]);
      int32_t* perm = p->perm_h + (size_t)c * D;
      gen_perm(seed, D, perm, (uint32_t)(1 + c));
      for (int t = 0; t < D; ++t)
        std::memcpy(p->M_h + (size_t)c * D * D + (size_t)t * D, M.data() + (size_t)perm[t] * D,
                    sizeof(double) * D);
    }
    return finish(p, out);
  }
  if (family <= SEVO_GRIEWANK) {
    sevo_problem* p = alloc_problem(family, D, 1);
    if (!p) return SEVO_ERR_OOM;
    gen_shift(seed, D, 0, p->o_h);
    gen_rotation(seed, D, 0, p->M_h);
    return finish(p, out);
  }
  if (family == SEVO_HYBRID) {
    uint4 w = sv_draw(seed, 0u, 0u, (uint32_t)D, SV_P_HYB);
    int K = 3 + (int)sv_below(w.x, 3u);
    double E[8], frac[8], sumE = 0.0;
    int32_t bodies[8];
    for (int k = 0; k < K; ++k) {
      uint4 v = sv_draw(seed, (uint32_t)(1 + k), 0u, (uint32_t)D, SV_P_HYB);
      E[k] = -std::log(1.0 - sv_u53(v.x, v.y));
      bodies[k] = (int32_t)sv_below(v.z, 6u);
      sumE += E[k];
    }
    for (int k = 0; k < K; ++k) frac[k] = 0.1 + (1.0 - 0.1 * (double)K) * E[k] / sumE;
    return make_hybrid(seed, D, K, frac, bodies, out);
  }
  uint4 w = sv_draw(seed, 0u, 0u, (uint32_t)D, SV_P_COMP);
  int Nc = 3 + (int)sv_below(w.x, 8u);
  sevo_problem* p = alloc_problem(SEVO_COMPOSITION, D, Nc);
  if (!p) return SEVO_ERR_OOM;
  for (int c = 0; c < Nc; ++c) {
    uint4 v = sv_draw(seed, (uint32_t)(1 + c), 0u, (uint32_t)D, SV_P_COMP);
    p->sigma[c] = 10.0 * (double)(1 + sv_below(v.x, 6u));
    p->lambda[c] = std::pow(10.0, -6.0 + 6.0 * sv_u53(v.y, v.z));
    p->cbody[c] = (int32_t)sv_below(v.w, 6u);
    p->bias[c] = 100.0 * (double)c;
    gen_shift(seed, D, c, p->o_h + (size_t)c * D);
    gen_rotation(seed, D, c, p->M_h + (size_t)c * D * D);
  }
  return finish(p, out);
}

extern "C" int32_t sevo_problem_destroy(sevo_problem* p) {
  if (!p) return SEVO_ERR_ARG;
  free_problem(p);
  return SEVO_OK;
}

extern "C" int32_t sevo_problem_info(const sevo_problem* p, int32_t* family, int32_t* D,
                                     int32_t* ncomp, double* fstar) {
  if (!p) return SEVO_ERR_ARG;
  if (family) *family = p->family;
  if (D) *D = p->D;
  if (ncomp) *ncomp = (p->family == SEVO_HYBRID) ? p->ngroups : p->ncomp;  // groups or components
  if (fstar) *fstar = p->fstar;
  return SEVO_OK;
}

extern "C" int32_t sevo_problem_export(const sevo_problem* p, int32_t comp, double* o, double* M,
                                       int32_t* perm, int32_t* gsize, int32_t* gbody,
                                       double* sigma, double* lambda, double* bias) {
  if (!p || comp < 0 || comp >= p->ncomp) return SEVO_ERR_ARG;
  const size_t D = (size_t)p->D;
  if (o) std::memcpy(o, p->o_h + comp * D, D * 8);
  if (M) std::memcpy(M, p->M_h + comp * D * D, D * D * 8);
  if (p->family == SEVO_HYBRID) {
    if (perm) std::memcpy(perm, p->perm_h, D * 4);
    if (gsize) std::memcpy(gsize, p->gsize, p->ngroups * 4);
    if (gbody) std::memcpy(gbody, p->gbody, p->ngroups * 4);
  }
  if (p->family == SEVO_COMP_HYBRID) {  // component comp's hybrid structure
    if (perm) std::memcpy(perm, p->perm_h + comp * D, D * 4);
    if (gsize) std::memcpy(gsize, p->cgsize[comp], p->cK[comp] * 4);
    if (gbody) std::memcpy(gbody, p->cgbody[comp], p->cK[comp] * 4);
  }
  if (p->family == SEVO_COMPOSITION || p->family == SEVO_COMP_HYBRID) {
    if (gbody && p->family == SEVO_COMPOSITION) std::memcpy(gbody, p->cbody, p->ncomp * 4);
    if (sigma) std::memcpy(sigma, p->sigma, p->ncomp * 8);
    if (lambda) std::memcpy(lambda, p->lambda, p->ncomp * 8);
    if (bias) std::memcpy(bias, p->bias, p->ncomp * 8);
  }
  return SEVO_OK;
}
