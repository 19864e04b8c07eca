// evo.cu -- DE and PSO generation kernels and the single-run state API.
//
// Operators (Listing 1 names the modules; the formulas are the library's
// readings, identical in every bit to the oracle's so that lock-step
// comparisons are exact):
//   DE/rand/1:           v = fma(F, x_r2 - x_r3, x_r1)
//   DE/current-to-pbest: v = fma(F, x_r1 - x~_r2, fma(F, x_pb - x_i, x_i))
//   binomial crossover:  u_j = v_j if word_j * 2^-32 < CR or j = j_rand
//   midpoint repair:     u_j < lb -> (lb + x_ij) / 2;  u_j > ub -> (ub + x_ij) / 2
//   selection:           x_i <- u_i iff f(u_i) <= f(x_i); current-to-pbest
//                        pushes the replaced parent into the archive (row
//                        order; random slot once full, later rows win)
//   PSO:                 v = fma(w, v, fma(c1 r1, p - x, (c2 r2)(g - x)));
//                        x += v; clamp to [lb,ub] with v = 0 there;
//                        p_i <- x_i iff f(x_i) < f(p_i); guide = gbest or
//                        ring {i-1,i,i+1} argmin (lowest index on ties)
// FP64 arithmetic uses explicit round-to-nearest intrinsics (no contraction
// beyond the stated fma), so trial vectors equal the oracle's bit for bit.
// Streaming kernels move 4 consecutive coordinates per thread (one Philox
// call covers the four crossover words).
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstring>
#include <vector>

#include "bodies.cuh"
#include "bounds.cuh"
#include "evo.cuh"
#include "ops.cuh"
#include "tc_ptx.cuh"

namespace {

// order-preserving integer key of a double (NaN sorts last)
__device__ __forceinline__ long long fkey(double f) {
  long long b = __double_as_longlong(f);
  if (f != f) return 0x7FFFFFFFFFFFFFFFll;
  return b >= 0 ? b : (b ^ 0x7FFFFFFFFFFFFFFFll);
}

__device__ __forceinline__ double dmin_pos(double a, double b) { return (b < a) ? b : a; }

// ---------------------------------------------------------------- control
__global__ void ctl_set_kernel(GenCtl* ctl, unsigned long long gen, int count) {
  ctl->gen = gen;
  ctl->count = count;
}

__global__ void ctl_advance_kernel(GenCtl* ctl, int NP, long long budget, int per_gen) {
  unsigned long long g = ctl->gen + 1;
  ctl->gen = g;
  long long before = (long long)NP + (long long)(g - 1) * per_gen;
  long long c = budget - before;
  ctl->count = (int)(c < 0 ? 0 : (c > per_gen ? per_gen : c));
}

// The generation's counter for its first kernel: from the launch when the
// caller set it (block 0 then publishes it to the control block for the
// generation's later kernels, which run after this one in stream order),
// else from the control block (generations replayed from a graph).
__device__ __forceinline__ unsigned long long gen_of(GenCtl* ctl, const CtlSet& cs) {
  if (!cs.on) return ctl->gen;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    ctl->gen = cs.gen;
    ctl->count = cs.count;
  }
  return cs.gen;
}

// ---------------------------------------------------------------- indexing
// n / d for 0 <= n < 2^31 by multiply-high (Granlund and Montgomery's
// round-up method): q = (umulhi(n, m) + n) >> l with l = ceil(log2 d) and
// m = floor(2^32 (2^l - d) / d) + 1, instead of a 64-bit division per thread.
struct FastDiv {
  uint32_t d, m, l;
};
FastDiv make_fastdiv(uint32_t d) {
  uint32_t l = 0;
  while ((1ull << l) < d) ++l;
  const uint64_t m = ((1ull << 32) * ((1ull << l) - d)) / d + 1;
  return FastDiv{d, (uint32_t)m, l};
}
__device__ __forceinline__ uint32_t fdiv(uint32_t n, const FastDiv& f) {
  return (__umulhi(n, f.m) + n) >> f.l;
}
// t = (hi * nmid + mid) * nlo + lo; row = hi * nmid + mid
struct Split3 {
  int lo, mid, hi;
  int64_t row;
};
__device__ __forceinline__ Split3 split3(int64_t t, bool fast, const FastDiv& flo,
                                         const FastDiv& fmid) {
  Split3 s;
  if (fast) {
    const uint32_t u = (uint32_t)t, q = fdiv(u, flo), q2 = fdiv(q, fmid);
    s.lo = (int)(u - q * flo.d);
    s.mid = (int)(q - q2 * fmid.d);
    s.hi = (int)q2;
    s.row = (int64_t)q;
  } else {
    const int64_t q = t / flo.d, q2 = q / fmid.d;
    s.lo = (int)(t - q * flo.d);
    s.mid = (int)(q - q2 * fmid.d);
    s.hi = (int)q2;
    s.row = q;
  }
  return s;
}

// ---------------------------------------------------------------- init
__global__ void init_pop_kernel(double* __restrict__ X, const uint64_t* __restrict__ seeds, int R,
                                int NP, int D, int ld, double lb, double ub, FastDiv fpair,
                                FastDiv fnp) {
  const int64_t total = (int64_t)R * NP * ((D + 1) / 2);
  const bool fast = total < (1ll << 31);
  const double span = __dsub_rn(ub, lb);
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    const Split3 sp = split3(t, fast, fpair, fnp);
    const int jp = sp.lo, i = sp.mid, r = sp.hi;
    const uint4 w = sv_draw(seeds[r], (uint32_t)jp, (uint32_t)i, 0u, SV_P_INIT);
    double* xr = X + ((int64_t)r * NP + i) * ld;
    const int j = 2 * jp;
    xr[j] = __dadd_rn(lb, __dmul_rn(span, u53_int(w.x, w.y)));
    if (j + 1 < D) xr[j + 1] = __dadd_rn(lb, __dmul_rn(span, u53_int(w.z, w.w)));
  }
}

// every run's o as its float hi/lo split (Osp: R rows of hi, then R rows of
// lo, apitch floats each, zero past D), gathered once so that the operators
// read it with one load per value
__global__ void gather_osplit_kernel(const ProblemDev* const* __restrict__ rp, int R, int D,
                                     int apitch, float* __restrict__ Osp) {
  const int64_t total = (int64_t)2 * R * apitch;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t rr = t / apitch;
    const int j = (int)(t - rr * apitch);
    const int r = (int)(rr < R ? rr : rr - R);
    const float* src = rr < R ? rp[r]->oh32[0] : rp[r]->ol32[0];
    Osp[t] = j < D ? src[j] : 0.f;
  }
}

// the TF32 operand of trial quad j0..j0+3 of run r's batch row `row` (one
// component) for the fused evaluation, which then loads it instead of
// converting the row (the same function, hence the same bits, either way);
// columns past D hold 0 and are never read
__device__ __forceinline__ void write_operand4(float* __restrict__ Ad, int apitch,
                                               const float* __restrict__ Osp, int R, int r,
                                               int64_t row, int j0, int D, const double (&u)[4]) {
  const float4 oh = __ldg(reinterpret_cast<const float4*>(Osp + (int64_t)r * apitch + j0));
  const float4 ol = __ldg(reinterpret_cast<const float4*>(Osp + (int64_t)(R + r) * apitch + j0));
  const float ohv[4] = {oh.x, oh.y, oh.z, oh.w}, olv[4] = {ol.x, ol.y, ol.z, ol.w};
  float d[4];
#pragma unroll
  for (int q = 0; q < 4; ++q)
    d[q] = (j0 + q < D) ? tc::to_tf32(sv_operand_d(u[q], ohv[q], olv[q])) : 0.f;
  *reinterpret_cast<float4*>(Ad + row * apitch + j0) = make_float4(d[0], d[1], d[2], d[3]);
}

constexpr int TRIAL_THREADS = 128;

// (at most 80 registers, so that 6 of these CTAs share an SM: measured 1 %
// faster in the step than 96 registers and 5 CTAs; 64 registers spilled)
template <int ALG>
__global__ void __launch_bounds__(TRIAL_THREADS, 6) de_trial_kernel(const double* __restrict__ X, double* __restrict__ U,
                                const double* __restrict__ A, const int32_t* __restrict__ asize,
                                const int32_t* __restrict__ order, int32_t* __restrict__ part,
                                const uint64_t* __restrict__ seeds, GenCtl* ctl, CtlSet cs,
                                int R, int NP, int D, int ld, double F, unsigned long long cr_thr,
                                double lb, double ub, int pk, FastDiv fq, FastDiv fnp,
                                const double* __restrict__ Fi, const double* __restrict__ CRi,
                                const int32_t* __restrict__ kpb, float* __restrict__ Ad,
                                int apitch, const float* __restrict__ Osp) {
  const int nq = (D + 3) >> 2;
  const int64_t total = (int64_t)R * NP * nq;
  const bool fast = total < (1ll << 31);
  const unsigned long long gen = gen_of(ctl, cs);
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    const Split3 sp = split3(t, fast, fq, fnp);
    double uq[4];
    de_trial_elem<ALG>(X, U, A, asize, order, part, seeds, NP, D, ld, F, cr_thr, lb, ub, pk, gen,
                       sp.hi, sp.mid, sp.lo, Fi, CRi, kpb, Ad ? uq : nullptr);
    if (Ad) write_operand4(Ad, apitch, Osp, R, sp.hi, sp.row, sp.lo * 4, D, uq);
  }
}

// ---------------------------------------------------------------- SHADE
// per row: memory slot, pbest pool, CR (normal, clipped), F (Cauchy, redrawn
// while <= 0, capped at 1) from the run's memory; the arithmetic is written
// with explicit roundings (no contraction) in the order of the definition
constexpr double SV_PI = 3.14159265358979323846;

__global__ void shade_param_kernel(const double* __restrict__ MF, const double* __restrict__ MCR,
                                   const uint64_t* __restrict__ seeds,
                                   GenCtl* ctl, CtlSet cs, int R, int NP, int H,
                                   double* __restrict__ Fi, double* __restrict__ CRi,
                                   int32_t* __restrict__ kpb) {
  const int64_t rows = (int64_t)R * NP;
  const unsigned long long gen = gen_of(ctl, cs);
  const double pmin = 2.0 / (double)NP;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < rows;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int r = (int)(t / NP), i = (int)(t - (int64_t)r * NP);
    const uint64_t seed = seeds[r];
    uint4 w = sv_draw(seed, 0u, (uint32_t)i, (uint32_t)gen, SV_P_SHADE);
    const int h = (int)sv_below(w.x, (uint32_t)H);
    const double p = __dadd_rn(pmin, __dmul_rn(__dsub_rn(0.2, pmin), u53_int(w.y, w.z)));
    int k = (int)floor(__dadd_rn(__dmul_rn(p, (double)NP), 0.5));
    k = k < 1 ? 1 : (k > NP ? NP : k);
    kpb[t] = k;
    const double mcr = MCR[(int64_t)r * H + h], mf = MF[(int64_t)r * H + h];
    w = sv_draw(seed, 1u, (uint32_t)i, (uint32_t)gen, SV_P_SHADE);
    const double u1 = u53_int(w.x, w.y), u2 = u53_int(w.z, w.w);
    const double z = __dmul_rn(sqrt(__dmul_rn(-2.0, log(__dsub_rn(1.0, u1)))),
                               cos(__dmul_rn(2.0 * SV_PI, u2)));
    double cr = __dadd_rn(mcr, __dmul_rn(0.1, z));
    cr = cr < 0.0 ? 0.0 : (cr > 1.0 ? 1.0 : cr);
    CRi[t] = cr;
    double f = mf;
    for (int a = 0; a < 64; ++a) {
      w = sv_draw(seed, 2u + (uint32_t)a, (uint32_t)i, (uint32_t)gen, SV_P_SHADE);
      const double c =
          __dadd_rn(mf, __dmul_rn(0.1, tan(__dmul_rn(SV_PI, __dsub_rn(u53_int(w.x, w.y), 0.5)))));
      if (c > 0.0) {
        f = c;
        break;
      }
    }
    Fi[t] = f > 1.0 ? 1.0 : f;
  }
}

// ---------------------------------------------------------------- DE rank
// top-k of each run by (fitness, index): order[rank] = row for rank < k.
// Grid (runs, row blocks): each CTA loads the run's integer sort keys into
// shared memory and ranks its 256 rows by counting (exact, deterministic).
constexpr int RANK_ROWS = 256;
__global__ void __launch_bounds__(RANK_ROWS)
    de_rank_kernel(const double* __restrict__ fx, int32_t* __restrict__ order, int NP, int k) {
  extern __shared__ long long keys[];
  const int r = blockIdx.x;
  const double* f = fx + (int64_t)r * NP;
  for (int i = threadIdx.x; i < NP; i += blockDim.x) keys[i] = fkey(f[i]);
  __syncthreads();
  const int i = blockIdx.y * RANK_ROWS + threadIdx.x;
  if (i >= NP) return;
  const long long ki = keys[i];
  int rank = 0;
  int j = 0;
  for (; j + 4 <= NP; j += 4) {
    const long long k0 = keys[j], k1 = keys[j + 1], k2 = keys[j + 2], k3 = keys[j + 3];
    rank += (k0 < ki) || (k0 == ki && j < i);
    rank += (k1 < ki) || (k1 == ki && j + 1 < i);
    rank += (k2 < ki) || (k2 == ki && j + 2 < i);
    rank += (k3 < ki) || (k3 == ki && j + 3 < i);
  }
  for (; j < NP; ++j) rank += (keys[j] < ki) || (keys[j] == ki && j < i);
  if (rank < k) order[(int64_t)r * NP + rank] = i;
}

// the same ranking for run r by one block (keys: NP entries of shared memory)
__device__ __forceinline__ void rank_run_block(const double* __restrict__ f,
                                               int32_t* __restrict__ order_r, int NP, int k,
                                               long long* keys) {
  for (int i = threadIdx.x; i < NP; i += blockDim.x) keys[i] = fkey(f[i]);
  __syncthreads();
  for (int i = threadIdx.x; i < NP; i += blockDim.x) {
    const long long ki = keys[i];
    int rank = 0;
    for (int j = 0; j < NP; ++j) rank += (keys[j] < ki) || (keys[j] == ki && j < i);
    if (rank < k) order_r[rank] = i;
  }
  __syncthreads();
}

// Larger populations: one CTA per run narrows down the k-th smallest key by
// an MSB-first radix select (8-bit digits, shared-memory histograms), gathers
// the rows whose key is at most the threshold it reaches (the k best plus the
// rest of the last selected bin) and sorts only those by (key, index) with a
// bitonic network; the first k indices are the p-best pool, identical to the
// counting rank.
constexpr int RSEL_THREADS = 512;

__host__ __device__ inline int pow2_at_least(int n) {
  int m = 1;
  while (m < n) m <<= 1;
  return m;
}
__host__ __device__ inline size_t rsel_smem_bytes(int NP) {
  return (size_t)NP * 8 + (size_t)pow2_at_least(NP) * 12 + 16;
}

__global__ void __launch_bounds__(RSEL_THREADS)
    de_rank_select_kernel(const double* __restrict__ fx, int32_t* __restrict__ order, int NP,
                          int npow2, int k) {
  extern __shared__ __align__(16) unsigned char rs_sm[];
  unsigned long long* uk = reinterpret_cast<unsigned long long*>(rs_sm);  // NP keys
  unsigned long long* ck = uk + NP;                                       // candidates
  int* ci = reinterpret_cast<int*>(ck + npow2);
  __shared__ unsigned int hist[256];
  __shared__ unsigned long long s_prefix, s_lo[RSEL_THREADS / 32], s_hi[RSEL_THREADS / 32];
  __shared__ int s_rem, s_below, s_cnt, s_ncand;
  const int r = blockIdx.x, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const double* f = fx + (int64_t)r * NP;
  unsigned long long lo = ~0ull, hi = 0ull;
  for (int i = tid; i < NP; i += blockDim.x) {
    const unsigned long long v = (unsigned long long)fkey(f[i]) ^ 0x8000000000000000ull;  // unsigned order
    uk[i] = v;
    lo = v < lo ? v : lo;
    hi = v > hi ? v : hi;
  }
  for (int o = 16; o >= 1; o >>= 1) {
    const unsigned long long a = __shfl_xor_sync(0xffffffffu, lo, o);
    const unsigned long long b = __shfl_xor_sync(0xffffffffu, hi, o);
    lo = a < lo ? a : lo;
    hi = b > hi ? b : hi;
  }
  if (lane == 0) {
    s_lo[warp] = lo;
    s_hi[warp] = hi;
  }
  if (tid == 0) s_ncand = 0;
  __syncthreads();
  lo = ~0ull;
  hi = 0ull;
  for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
    lo = s_lo[w] < lo ? s_lo[w] : lo;
    hi = s_hi[w] > hi ? s_hi[w] : hi;
  }
  // The digits above the highest bit where the smallest and largest keys
  // differ are common to every key: the select starts at the digit holding
  // that bit.  It stops as soon as the keys up to the selected digit's bin
  // are few enough to be sorted directly (at most cap: the sort size that k
  // keys need anyway); the gather below then takes every key whose digits so
  // far are at most the selected ones.
  const int cap = pow2_at_least(k);
  unsigned long long thresh = lo;  // all keys equal: every key is a candidate
  if (lo != hi) {
    int shift = ((63 - __clzll((long long)(lo ^ hi))) >> 3) << 3;
    unsigned long long pmask = shift == 56 ? 0ull : ~((1ull << (shift + 8)) - 1ull);
    unsigned long long prefix = lo & pmask;
    int rem = k;    // rank (1-based) of the k-th key among the keys matching prefix
    int below = 0;  // keys below the prefix's range (all among the k best)
    for (;;) {
      for (int b = tid; b < 256; b += blockDim.x) hist[b] = 0u;
      __syncthreads();
      for (int i = tid; i < NP; i += blockDim.x) {
        const unsigned long long v = uk[i];
        if ((v & pmask) == prefix) atomicAdd(&hist[(unsigned)((v >> shift) & 255u)], 1u);
      }
      __syncthreads();
      if (tid < 32) {  // lane owns bins 8*lane .. 8*lane+7
        unsigned c[8], sum = 0u;
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          c[q] = hist[lane * 8 + q];
          sum += c[q];
        }
        unsigned incl = sum;
        for (int o = 1; o < 32; o <<= 1) {
          const unsigned v = __shfl_up_sync(0xffffffffu, incl, o);
          if (lane >= o) incl += v;
        }
        const unsigned excl = incl - sum;
        if (excl < (unsigned)rem && (unsigned)rem <= incl) {
          unsigned acc = excl;
          int b = lane * 8 + 7;
#pragma unroll
          for (int q = 0; q < 8; ++q) {
            if (acc + c[q] >= (unsigned)rem) {
              b = lane * 8 + q;
              break;
            }
            acc += c[q];
          }
          s_prefix = prefix | ((unsigned long long)b << shift);
          s_rem = rem - (int)acc;
          s_below = below + (int)acc;
          s_cnt = (int)hist[b];
        }
      }
      __syncthreads();
      prefix = s_prefix;
      rem = s_rem;
      below = s_below;
      const int cnt = s_cnt;
      if (shift == 0 || below + cnt <= cap) {
        thresh = prefix | (shift == 0 ? 0ull : (1ull << shift) - 1ull);
        break;
      }
      pmask |= 255ull << shift;
      shift -= 8;
    }
  }
  // gather every key <= thresh: the k best and the rest of the last selected
  // bin (one atomic per warp; the candidates' order does not matter, they are
  // sorted by (key, index) below)
  const int NPw = (NP + (int)blockDim.x - 1) / (int)blockDim.x * (int)blockDim.x;
  for (int i = tid; i < NPw; i += blockDim.x) {
    const unsigned long long v = (i < NP) ? uk[i] : ~0ull;
    const bool c = (i < NP) && v <= thresh;
    const unsigned bal = __ballot_sync(0xffffffffu, c);
    int base = 0;
    if (lane == 0 && bal) base = atomicAdd(&s_ncand, __popc(bal));
    base = __shfl_sync(0xffffffffu, base, 0);
    if (c) {
      const int slot = base + __popc(bal & ((1u << lane) - 1u));
      ck[slot] = v;
      ci[slot] = i;
    }
  }
  __syncthreads();
  const int n = s_ncand;  // >= k
  const int m = pow2_at_least(n);
  for (int i = n + tid; i < m; i += blockDim.x) {
    ck[i] = ~0ull;
    ci[i] = 0x7FFFFFFF;
  }
  __syncthreads();
  for (int size = 2; size <= m; size <<= 1) {
    for (int stride = size >> 1; stride > 0; stride >>= 1) {
      for (int t = tid; t < m / 2; t += blockDim.x) {
        const int lo = 2 * t - (t & (stride - 1));
        const int hi = lo + stride;
        const bool up = ((lo & size) == 0);
        const unsigned long long ka = ck[lo], kb = ck[hi];
        const int ia = ci[lo], ib = ci[hi];
        const bool a_gt_b = (ka > kb) || (ka == kb && ia > ib);
        if (a_gt_b == up) {
          ck[lo] = kb;
          ck[hi] = ka;
          ci[lo] = ib;
          ci[hi] = ia;
        }
      }
      __syncthreads();
    }
  }
  for (int q = tid; q < k; q += blockDim.x) order[(int64_t)r * NP + q] = ci[q];
}

// ---------------------------------------------------------------- DE select
// per run: acceptance, best-so-far, archive slots (row order, random slot
// once full, the last row targeting a slot wins), fitness update.
// action[i]: -2 rejected, -1 accepted without archive write, >= 0 slot.
constexpr int SEL_THREADS = 512;

__device__ __forceinline__ void block_min_update(double v, double* best_r) {
  __shared__ double red[SEL_THREADS / 32];
  for (int m = 16; m >= 1; m >>= 1) v = dmin_pos(v, __shfl_xor_sync(0xffffffffu, v, m));
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) red[warp] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double b = red[0];
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) b = dmin_pos(b, red[w]);
    *best_r = dmin_pos(*best_r, b);
  }
  __syncthreads();
}

// One CTA per run stages the run's current and trial fitness in shared
// memory with coalesced loads; acceptance flags, the row-order scan and the
// slot resolution then run on shared memory.
__host__ __device__ constexpr size_t sel_smem_bytes(int NP) {
  return (size_t)NP * (8 + 8 + 4 + 4 + 1) + 16;
}

// run r by the whole block; sel_sm: sel_smem_bytes(NP) of shared memory
__device__ __forceinline__ void de_select_run(double* __restrict__ fx, const double* __restrict__ fu,
                                              int32_t* __restrict__ asize,
                                              int32_t* __restrict__ action,
                                              double* __restrict__ best,
                                              const uint64_t* __restrict__ seeds, int count,
                                              unsigned long long gen, int NP, int use_archive,
                                              int r, unsigned char* sel_sm,
                                              const double* __restrict__ Fi = nullptr,
                                              const double* __restrict__ CRi = nullptr,
                                              double* __restrict__ MF = nullptr,
                                              double* __restrict__ MCR = nullptr,
                                              int32_t* __restrict__ mk = nullptr, int H = 0) {
  double* sf = reinterpret_cast<double*>(sel_sm);  // current fitness
  double* sg = sf + NP;                             // trial fitness
  int* owner = reinterpret_cast<int*>(sg + NP);     // archive slot -> last row
  int* sact = owner + NP;                           // action per row
  unsigned char* sacc = reinterpret_cast<unsigned char*>(sact + NP);  // accepted
  __shared__ int wsum[SEL_THREADS / 32];
  const int tid = threadIdx.x;
  double* f = fx + (int64_t)r * NP;
  const double* g = fu + (int64_t)r * NP;
  int32_t* act = action + (int64_t)r * NP;
  for (int i = tid; i < NP; i += blockDim.x) {
    sf[i] = f[i];
    sg[i] = g[i];
    owner[i] = -1;
  }
  __syncthreads();
  // best-so-far over the rows that count toward the budget
  double m = INFINITY;
  for (int i = tid; i < count; i += blockDim.x) m = dmin_pos(m, sg[i]);
  block_min_update(m, best + r);
  for (int i = tid; i < NP; i += blockDim.x) sacc[i] = (sg[i] <= sf[i]) ? 1 : 0;
  __syncthreads();
  // contiguous chunk of rows per thread, so the scan follows row order
  const int per = (NP + blockDim.x - 1) / blockDim.x;
  const int i0 = min(NP, tid * per), i1 = min(NP, i0 + per);
  int cnt = 0;
  for (int i = i0; i < i1; ++i) cnt += sacc[i];
  const int warp = tid >> 5, lane = tid & 31;
  int incl = cnt;
  for (int o = 1; o < 32; o <<= 1) {
    int v = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += v;
  }
  if (lane == 31) wsum[warp] = incl;
  __syncthreads();
  int woff = 0;
  for (int w = 0; w < warp; ++w) woff += wsum[w];
  int nacc_total = 0;
  for (int w = 0; w < (int)(blockDim.x >> 5); ++w) nacc_total += wsum[w];
  int k = woff + incl - cnt;
  if (MF) {  // SHADE: the strict improvements update memory slot mk[r]
    __shared__ double ssum[SEL_THREADS / 32][4];
    double sw = 0.0, swf = 0.0, swf2 = 0.0, swcr = 0.0;
    for (int i = i0; i < i1; ++i) {
      if (!(sg[i] < sf[i])) continue;
      const int64_t row = (int64_t)r * NP + i;
      const double d = __dsub_rn(sf[i], sg[i]), F = Fi[row];
      sw = __dadd_rn(sw, d);
      swf = __dadd_rn(swf, __dmul_rn(d, F));
      swf2 = __dadd_rn(swf2, __dmul_rn(__dmul_rn(d, F), F));
      swcr = __dadd_rn(swcr, __dmul_rn(d, CRi[row]));
    }
    for (int o = 16; o >= 1; o >>= 1) {  // fixed-order tree: deterministic sums
      sw += __shfl_down_sync(0xffffffffu, sw, o);
      swf += __shfl_down_sync(0xffffffffu, swf, o);
      swf2 += __shfl_down_sync(0xffffffffu, swf2, o);
      swcr += __shfl_down_sync(0xffffffffu, swcr, o);
    }
    if (lane == 0) {
      ssum[warp][0] = sw;
      ssum[warp][1] = swf;
      ssum[warp][2] = swf2;
      ssum[warp][3] = swcr;
    }
    __syncthreads();
    if (tid == 0) {
      double a = 0.0, b = 0.0, c = 0.0, e = 0.0;
      for (int q = 0; q < (int)(blockDim.x >> 5); ++q) {
        a += ssum[q][0];
        b += ssum[q][1];
        c += ssum[q][2];
        e += ssum[q][3];
      }
      if (a > 0.0 && b > 0.0) {
        const int slot = mk[r];
        MF[(int64_t)r * H + slot] = c / b;
        MCR[(int64_t)r * H + slot] = e / a;
        mk[r] = (slot + 1) % H;
      }
    }
  }
  const int as0 = use_archive ? asize[r] : 0;  // rand/1 has no archive (asize null)
  for (int i = i0; i < i1; ++i) {
    int a = -2;
    if (sacc[i]) {
      a = -1;
      if (use_archive) {
        int slot;
        if (as0 + k < NP) {
          slot = as0 + k;
        } else {
          const uint4 w = sv_draw(seeds[r], 0u, (uint32_t)i, (uint32_t)gen, SV_P_ARCH);
          slot = (int)sv_below(w.x, (uint32_t)NP);
        }
        atomicMax(&owner[slot], i);
        a = slot;
      }
      ++k;
    }
    sact[i] = a;
  }
  __syncthreads();
  for (int i = tid; i < NP; i += blockDim.x) {
    int a = sact[i];
    if (a >= 0 && owner[a] != i) a = -1;  // a later row overwrote this slot
    act[i] = a;
    if (a != -2) f[i] = sg[i];
  }
  if (tid == 0 && use_archive) asize[r] = min(NP, as0 + nacc_total);
  __syncthreads();
}

__global__ void __launch_bounds__(SEL_THREADS)
    de_select_kernel(double* __restrict__ fx, const double* __restrict__ fu,
                     int32_t* __restrict__ asize, int32_t* __restrict__ action,
                     double* __restrict__ best, const uint64_t* __restrict__ seeds,
                     const GenCtl* __restrict__ ctl, int NP, int use_archive,
                     const double* __restrict__ Fi, const double* __restrict__ CRi,
                     double* __restrict__ MF, double* __restrict__ MCR, int32_t* __restrict__ mk,
                     int H, int count_skip) {
  extern __shared__ __align__(16) unsigned char sel_sm[];
  // the trials follow count_skip rows of this generation in the budget order
  const int count = max(0, min(ctl->count - count_skip, NP));
  de_select_run(fx, fu, asize, action, best, seeds, count, ctl->gen, NP, use_archive,
                blockIdx.x, sel_sm, Fi, CRi, MF, MCR, mk, H);
}

// accepted row ri (run r): archive <- old x (if slot), x <- u; one quad
__device__ __forceinline__ void de_apply_elem(double* __restrict__ X, const double* __restrict__ U,
                                              double* __restrict__ A,
                                              const int32_t* __restrict__ action, int NP, int D,
                                              int ld, int r, int64_t ri, int jq) {
  {
    const int a = action[ri];
    if (a == -2) return;
    double* xi = X + ri * ld;
    const double* ui = U + ri * ld;
    double* as = (a >= 0) ? A + ((int64_t)r * NP + a) * ld : nullptr;
    const int j0 = jq * 4;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int j = j0 + q;
      if (j >= D) break;
      if (as) as[j] = xi[j];
      xi[j] = ui[j];
    }
  }
}

// accepted rows: archive <- old x (if slot), x <- u
__global__ void de_apply_kernel(double* __restrict__ X, const double* __restrict__ U,
                                double* __restrict__ A, const int32_t* __restrict__ action, int R,
                                int NP, int D, int ld, FastDiv fq, FastDiv fnp) {
  const int nq = (D + 3) >> 2;
  const int64_t total = (int64_t)R * NP * nq;
  const bool fast = total < (1ll << 31);
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    const Split3 sp = split3(t, fast, fq, fnp);
    const int jq = sp.lo;
    const int64_t ri = sp.row;
    de_apply_elem(X, U, A, action, NP, D, ld, sp.hi, ri, jq);
  }
}

// ---------------------------------------------------------------- CSO
// pairing: one CTA per run sorts (Philox key, index) ascending with a bitonic
// network in shared memory (padded with keys past every real one) and takes
// the sorted indices two by two; the lower fitness wins (ties: the first)
constexpr int CSO_THREADS = 512;

__global__ void __launch_bounds__(CSO_THREADS)
    cso_pair_kernel(const double* __restrict__ fx, int32_t* __restrict__ pair,
                    const uint64_t* __restrict__ seeds, GenCtl* ctl, CtlSet cs, int NP,
                    int npow2) {
  extern __shared__ __align__(16) unsigned char cs_sm[];
  uint32_t* key = reinterpret_cast<uint32_t*>(cs_sm);
  int32_t* idx = reinterpret_cast<int32_t*>(key + npow2);
  const int r = blockIdx.x, tid = threadIdx.x;
  const unsigned long long gen = gen_of(ctl, cs);
  for (int i = tid; i < npow2; i += blockDim.x) {
    key[i] = (i < NP) ? sv_draw(seeds[r], 0u, (uint32_t)i, (uint32_t)gen, SV_P_CSO).x : 0xFFFFFFFFu;
    idx[i] = (i < NP) ? i : 0x7FFFFFFF;
  }
  __syncthreads();
  for (int size = 2; size <= npow2; size <<= 1) {
    for (int stride = size >> 1; stride > 0; stride >>= 1) {
      for (int t = tid; t < npow2 / 2; t += blockDim.x) {
        const int lo = 2 * t - (t & (stride - 1)), hi = lo + stride;
        const bool up = ((lo & size) == 0);
        const uint32_t ka = key[lo], kb = key[hi];
        const int ia = idx[lo], ib = idx[hi];
        const bool a_gt_b = (ka > kb) || (ka == kb && ia > ib);
        if (a_gt_b == up) {
          key[lo] = kb;
          key[hi] = ka;
          idx[lo] = ib;
          idx[hi] = ia;
        }
      }
      __syncthreads();
    }
  }
  const double* f = fx + (int64_t)r * NP;
  for (int k = tid; k < NP / 2; k += blockDim.x) {
    const int a = idx[2 * k], b = idx[2 * k + 1];
    const int w = (f[a] <= f[b]) ? a : b;
    pair[(int64_t)r * NP + 2 * k] = w;
    pair[(int64_t)r * NP + 2 * k + 1] = (w == a) ? b : a;
  }
}

// the swarm's mean position: one thread per (run, coordinate), rows summed
// in index order (the order of the definition), then divided by NP
__global__ void cso_mean_kernel(const double* __restrict__ X, double* __restrict__ xbar, int R,
                                int NP, int D, int ld) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= D) return;
  for (int r = blockIdx.y; r < R; r += gridDim.y) {
    const double* Xr = X + (int64_t)r * NP * ld + j;
    double s = 0.0;
    for (int i = 0; i < NP; ++i) s = __dadd_rn(s, Xr[(int64_t)i * ld]);
    xbar[(int64_t)r * ld + j] = __ddiv_rn(s, (double)NP);
  }
}

// the loser of pair k, coordinate j: velocity and position update (the
// multiply-adds fused as in the definition); the new position is also written
// to row k of the run's block of U (the rows to evaluate)
__global__ void cso_update_kernel(double* __restrict__ X, double* __restrict__ V,
                                  double* __restrict__ U, const int32_t* __restrict__ pair,
                                  const double* __restrict__ xbar,
                                  const uint64_t* __restrict__ seeds,
                                  const GenCtl* __restrict__ ctl, int R, int NP, int D, int ld,
                                  double phi, double lb, double ub, FastDiv fd, FastDiv fhalf) {
  const int half = NP / 2;
  const int64_t total = (int64_t)R * half * D;
  const bool fast = total < (1ll << 31);
  const unsigned long long gen = ctl->gen;
  const SvBound lbb = sv_bound(lb), ubb = sv_bound(ub);
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    const Split3 sp = split3(t, fast, fd, fhalf);
    const int j = sp.lo, k = sp.mid, r = sp.hi;
    const int64_t r0 = (int64_t)r * NP;
    const int w = pair[r0 + 2 * k], l = pair[r0 + 2 * k + 1];
    const uint64_t seed = seeds[r];
    const uint4 a = sv_draw(seed, (uint32_t)(1 + 2 * j), (uint32_t)l, (uint32_t)gen, SV_P_CSO);
    const uint4 b = sv_draw(seed, (uint32_t)(2 + 2 * j), (uint32_t)l, (uint32_t)gen, SV_P_CSO);
    const double R1 = u53_int(a.x, a.y), R2 = u53_int(a.z, a.w), R3 = u53_int(b.x, b.y);
    const int64_t el = (r0 + l) * ld + j;
    const double xl = X[el], xw = X[(r0 + w) * ld + j];
    const double v =
        __fma_rn(R1, V[el],
                 __fma_rn(R2, __dsub_rn(xw, xl),
                          __dmul_rn(__dmul_rn(phi, R3), __dsub_rn(xbar[(int64_t)r * ld + j], xl))));
    double x = __dadd_rn(xl, v);
    if (sv_lt_bound(x, lbb)) x = lb;
    if (sv_gt_bound(x, ubb)) x = ub;
    V[el] = v;
    X[el] = x;
    U[((int64_t)r * half + k) * ld + j] = x;
  }
}

// losers' fitness into fx; best-so-far over the first `count` losers
__global__ void __launch_bounds__(SEL_THREADS)
    cso_scatter_kernel(double* __restrict__ fx, const double* __restrict__ fu,
                       const int32_t* __restrict__ pair, double* __restrict__ best,
                       const GenCtl* __restrict__ ctl, int NP) {
  const int r = blockIdx.x, half = NP / 2, count = ctl->count;
  double m = INFINITY;
  for (int k = threadIdx.x; k < half; k += blockDim.x) {
    const double v = fu[(int64_t)r * half + k];
    fx[(int64_t)r * NP + pair[(int64_t)r * NP + 2 * k + 1]] = v;
    if (k < count) m = dmin_pos(m, v);
  }
  block_min_update(m, best + r);
}

// the same, in place: x <- moved x, v <- moved v
__device__ __forceinline__ void pso_move_elem(double* __restrict__ X, double* __restrict__ V,
                                              const double* __restrict__ P,
                                              const int32_t* __restrict__ guide,
                                              const uint64_t* __restrict__ seeds,
                                              unsigned long long gen, int NP, int ld, double w,
                                              double c1, double c2, double lb, double ub, int r,
                                              int i, int j, int64_t ri) {
  const int64_t e = ri * ld + j;
  double v;
  const double xn = pso_moved(X, V, P, guide, seeds, gen, NP, ld, w, c1, c2, lb, ub, r, i, j, ri,
                              e, &v);
  X[e] = xn;
  V[e] = v;
}

__global__ void pso_move_kernel(double* __restrict__ X, double* __restrict__ V,
                                const double* __restrict__ P, const int32_t* __restrict__ guide,
                                const uint64_t* __restrict__ seeds, GenCtl* ctl, CtlSet cs,
                                int R, int NP, int D, int ld, double w, double c1, double c2,
                                double lb, double ub, FastDiv fd, FastDiv fnp,
                                float* __restrict__ Ad, int apitch,
                                const float* __restrict__ Osp) {
  const int64_t total = (int64_t)R * NP * D;
  const bool fast = total < (1ll << 31);
  const unsigned long long gen = gen_of(ctl, cs);
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    const Split3 sp = split3(t, fast, fd, fnp);
    const int64_t e = sp.row * ld + sp.lo;
    double v;
    const double xn = pso_moved(X, V, P, guide, seeds, gen, NP, ld, w, c1, c2, lb, ub, sp.hi,
                                sp.mid, sp.lo, sp.row, e, &v);
    X[e] = xn;
    V[e] = v;
    if (Ad) {
      const int64_t o = (int64_t)sp.hi * apitch + sp.lo;
      Ad[sp.row * apitch + sp.lo] = tc::to_tf32(
          sv_operand_d(xn, __ldg(Osp + o), __ldg(Osp + o + (int64_t)R * apitch)));
    }
  }
}

// run r by the whole block: strict pbest update flags, best-so-far, guides
// (gbest / ring); sp: NP doubles of shared memory
__device__ __forceinline__ void pso_update_run(const double* __restrict__ fx,
                                               double* __restrict__ fp, int32_t* __restrict__ flag,
                                               int32_t* __restrict__ guide,
                                               double* __restrict__ best, int count, int NP,
                                               int topology, int update_best, int r, double* sp) {
  __shared__ long long kbest[SEL_THREADS / 32];
  __shared__ int ibest[SEL_THREADS / 32];
  const int tid = threadIdx.x;
  const double* f = fx + (int64_t)r * NP;
  double* p = fp + (int64_t)r * NP;
  int32_t* fl = flag + (int64_t)r * NP;
  int32_t* gd = guide + (int64_t)r * NP;
  if (update_best) {
    double m = INFINITY;
    for (int i = tid; i < count; i += blockDim.x) m = dmin_pos(m, f[i]);
    block_min_update(m, best + r);
  }
  for (int i = tid; i < NP; i += blockDim.x) {
    const double fi = f[i];
    double pi = p[i];
    const bool up = fi < pi;
    fl[i] = up;
    if (up) {
      p[i] = fi;
      pi = fi;
    }
    sp[i] = pi;
  }
  __syncthreads();
  if (topology == 0) {
    long long kb = 0x7FFFFFFFFFFFFFFFll;
    int ib = 0x7FFFFFFF;
    for (int i = tid; i < NP; i += blockDim.x) {
      const long long k = fkey(sp[i]);
      if (k < kb || (k == kb && i < ib)) {
        kb = k;
        ib = i;
      }
    }
    for (int o = 16; o >= 1; o >>= 1) {
      const long long k2 = __shfl_xor_sync(0xffffffffu, kb, o);
      const int i2 = __shfl_xor_sync(0xffffffffu, ib, o);
      if (k2 < kb || (k2 == kb && i2 < ib)) {
        kb = k2;
        ib = i2;
      }
    }
    if ((tid & 31) == 0) {
      kbest[tid >> 5] = kb;
      ibest[tid >> 5] = ib;
    }
    __syncthreads();
    if (tid == 0) {
      for (int w = 1; w < (int)(blockDim.x >> 5); ++w)
        if (kbest[w] < kbest[0] || (kbest[w] == kbest[0] && ibest[w] < ibest[0])) {
          kbest[0] = kbest[w];
          ibest[0] = ibest[w];
        }
    }
    __syncthreads();
    const int b = ibest[0];
    for (int i = tid; i < NP; i += blockDim.x) gd[i] = b;
  } else {
    for (int i = tid; i < NP; i += blockDim.x) {
      int nb[3] = {(i + NP - 1) % NP, i, (i + 1) % NP};
      // ascending indices, then strict improvement keeps the lowest index
      for (int a = 0; a < 2; ++a)
        for (int c = 0; c < 2 - a; ++c)
          if (nb[c] > nb[c + 1]) {
            int t = nb[c];
            nb[c] = nb[c + 1];
            nb[c + 1] = t;
          }
      int b = nb[0];
      for (int t = 1; t < 3; ++t)
        if (sp[nb[t]] < sp[b]) b = nb[t];
      gd[i] = b;
    }
  }
  __syncthreads();
}

__global__ void __launch_bounds__(SEL_THREADS)
    pso_update_kernel(const double* __restrict__ fx, double* __restrict__ fp,
                      int32_t* __restrict__ flag, int32_t* __restrict__ guide,
                      double* __restrict__ best, const GenCtl* __restrict__ ctl, int NP,
                      int topology, int use_count, int update_best) {
  extern __shared__ double sp_sm[];  // the run's personal-best fitness
  pso_update_run(fx, fp, flag, guide, best, use_count ? min(ctl->count, NP) : NP, NP, topology,
                 update_best, blockIdx.x, sp_sm);
}

// improved row ri: pbest <- x, one quad
__device__ __forceinline__ void pso_copy_elem(double* __restrict__ P, const double* __restrict__ X,
                                              const int32_t* __restrict__ flag, int D, int ld,
                                              int64_t ri, int jq) {
  if (!flag[ri]) return;
  const int j0 = jq * 4;
  double* pi = P + ri * ld;
  const double* xi = X + ri * ld;
#pragma unroll
  for (int q = 0; q < 4; ++q)
    if (j0 + q < D) pi[j0 + q] = xi[j0 + q];
}

// improved rows: pbest <- x
__global__ void pso_copy_kernel(double* __restrict__ P, const double* __restrict__ X,
                                const int32_t* __restrict__ flag, int R, int NP, int D, int ld,
                                FastDiv fq, FastDiv fnp) {
  const int nq = (D + 3) >> 2;
  const int64_t total = (int64_t)R * NP * nq;
  const bool fast = total < (1ll << 31);
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    const Split3 sp = split3(t, fast, fq, fnp);
    pso_copy_elem(P, X, flag, D, ld, sp.row, sp.lo);
  }
}

// ---------------------------------------------------------------- PSODE
// The PSO component's offspring: particle i moves from the population X with
// the carried velocity V into Y; X and V are left as they are (the moved
// velocity is not kept: the generation ends by setting V to the DE
// displacement)
__global__ void psode_move_kernel(const double* __restrict__ X, const double* __restrict__ V,
                                  const double* __restrict__ P,
                                  const int32_t* __restrict__ guide, double* __restrict__ Y,
                                  const uint64_t* __restrict__ seeds,
                                  GenCtl* ctl, CtlSet cs, int R, int NP, int D, int ld,
                                  double w, double c1, double c2, double lb, double ub,
                                  FastDiv fd, FastDiv fnp) {
  const int64_t total = (int64_t)R * NP * D;
  const bool fast = total < (1ll << 31);
  const unsigned long long gen = gen_of(ctl, cs);
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    const Split3 sp = split3(t, fast, fd, fnp);
    const int64_t e = sp.row * ld + sp.lo;
    double v;
    Y[e] = pso_moved(X, V, P, guide, seeds, gen, NP, ld, w, c1, c2, lb, ub, sp.hi, sp.mid, sp.lo,
                     sp.row, e, &v);
  }
}

// pairwise/3 choice per row, after the DE selection left the survivor's
// fitness f3 in fx: the PSO offspring is taken when strictly better.  action
// becomes bit 0 = DE trial accepted, bit 1 = PSO offspring taken.
__global__ void psode_pick_kernel(double* __restrict__ fx, const double* __restrict__ fy,
                                  int32_t* __restrict__ action, int64_t rows) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < rows;
       t += (int64_t)gridDim.x * blockDim.x) {
    const double f3 = fx[t], y = fy[t];
    const bool take = y < f3;
    if (take) fx[t] = y;
    action[t] = (action[t] != -2 ? 1 : 0) | (take ? 2 : 0);
  }
}

// per element, one quad of row ri: x3 = u if the DE trial was accepted else
// x; v <- x3 - x (the DE displacement); x <- y if the PSO offspring was
// taken else x3
__global__ void psode_combine_kernel(double* __restrict__ X, const double* __restrict__ U,
                                     const double* __restrict__ Y, double* __restrict__ V,
                                     const int32_t* __restrict__ action, int R, int NP, int D,
                                     int ld, FastDiv fq, FastDiv fnp) {
  const int nq = (D + 3) >> 2;
  const int64_t total = (int64_t)R * NP * nq;
  const bool fast = total < (1ll << 31);
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    const Split3 sp = split3(t, fast, fq, fnp);
    const int code = action[sp.row];
    const int j0 = sp.lo * 4;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      if (j0 + q >= D) break;
      const int64_t e = sp.row * ld + j0 + q;
      const double x = X[e];
      const double x3 = (code & 1) ? U[e] : x;
      V[e] = __dsub_rn(x3, x);
      X[e] = (code & 2) ? Y[e] : x3;
    }
  }
}

__global__ void fill_kernel(double* __restrict__ a, int64_t n, double v) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n;
       t += (int64_t)gridDim.x * blockDim.x)
    a[t] = v;
}

// ---------------------------------------------------------------- small runs
// One CTA per run carries whole generations of a small run (D <= 32,
// NP <= 512): launched with G > 1 it runs G consecutive generations without
// returning to the host.  The operators are the batched kernels' device
// functions above (same draws, same arithmetic); the evaluation is a warp
// per row on CUDA cores -- FP64, or FP32 with the operand rounding of the
// requested mode (TF32, BF16 hi/lo products, plain FP32) and FP64
// refinement below the threshold -- so one evaluator serves a run throughout.
constexpr int SRK_THREADS = 256;
constexpr int SRK_MAX_D = 32, SRK_MAX_NP = 512;

struct SrkArgs {
  double *X, *fx, *U, *fu, *A, *V, *P, *fp, *best;
  int32_t *asize, *guide, *part, *order, *action;
  const uint64_t* seeds;
  const ProblemDev* const* rp;
  const GenCtl* ctl;
  unsigned long long* refined;
  int NP, D, ld, pk, topology;
  double F, lb, ub, w, c1, c2;
  unsigned long long cr_thr;
  long long budget;
};

__host__ __device__ inline size_t srk_smem_bytes(int NP) {
  const size_t a = sel_smem_bytes(NP), b = (size_t)NP * 8;
  return a > b ? a : b;
}

__device__ __forceinline__ void warp_sum64(int body, Acc64& a) {
#pragma unroll
  for (int m = 16; m >= 1; m >>= 1) {
    const double b0 = __shfl_xor_sync(0xffffffffu, a.a0, m);
    const double b1 = __shfl_xor_sync(0xffffffffu, a.a1, m);
    const double b2 = __shfl_xor_sync(0xffffffffu, a.a2, m);
    a.a0 += b0;
    a.a1 = slot1_is_product64(body) ? a.a1 * b1 : a.a1 + b1;
    a.a2 += b2;
  }
}

__device__ __forceinline__ void warp_sum32(Acc32& a) {
#pragma unroll
  for (int m = 16; m >= 1; m >>= 1) {
    a.a0 += __shfl_xor_sync(0xffffffffu, a.a0, m);
    a.a1 += __shfl_xor_sync(0xffffffffu, a.a1, m);
    a.a2 += __shfl_xor_sync(0xffffffffu, a.a2, m);
  }
}

__device__ __forceinline__ double warp_sumd(double v) {
#pragma unroll
  for (int m = 16; m >= 1; m >>= 1) v += __shfl_xor_sync(0xffffffffu, v, m);
  return v;
}

// FP64 error of row x by one warp: lane = coordinate (D <= 32)
__device__ double srk_eval64(const ProblemDev& P, const double* __restrict__ x, int lane) {
  const int D = P.D;
  const bool comp = (P.weighted);
  const double xj = (lane < D) ? x[lane] : 0.0;
  double gv[SV_MAXC], sv[SV_MAXC];
  double total = 0.0;
  for (int c = 0; c < P.ncomp; ++c) {
    const double dj = (lane < D) ? __dsub_rn(xj, P.o[c][lane]) : 0.0;
    const double* __restrict__ MT = P.MT64[c];
    double z = 0.0;
    for (int j = 0; j < D; ++j) {
      const double dd = __shfl_sync(0xffffffffu, dj, j);
      if (lane < D) z = __fma_rn(MT[(size_t)j * D + lane], dd, z);
    }
    const int gi = (lane < D) ? P.gid[c][lane] : -1;
    const double zn = __shfl_down_sync(0xffffffffu, z, 1);
    const int gn = __shfl_down_sync(0xffffffffu, gi, 1);
    const int ng = P.ngc[c];
    double gc = 0.0;
    for (int g = 0; g < ng; ++g) {
      const int body = P.gbody[c][g];
      Acc64 a;
      acc64_init(body, a);
      if (lane < D && gi == g)
        term64(body, z, P.aux64[c][lane], lane + 1 < D && gn == g, zn, P, a);
      warp_sum64(body, a);
      gc += finalize64(body, a, P.gstart[c][g + 1] - P.gstart[c][g]);
    }
    if (comp) {
      gv[c] = gc;
      sv[c] = warp_sumd(dj * dj);
    } else {
      total = gc;
    }
  }
  const double err = comp ? compose(P, sv, gv) : total;
  return isfinite(err) ? err : __longlong_as_double(0x7ff8000000000000ll);
}

// mixed-precision error of row x by one warp; rows below the refinement
// threshold are re-evaluated by srk_eval64 (*refined = true)
template <int PREC>
__device__ double srk_eval32(const ProblemDev& P, const double* __restrict__ x, int lane,
                             bool* refined) {
  const int D = P.D;
  const bool comp = (P.weighted);
  float xh = 0.f, xl = 0.f;
  if (lane < D) sv_split_hi_lo(x[lane], xh, xl);
  double gv[SV_MAXC], sv[SV_MAXC];
  double total = 0.0;
  for (int c = 0; c < P.ncomp; ++c) {
    const float d = (lane < D) ? (xh - P.oh32[c][lane]) + (xl - P.ol32[c][lane]) : 0.f;
    float z = 0.f;
    if (PREC == SEVO_FP32) {
      const float* __restrict__ MT = P.MT32[c];
      for (int j = 0; j < D; ++j) {
        const float dd = __shfl_sync(0xffffffffu, d, j);
        if (lane < D) z = fmaf(MT[(size_t)j * D + lane], dd, z);
      }
    } else if (PREC == SEVO_TF32) {
      const float dt = tc::to_tf32(d);
      const float* __restrict__ Mr = P.M32[c] + (size_t)lane * P.kpad;
      for (int j = 0; j < D; ++j) {
        const float dd = __shfl_sync(0xffffffffu, dt, j);
        if (lane < D) z = fmaf(Mr[j], dd, z);
      }
    } else {  // BF16X3: hi*hi + hi*lo + lo*hi, products exact in FP32
      const __nv_bfloat16 h = __float2bfloat16_rn(d);
      const float dh = __bfloat162float(h);
      const float dl = __bfloat162float(__float2bfloat16_rn(d - dh));
      const __nv_bfloat16* __restrict__ Mh = P.Mhi[c] + (size_t)lane * P.kpad;
      const __nv_bfloat16* __restrict__ Ml = P.Mlo[c] + (size_t)lane * P.kpad;
      for (int j = 0; j < D; ++j) {
        const float hj = __shfl_sync(0xffffffffu, dh, j), lj = __shfl_sync(0xffffffffu, dl, j);
        if (lane < D) {
          const float mh = __bfloat162float(Mh[j]), ml = __bfloat162float(Ml[j]);
          z = fmaf(mh, hj, z);
          z = fmaf(mh, lj, z);
          z = fmaf(ml, hj, z);
        }
      }
    }
    const int gi = (lane < D) ? P.gid[c][lane] : -1;
    const float zn = __shfl_down_sync(0xffffffffu, z, 1);
    const int gn = __shfl_down_sync(0xffffffffu, gi, 1);
    const int ng = P.ngc[c];
    double gc = 0.0;
    for (int g = 0; g < ng; ++g) {
      const int body = P.gbody[c][g];
      Acc32 a;
      acc32_init(a);
      if (lane < D && gi == g)
        term32t<PREC == SEVO_TF32>(body, z, P.aux32[c][lane], lane + 1 < D && gn == g, zn, P, a);
      warp_sum32(a);
      gc += (double)finalize32(body, a, P.gstart[c][g + 1] - P.gstart[c][g]);
    }
    if (comp) {
      gv[c] = gc;
      sv[c] = warp_sumd((double)(d * d));
    } else {
      total = gc;
    }
  }
  double err = comp ? compose(P, sv, gv) : total;
  if (!isfinite(err)) return __longlong_as_double(0x7ff8000000000000ll);
  if (err < SEVO_REFINE_THRESHOLD) {
    err = srk_eval64(P, x, lane);
    *refined = true;
  }
  return err;
}

template <int PREC>
__device__ __forceinline__ double srk_eval(const ProblemDev& P, const double* x, int lane,
                                           bool* refined) {
  if (PREC == SEVO_FP64) return srk_eval64(P, x, lane);
  return srk_eval32<PREC>(P, x, lane, refined);
}

// advance = 0: one generation with the counter and count of ctl;
// advance = 1: G generations gen0 + 1 .. gen0 + G (gen0 = ctl->gen), each
// with the evaluation count ctl_advance_kernel would give it
template <int ALG, int PREC>
__global__ void __launch_bounds__(SRK_THREADS)
    srk_kernel(const SrkArgs a, int G, int advance) {
  extern __shared__ __align__(16) unsigned char srk_sm[];
  __shared__ ProblemDev P;
  const int r = blockIdx.x, tid = threadIdx.x, lane = tid & 31;
  const int nwarp = blockDim.x >> 5, warp = tid >> 5;
  {  // the run's problem descriptor, with the Schwefel constant computed by
     // the device sin as in the FP64 bodies (term exactly 0 at the optimum)
    const int* src = reinterpret_cast<const int*>(a.rp[r]);
    int* dst = reinterpret_cast<int*>(&P);
    for (int q = tid; q < (int)(sizeof(ProblemDev) / 4); q += blockDim.x) dst[q] = src[q];
    __syncthreads();
    if (tid == 0) P.sch_c = __dmul_rn(P.sch_s, sin(sqrt(P.sch_s)));
    __syncthreads();
  }
  const int NP = a.NP, D = a.D, nq = (D + 3) >> 2;
  const int64_t r0 = (int64_t)r * NP;
  unsigned long long gen = a.ctl->gen;
  int count = a.ctl->count;
  unsigned long long nref = 0;
  for (int k = 0; k < G; ++k) {
    if (advance) {
      ++gen;
      const long long c = a.budget - ((long long)NP + (long long)(gen - 1) * NP);
      count = (int)(c < 0 ? 0 : (c > NP ? NP : c));
    }
    if (ALG == SEVO_DE_RAND1 || ALG == SEVO_DE_CTPB) {
      if (ALG == SEVO_DE_CTPB)
        rank_run_block(a.fx + r0, a.order + r0, NP, a.pk, reinterpret_cast<long long*>(srk_sm));
      for (int t = tid; t < NP * nq; t += blockDim.x) {
        const int i = t / nq;
        de_trial_elem<ALG>(a.X, a.U, a.A, a.asize, a.order, a.part, a.seeds, NP, D, a.ld, a.F,
                           a.cr_thr, a.lb, a.ub, a.pk, gen, r, i, t - i * nq);
      }
      __syncthreads();
      for (int i = warp; i < NP; i += nwarp) {
        bool ref = false;
        const double e = srk_eval<PREC>(P, a.U + (r0 + i) * a.ld, lane, &ref);
        if (lane == 0) {
          a.fu[r0 + i] = e;
          nref += ref;
        }
      }
      __syncthreads();
      de_select_run(a.fx, a.fu, a.asize, a.action, a.best, a.seeds, count, gen, NP,
                    ALG == SEVO_DE_CTPB, r, srk_sm);
      for (int t = tid; t < NP * nq; t += blockDim.x) {
        const int i = t / nq;
        de_apply_elem(a.X, a.U, a.A, a.action, NP, D, a.ld, r, r0 + i, t - i * nq);
      }
      __syncthreads();
    } else {
      for (int t = tid; t < NP * D; t += blockDim.x) {
        const int i = t / D;
        pso_move_elem(a.X, a.V, a.P, a.guide, a.seeds, gen, NP, a.ld, a.w, a.c1, a.c2, a.lb, a.ub,
                      r, i, t - i * D, r0 + i);
      }
      __syncthreads();
      for (int i = warp; i < NP; i += nwarp) {
        bool ref = false;
        const double e = srk_eval<PREC>(P, a.X + (r0 + i) * a.ld, lane, &ref);
        if (lane == 0) {
          a.fx[r0 + i] = e;
          nref += ref;
        }
      }
      __syncthreads();
      pso_update_run(a.fx, a.fp, a.action, a.guide, a.best, count, NP, a.topology, 1, r,
                     reinterpret_cast<double*>(srk_sm));
      for (int t = tid; t < NP * nq; t += blockDim.x) {
        const int i = t / nq;
        pso_copy_elem(a.P, a.X, a.action, D, a.ld, r0 + i, t - i * nq);
      }
      __syncthreads();
    }
  }
  if (PREC != SEVO_FP64 && lane == 0 && nref) atomicAdd(a.refined, nref);
}

template <int ALG>
cudaError_t srk_launch_prec(const Batch* b, const SrkArgs& a, int G, int advance) {
  const size_t sm = srk_smem_bytes(b->NP);
  switch (b->prec) {
    case SEVO_FP64: srk_kernel<ALG, SEVO_FP64><<<b->R, SRK_THREADS, sm, b->stream>>>(a, G, advance); break;
    case SEVO_TF32: srk_kernel<ALG, SEVO_TF32><<<b->R, SRK_THREADS, sm, b->stream>>>(a, G, advance); break;
    case SEVO_BF16X3: srk_kernel<ALG, SEVO_BF16X3><<<b->R, SRK_THREADS, sm, b->stream>>>(a, G, advance); break;
    default: srk_kernel<ALG, SEVO_FP32><<<b->R, SRK_THREADS, sm, b->stream>>>(a, G, advance); break;
  }
  return cudaGetLastError();
}

cudaError_t srk_launch(const Batch* b, int G, int advance) {
  SrkArgs a;
  a.X = b->X;
  a.fx = b->fx;
  a.U = b->U;
  a.fu = b->fu;
  a.A = b->A;
  a.V = b->V;
  a.P = b->P;
  a.fp = b->fp;
  a.best = b->best;
  a.asize = b->asize;
  a.guide = b->guide;
  a.part = b->part;
  a.order = b->order;
  a.action = b->action;
  a.seeds = b->seeds;
  a.rp = b->rp;
  a.ctl = b->ctl;
  a.refined = b->refined;
  a.NP = b->NP;
  a.D = b->D;
  a.ld = b->ld;
  a.pk = b->pbest_k;
  a.topology = (b->alg == SEVO_PSO_RING) ? 1 : 0;
  a.F = b->F;
  a.lb = b->lb;
  a.ub = b->ub;
  a.w = b->w;
  a.c1 = b->c1;
  a.c2 = b->c2;
  a.cr_thr = b->cr_thr;
  a.budget = (long long)b->budget;
  switch (b->alg) {
    case SEVO_DE_RAND1: return srk_launch_prec<SEVO_DE_RAND1>(b, a, G, advance);
    case SEVO_DE_CTPB: return srk_launch_prec<SEVO_DE_CTPB>(b, a, G, advance);
    case SEVO_PSO_GBEST: return srk_launch_prec<SEVO_PSO_GBEST>(b, a, G, advance);
    default: return srk_launch_prec<SEVO_PSO_RING>(b, a, G, advance);
  }
}

// Grid of a grid-stride streaming kernel: at most 1024 threads per SM, so
// that the whole grid is dispatched at once and kernels of other streams
// queued behind it still find room on every SM (the CTA dispatcher serves
// grids of equal priority in launch order)
unsigned grid_for(int64_t work, int threads) {
  int64_t b = (work + threads - 1) / threads;
  int64_t cap = (int64_t)sv_num_sms() * std::max(1, 1024 / threads);
  if (b > cap) b = cap;
  if (b < 1) b = 1;
  return (unsigned)b;
}

}  // namespace

#include "post.cuh"

// ====================================================================== host
static std::atomic<int> g_policy_small_runs{0};
static std::atomic<int> g_policy_refine{1};
static std::atomic<long long> g_policy_test_wait{0};
static std::atomic<int> g_policy_fuse_ops{0};

int sv_policy_fuse_ops() { return g_policy_fuse_ops.load(); }

int sv_policy_refine() { return g_policy_refine.load(); }
long long sv_policy_test_wait() { return g_policy_test_wait.load(); }

extern "C" int32_t sevo_set_policy(int32_t key, int64_t value) {
  if (key == SEVO_POLICY_AUTOTUNE) return sv_tune_set_policy(value);
  if (key == SEVO_POLICY_TEST_WAIT) {
    if (value < 0 || value > SEVO_TEST_WAIT_MAX) return SEVO_ERR_ARG;
    g_policy_test_wait.store((long long)value);
    return SEVO_OK;
  }
  if (value != 0 && value != 1) return SEVO_ERR_ARG;
  if (key == SEVO_POLICY_SMALL_RUNS) {
    g_policy_small_runs.store((int)value);
  } else if (key == SEVO_POLICY_REFINE) {
    g_policy_refine.store((int)value);
  } else if (key == SEVO_POLICY_FUSE_OPS) {
    g_policy_fuse_ops.store((int)value);
  } else {
    return SEVO_ERR_ARG;
  }
  return SEVO_OK;
}

extern "C" int64_t sevo_get_policy(int32_t key) {
  if (key == SEVO_POLICY_SMALL_RUNS) return g_policy_small_runs.load();
  if (key == SEVO_POLICY_REFINE) return g_policy_refine.load();
  if (key == SEVO_POLICY_TEST_WAIT) return g_policy_test_wait.load();
  if (key == SEVO_POLICY_FUSE_OPS) return g_policy_fuse_ops.load();
  if (key == SEVO_POLICY_AUTOTUNE) return sv_policy_autotune();
  return -1;
}

int sv_pbest_k(double p, int NP) {
  int k = (int)std::ceil(p * (double)NP - 1e-9);
  if (k < 1) k = 1;
  if (k > NP) k = NP;
  return k;
}

static size_t al256(size_t b) { return (b + 255) & ~(size_t)255; }

int32_t sv_batch_alloc(Batch* b, const std::vector<const sevo_problem*>& probs,
                       const std::vector<uint64_t>& seeds, const sevo_alg_params* a,
                       cudaStream_t st) {
  b->alg = a->alg;
  b->D = probs[0]->D;
  b->NP = a->NP;
  b->R = (int)probs.size();
  b->ld = (b->D + 1) & ~1;
  b->F = a->F;
  b->CR = a->CR;
  b->p = a->p;
  b->w = a->w;
  b->c1 = a->c1;
  b->c2 = a->c2;
  b->lb = a->lb;
  b->ub = a->ub;
  b->budget = a->budget;
  b->prec = a->prec;
  b->stream = st;
  {
    double t = std::ceil(a->CR * 4294967296.0);
    if (t < 0) t = 0;
    if (t > 4294967296.0) t = 4294967296.0;
    b->cr_thr = (unsigned long long)t;
  }
  b->pbest_k = sv_pbest_k(a->p, a->NP);
  if (sv_has_shade(b->alg)) {  // largest pool: round(max(0.2, 2/NP) NP)
    const double pm = std::max(0.2, 2.0 / (double)a->NP);
    b->pbest_k = std::min(a->NP, std::max(1, (int)std::floor(pm * (double)a->NP + 0.5)));
  }
  b->small = g_policy_small_runs.load() != 0 && b->D <= SRK_MAX_D && b->NP <= SRK_MAX_NP &&
             (b->alg == SEVO_DE_RAND1 || b->alg == SEVO_DE_CTPB || b->alg == SEVO_PSO_GBEST ||
              b->alg == SEVO_PSO_RING);
  b->per_gen = (b->alg == SEVO_CSO) ? b->NP / 2 : (b->alg == SEVO_PSODE) ? 2 * b->NP : b->NP;
  b->run_prob = probs;
  b->seg_begin.clear();
  for (int r = 0; r < b->R; ++r)
    if (r == 0 || probs[r] != probs[r - 1]) b->seg_begin.push_back(r);
  b->seg_begin.push_back(b->R);
  const int64_t rows = (int64_t)b->R * b->NP;
  const size_t mat = al256((size_t)rows * b->ld * 8), vec = al256((size_t)rows * 8),
               ivec = al256((size_t)rows * 4);
  const bool de = sv_is_de(b->alg), psode = (b->alg == SEVO_PSODE);
  const bool ctpb = (b->alg == SEVO_DE_CTPB), shade = sv_has_shade(b->alg);
  size_t bytes = mat /*X*/ + vec /*fx*/ + al256((size_t)b->R * 8) /*best*/ + al256(16) /*err*/ +
                 al256(8) /*refined*/ + al256((size_t)b->R * 8) /*rp*/ +
                 al256((size_t)b->R * 8) /*seeds*/ + al256(sizeof(GenCtl)) + ivec /*guide/flag*/ +
                 al256((size_t)rows * 16) /*part*/ + ivec /*action*/;
  const bool cso = (b->alg == SEVO_CSO), pso = sv_has_pbest(b->alg);
  if (de || cso || psode) bytes += mat /*U*/ + vec /*fu*/;
  if (psode) bytes += mat /*Y*/ + vec /*fy*/;
  if (cso) bytes += mat /*V*/ + ivec /*pair*/ + al256((size_t)b->R * b->ld * 8) /*xbar*/;
  if (ctpb) bytes += mat /*A*/ + al256((size_t)b->R * 4) /*asize*/ + ivec /*order*/;
  if (shade)
    bytes += ivec /*order*/ + 2 * al256((size_t)b->R * SEVO_SHADE_H * 8) /*MF, MCR*/ +
             al256((size_t)b->R * 4) /*mk*/ + 2 * vec /*Fi, CRi*/ + ivec /*kpb*/;
  if (pso) bytes += 2 * mat /*V,P*/ + vec /*fp*/;
  b->block_bytes = bytes;
  if ((ctpb || shade) && rsel_smem_bytes(b->NP) > 48 * 1024)
    SV_CUDA(cudaFuncSetAttribute(de_rank_select_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)rsel_smem_bytes(SV_MAX_NP)));
  if (ctpb && post_cand_bytes(pow2_at_least(b->pbest_k)) > 48 * 1024)
    SV_CUDA(cudaFuncSetAttribute(de_post_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)post_cand_bytes(SV_MAX_NP)));
  if ((de || psode) && sel_smem_bytes(b->NP) > 48 * 1024)
    SV_CUDA(cudaFuncSetAttribute(de_select_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)sel_smem_bytes(SV_MAX_NP)));
  SV_CUDA(cudaMalloc(&b->block, bytes));
  SV_CUDA(cudaMemsetAsync(b->block, 0, bytes, st));
  char* c = (char*)b->block;
  auto take = [&](size_t n) {
    char* p = c;
    c += n;
    return p;
  };
  b->X = (double*)take(mat);
  b->fx = (double*)take(vec);
  b->best = (double*)take(al256((size_t)b->R * 8));
  b->err = (uint32_t*)take(al256(16));
  b->refined = (unsigned long long*)take(al256(8));
  b->rp = (const ProblemDev**)take(al256((size_t)b->R * 8));
  b->seeds = (uint64_t*)take(al256((size_t)b->R * 8));
  b->ctl = (GenCtl*)take(al256(sizeof(GenCtl)));
  b->guide = (int32_t*)take(ivec);
  b->part = (int32_t*)take(al256((size_t)rows * 16));
  b->action = (int32_t*)take(ivec);
  b->U = b->fu = b->A = b->V = b->P = b->fp = nullptr;
  b->asize = b->order = nullptr;
  b->xbar = nullptr;
  b->Y = b->fy = nullptr;
  if (de || cso || psode) {
    b->U = (double*)take(mat);
    b->fu = (double*)take(vec);
  }
  if (psode) {
    b->Y = (double*)take(mat);
    b->fy = (double*)take(vec);
  }
  if (cso) {
    b->V = (double*)take(mat);
    b->order = (int32_t*)take(ivec);  // the pairing: winner, loser of pair k at 2k, 2k + 1
    b->xbar = (double*)take(al256((size_t)b->R * b->ld * 8));
  }
  if (ctpb) {
    b->A = (double*)take(mat);
    b->asize = (int32_t*)take(al256((size_t)b->R * 4));
    b->order = (int32_t*)take(ivec);
  }
  b->MF = b->MCR = b->Fi = b->CRi = nullptr;
  b->mk = b->kpb = nullptr;
  if (shade) {
    b->order = (int32_t*)take(ivec);
    b->MF = (double*)take(al256((size_t)b->R * SEVO_SHADE_H * 8));
    b->MCR = (double*)take(al256((size_t)b->R * SEVO_SHADE_H * 8));
    b->mk = (int32_t*)take(al256((size_t)b->R * 4));
    b->Fi = (double*)take(vec);
    b->CRi = (double*)take(vec);
    b->kpb = (int32_t*)take(ivec);
  }
  if (pso) {
    b->V = (double*)take(mat);
    b->P = (double*)take(mat);
    b->fp = (double*)take(vec);
  }
  SV_CUDA(cudaMemcpyAsync(b->seeds, seeds.data(), (size_t)b->R * 8, cudaMemcpyHostToDevice, st));
  {
    std::vector<const ProblemDev*> rp(b->R);
    for (int r = 0; r < b->R; ++r) rp[r] = probs[r]->desc_d;
    SV_CUDA(cudaMemcpyAsync(b->rp, rp.data(), (size_t)b->R * 8, cudaMemcpyHostToDevice, st));
  }
  // evaluation scratch for all rows (refine sub-lists per segment and the
  // tensor-core composition staging)
  bool any_comp = false;
  for (const sevo_problem* q : probs) any_comp |= sv_weighted_family(q->family);
  b->any_comp = any_comp;
  b->eval_bytes = sv_eval_scratch_bytes(b->D, any_comp, b->prec, rows);
  SV_CUDA(cudaMalloc(&b->eval_block, b->eval_bytes));
  // the operators hand the evaluation its TF32 operand when every problem has
  // one component (the operand is d = x - o of that component)
  bool single = true;
  for (const sevo_problem* q : probs) single = single && q->ncomp == 1 && !sv_weighted_family(q->family);
  const bool makes_rows = b->alg == SEVO_DE_RAND1 || b->alg == SEVO_DE_CTPB ||
                          b->alg == SEVO_DE_SHADE || b->alg == SEVO_PSO_GBEST ||
                          b->alg == SEVO_PSO_RING;
  b->Ad = nullptr;
  b->Osp = nullptr;
  if (b->prec == SEVO_TF32 && b->D <= 128 && single && makes_rows && !b->small) {
    b->apitch = (b->D + 3) & ~3;
    const size_t osp = (size_t)2 * b->R * b->apitch;
    SV_CUDA(cudaMalloc(&b->Ad, (size_t)rows * b->apitch * 4 + osp * 4));
    b->Osp = b->Ad + (size_t)rows * b->apitch;
    if (!sv_make_operand_map(&b->amap, b->Ad, b->D, rows, b->apitch)) {
      cudaFree(b->Ad);
      b->Ad = nullptr;
      b->Osp = nullptr;
    } else {
      gather_osplit_kernel<<<grid_for((int64_t)osp, 256), 256, 0, st>>>(b->rp, b->R, b->D,
                                                                       b->apitch, b->Osp);
      sv_note_launch();
      SV_CUDA(cudaGetLastError());
    }
  }
  return SEVO_OK;
}

void sv_batch_free(Batch* b) {
  if (b->block) cudaFree(b->block);
  if (b->eval_block) cudaFree(b->eval_block);
  if (b->Ad) cudaFree(b->Ad);
  b->block = b->eval_block = nullptr;
  b->Ad = nullptr;
}

// evaluate every row of `M` (X or U) into `f`: one pass over the batch's
// problem segments (runs sharing a problem)
// evaluate `rpr` rows per run of M (runs in blocks of rpr rows) into f
void sv_batch_segments(const Batch* b, const EvalReq& q, std::vector<TcSegment>* segs) {
  for (size_t s = 0; s + 1 < b->seg_begin.size(); ++s) {
    const int r0 = b->seg_begin[s], r1 = b->seg_begin[s + 1];
    TcSegment t{b->run_prob[r0], (int64_t)r0 * q.rpr, (int64_t)(r1 - r0) * q.rpr};
    t.X = q.M;
    t.out = q.f;
    t.err = b->err;
    t.refined = b->refined;
    t.op = q.op;
    t.amap = q.amap;
    segs->push_back(t);
  }
}

static cudaError_t eval_rows(Batch* b, const double* M, double* f, int rpr = -1,
                             const GenOp* op = nullptr, const CUtensorMap* amap = nullptr) {
  std::vector<TcSegment> segs;
  sv_batch_segments(b, EvalReq{M, f, rpr < 0 ? b->NP : rpr, op, amap}, &segs);
  EvalScratch sc;
  sv_eval_scratch_carve(b->eval_block, b->D, b->any_comp, b->prec, (int64_t)b->R * b->NP, &sc);
  sc.err = b->err;
  sc.refined = b->refined;
  return sv_eval_segments(segs.data(), (int)segs.size(), b->prec, M, b->ld, f, sc, b->stream);
}

cudaError_t sv_ctl_set(Batch* b, unsigned long long gen, int count) {
  const int tk1 = sv_trace_begin(SEVO_TK_CONTROL, b->stream);
  ctl_set_kernel<<<1, 1, 0, b->stream>>>(b->ctl, gen, count);
  sv_trace_end(tk1, b->stream);
  return cudaGetLastError();
}

void sv_ctl_defer(Batch* b, unsigned long long gen, int count) {
  b->pending = CtlSet{gen, count, 1};
}

// the pending control update, for the generation's first kernel
static CtlSet take_ctl(Batch* b) {
  const CtlSet c = b->pending;
  b->pending.on = 0;
  return c;
}

cudaError_t sv_ctl_advance(Batch* b) {
  const int tk2 = sv_trace_begin(SEVO_TK_CONTROL, b->stream);
  ctl_advance_kernel<<<1, 1, 0, b->stream>>>(b->ctl, b->NP, (long long)b->budget, b->per_gen);
  sv_trace_end(tk2, b->stream);
  return cudaGetLastError();
}

cudaError_t sv_batch_init(Batch* b) {
  cudaStream_t st = b->stream;
  const int64_t rows = (int64_t)b->R * b->NP;
  const int T = 256;
  b->rank_fresh = false;
  const int tk3 = sv_trace_begin(SEVO_TK_INIT, st);
  init_pop_kernel<<<grid_for(rows * ((b->D + 1) / 2), T), T, 0, st>>>(b->X, b->seeds, b->R, b->NP,
                                                                     b->D, b->ld, b->lb, b->ub,
                                                                     make_fastdiv((b->D + 1) / 2),
                                                                     make_fastdiv(b->NP));
  sv_trace_end(tk3, st);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const int tk4 = sv_trace_begin(SEVO_TK_CONTROL, st);
  fill_kernel<<<grid_for(b->R, T), T, 0, st>>>(b->best, b->R, INFINITY);
  sv_trace_end(tk4, st);
  if (sv_has_shade(b->alg)) {  // memory: every slot 0.5, write position 0
    const int64_t hm = (int64_t)b->R * SEVO_SHADE_H;
    const int tkm = sv_trace_begin(SEVO_TK_CONTROL, st);
    fill_kernel<<<grid_for(hm, T), T, 0, st>>>(b->MF, hm, 0.5);
    fill_kernel<<<grid_for(hm, T), T, 0, st>>>(b->MCR, hm, 0.5);
    sv_trace_end(tkm, st);
    sv_note_launch();
    if ((e = cudaMemsetAsync(b->mk, 0, (size_t)b->R * 4, st)) != cudaSuccess) return e;
  }
  const int count0 = (int)std::min<int64_t>(b->budget, b->NP);
  if ((e = sv_ctl_set(b, 0ull, count0)) != cudaSuccess) return e;
  if ((e = eval_rows(b, b->X, b->fx)) != cudaSuccess) return e;
  if (!sv_has_pbest(b->alg)) {
    // best-so-far of the initial population (the select kernel's min part
    // with no trials: fu == fx, every row "accepted" onto itself is avoided
    // by using the PSO-style per-run reducer on fx)
    const int tk5 = sv_trace_begin(SEVO_TK_PSO_UPDATE, st);
    pso_update_kernel<<<b->R, SEL_THREADS, (size_t)b->NP * 8, st>>>(b->fx, b->fx, b->action, b->guide, b->best,
                                                    b->ctl, b->NP, 0, 1, 1);
    sv_trace_end(tk5, st);
  } else {
    const size_t m = (size_t)rows * b->ld * 8;
    if ((e = cudaMemcpyAsync(b->P, b->X, m, cudaMemcpyDeviceToDevice, st)) != cudaSuccess) return e;
    const int tk6 = sv_trace_begin(SEVO_TK_CONTROL, st);
    fill_kernel<<<grid_for(rows, T), T, 0, st>>>(b->fp, rows, INFINITY);
    sv_trace_end(tk6, st);
    const int tk7 = sv_trace_begin(SEVO_TK_PSO_UPDATE, st);
    pso_update_kernel<<<b->R, SEL_THREADS, (size_t)b->NP * 8, st>>>(b->fx, b->fp, b->action, b->guide, b->best,
                                                    b->ctl, b->NP, sv_topology(b->alg), 1, 1);
    sv_trace_end(tk7, st);
  }
  return cudaGetLastError();
}

cudaError_t sv_batch_run_small(Batch* b, unsigned long long gen0, int64_t gens) {
  const int64_t chunk = 1 << 16;  // generations per launch
  cudaError_t e = cudaSuccess;
  for (int64_t done = 0; done < gens && e == cudaSuccess;) {
    const int G = (int)std::min<int64_t>(chunk, gens - done);
    const int tk = sv_trace_begin(SEVO_TK_SMALL_RUN, b->stream);
    e = srk_launch(b, G, 1);
    sv_trace_end(tk, b->stream);
    done += G;
    if (e != cudaSuccess) break;
    // the counter and count of the last generation run, as ctl_advance leaves them
    const unsigned long long g = gen0 + (unsigned long long)done;
    const long long c = (long long)b->budget - ((long long)b->NP + (long long)(g - 1) * b->NP);
    e = sv_ctl_set(b, g, (int)(c < 0 ? 0 : (c > b->NP ? b->NP : c)));
  }
  return e;
}

// Whether this batch's operator (DE trial or PSO move) is applied by the
// producer warps of the fused tensor-core evaluation instead of a kernel of
// its own: TF32 / BF16X3 at D <= 128, batched kernels, the policy on.
static bool fusable(const Batch* b) {
  return !b->small && sv_policy_fuse_ops() && b->D <= 128 &&
         (b->prec == SEVO_TF32 || b->prec == SEVO_BF16X3) &&
         (sv_is_de(b->alg) || b->alg == SEVO_PSO_GBEST || b->alg == SEVO_PSO_RING);
}

// the operator descriptor of this generation (the counter as the next
// kernel would take it)
static void fill_op(Batch* b) {
  GenOp& o = b->gop;
  std::memset(&o, 0, sizeof(o));
  o.alg = b->alg;
  o.NP = b->NP;
  o.D = b->D;
  o.ld = b->ld;
  o.pk = b->pbest_k;
  o.F = b->F;
  o.lb = b->lb;
  o.ub = b->ub;
  o.w = b->w;
  o.c1 = b->c1;
  o.c2 = b->c2;
  o.cr_thr = b->cr_thr;
  o.seeds = b->seeds;
  o.ctl = b->ctl;
  o.cs = take_ctl(b);
  if (sv_is_de(b->alg)) {
    o.X = b->X;
    o.U = b->U;
    o.A = (b->alg == SEVO_DE_CTPB) ? b->A : nullptr;
    o.asize = (b->alg == SEVO_DE_CTPB) ? b->asize : nullptr;
    o.order = b->order;
    o.part = b->part;
    o.Fi = b->Fi;
    o.CRi = b->CRi;
    o.kpb = b->kpb;
  } else {
    o.U = b->X;  // moved in place
    o.V = b->V;
    o.P = b->P;
    o.guide = b->guide;
  }
}

// The DE trials of a generation: (SHADE parameters,) p-best ranking, trials
// U from X (fused: everything but the trials themselves).
static cudaError_t de_trials(Batch* b, bool fused = false) {
  cudaStream_t st = b->stream;
  const int64_t rows = (int64_t)b->R * b->NP;
  const int nq = (b->D + 3) >> 2;
  const int T = 256;
  // trial CTAs of 128 threads (about 9K registers) fit on an SM beside a
  // resident fused-evaluation CTA, so one batch's trials run while another
  // batch's evaluation holds the SMs
  const int TT = TRIAL_THREADS;
  const bool shade = sv_has_shade(b->alg);
  if (shade) {
    const int tks = sv_trace_begin(SEVO_TK_DE_TRIAL, st);
    shade_param_kernel<<<grid_for(rows, T), T, 0, st>>>(b->MF, b->MCR, b->seeds, b->ctl,
                                                        take_ctl(b), b->R,
                                                        b->NP, SEVO_SHADE_H, b->Fi, b->CRi,
                                                        b->kpb);
    sv_trace_end(tks, st);
  }
  // current-to-pbest: the previous generation's selection ranked the
  // population it left (de_post_kernel) unless the host changed it since
  const bool ranked = b->rank_fresh && !shade;
  b->rank_fresh = false;
  if ((b->alg == SEVO_DE_CTPB || shade) && !ranked) {
    const int tk_rank = sv_trace_begin(SEVO_TK_DE_RANK, st);
    // counting rank (O(NP^2) per run, parallel over row blocks) for small
    // populations; radix select + sort of the candidates above that
    if (b->NP <= 512) {
      de_rank_kernel<<<dim3(b->R, (b->NP + RANK_ROWS - 1) / RANK_ROWS), RANK_ROWS,
                       (size_t)b->NP * 8, st>>>(b->fx, b->order, b->NP, b->pbest_k);
    } else {
      de_rank_select_kernel<<<b->R, RSEL_THREADS, rsel_smem_bytes(b->NP), st>>>(
          b->fx, b->order, b->NP, pow2_at_least(b->NP), b->pbest_k);
    }
    sv_trace_end(tk_rank, st);
  }
  if (fused) {  // the evaluation's producers make the trials
    fill_op(b);
    return cudaGetLastError();
  }
  if (b->alg == SEVO_DE_CTPB || shade) {
    const int tk8 = sv_trace_begin(SEVO_TK_DE_TRIAL, st);
    if (shade)
      de_trial_kernel<SEVO_DE_SHADE><<<grid_for(rows * nq, TT), TT, 0, st>>>(
          b->X, b->U, nullptr, nullptr, b->order, b->part, b->seeds, b->ctl, take_ctl(b), b->R,
          b->NP, b->D, b->ld, 0.0, 0ull, b->lb, b->ub, b->pbest_k, make_fastdiv(nq), make_fastdiv(b->NP),
          b->Fi, b->CRi, b->kpb, b->Ad, b->apitch, b->Osp);
    else
      de_trial_kernel<SEVO_DE_CTPB><<<grid_for(rows * nq, TT), TT, 0, st>>>(
          b->X, b->U, b->A, b->asize, b->order, b->part, b->seeds, b->ctl, take_ctl(b), b->R,
          b->NP, b->D, b->ld, b->F, b->cr_thr, b->lb, b->ub, b->pbest_k, make_fastdiv(nq),
          make_fastdiv(b->NP), nullptr, nullptr, nullptr, b->Ad, b->apitch, b->Osp);
    sv_trace_end(tk8, st);
  } else {
    const int tk9 = sv_trace_begin(SEVO_TK_DE_TRIAL, st);
    de_trial_kernel<SEVO_DE_RAND1><<<grid_for(rows * nq, TT), TT, 0, st>>>(
        b->X, b->U, nullptr, nullptr, nullptr, b->part, b->seeds, b->ctl, take_ctl(b), b->R,
        b->NP, b->D, b->ld, b->F, b->cr_thr, b->lb, b->ub, 0, make_fastdiv(nq), make_fastdiv(b->NP),
        nullptr, nullptr, nullptr, b->Ad, b->apitch, b->Osp);
    sv_trace_end(tk9, st);
  }
  return cudaGetLastError();
}

// The one-to-one selection of evaluated trials, whose best-so-far counts the
// trials after `count_skip` rows of the generation.  Leaves the per-row
// action for de_apply_kernel / psode_pick_kernel.
static cudaError_t de_select(Batch* b, int count_skip) {
  cudaStream_t st = b->stream;
  const int tk10 = sv_trace_begin(SEVO_TK_DE_SELECT, st);
  de_select_kernel<<<b->R, SEL_THREADS, sel_smem_bytes(b->NP), st>>>(
      b->fx, b->fu, b->asize, b->action, b->best, b->seeds, b->ctl, b->NP,
      b->alg == SEVO_DE_CTPB, b->Fi, b->CRi, b->MF, b->MCR, b->mk, SEVO_SHADE_H, count_skip);
  sv_trace_end(tk10, st);
  return cudaGetLastError();
}

// cluster launch of a per-run post kernel: R clusters of post_cluster(NP) CTAs
template <class... K, class... A>
static cudaError_t post_launch(const Batch* b, size_t smem, void (*kern)(K...), A... args) {
  const int C = post_cluster(b->NP);
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(b->R * C));
  cfg.blockDim = dim3(POST_THREADS);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = b->stream;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = (unsigned)C;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kern, args...);
}

// DE/rand/1 and current-to-pbest selection in one cluster launch per batch;
// current-to-pbest also ranks the new population for the next generation
static bool de_post_applies(const Batch* b) {
  return b->alg == SEVO_DE_RAND1 || b->alg == SEVO_DE_CTPB;
}
static cudaError_t de_post(Batch* b) {
  cudaStream_t st = b->stream;
  const bool arch = b->alg == SEVO_DE_CTPB;
  const int cap = arch ? pow2_at_least(b->pbest_k) : 1;
  const int tk = sv_trace_begin(SEVO_TK_DE_SELECT, st);
  cudaError_t e;
  if (arch)
    e = post_launch(b, post_cand_bytes(cap), de_post_kernel<true>, b->fx, (const double*)b->fu,
                    b->asize, b->action, b->order, b->best, (const uint64_t*)b->seeds,
                    (const GenCtl*)b->ctl, b->NP, b->pbest_k, cap);
  else
    e = post_launch(b, 0, de_post_kernel<false>, b->fx, (const double*)b->fu, (int32_t*)nullptr,
                    b->action, (int32_t*)nullptr, b->best, (const uint64_t*)b->seeds,
                    (const GenCtl*)b->ctl, b->NP, 0, cap);
  sv_trace_end(tk, st);
  b->rank_fresh = arch && e == cudaSuccess;
  return e;
}

static cudaError_t pso_post(Batch* b) {
  cudaStream_t st = b->stream;
  const int tk = sv_trace_begin(SEVO_TK_PSO_UPDATE, st);
  const cudaError_t e = post_launch(b, 0, pso_post_kernel, (const double*)b->fx, b->fp, b->action,
                                    b->guide, b->best, (const GenCtl*)b->ctl, b->NP,
                                    sv_topology(b->alg));
  sv_trace_end(tk, st);
  return e;
}

static cudaError_t de_trials_and_select(Batch* b, int count_skip) {
  cudaError_t e;
  if ((e = de_trials(b)) != cudaSuccess) return e;
  if ((e = eval_rows(b, b->U, b->fu)) != cudaSuccess) return e;
  return de_select(b, count_skip);
}

bool sv_batch_splittable(const Batch* b) { return !b->small && b->alg != SEVO_PSODE; }

cudaError_t sv_batch_pre_eval(Batch* b, EvalReq* q) {
  cudaStream_t st = b->stream;
  const int64_t rows = (int64_t)b->R * b->NP;
  const int T = 256;
  const bool fused = fusable(b);
  if (sv_is_de(b->alg)) {
    *q = EvalReq{b->U, b->fu, b->NP, fused ? &b->gop : nullptr,
                 (b->Ad && !fused) ? &b->amap : nullptr};
    return de_trials(b, fused);
  }
  if (b->alg == SEVO_CSO) {
    const int half = b->NP / 2;
    const int np2 = pow2_at_least(b->NP);
    const int tkp = sv_trace_begin(SEVO_TK_DE_RANK, st);
    cso_pair_kernel<<<b->R, CSO_THREADS, (size_t)np2 * 8, st>>>(b->fx, b->order, b->seeds, b->ctl,
                                                                take_ctl(b), b->NP, np2);
    sv_trace_end(tkp, st);
    const int tkm = sv_trace_begin(SEVO_TK_PSO_MOVE, st);
    cso_mean_kernel<<<dim3((b->D + 127) / 128, std::min(b->R, 65535)), 128, 0, st>>>(
        b->X, b->xbar, b->R, b->NP, b->D, b->ld);
    cso_update_kernel<<<grid_for((int64_t)b->R * half * b->D, T), T, 0, st>>>(
        b->X, b->V, b->U, b->order, b->xbar, b->seeds, b->ctl, b->R, b->NP, b->D, b->ld, b->w,
        b->lb, b->ub, make_fastdiv(b->D), make_fastdiv(half));
    sv_trace_end(tkm, st);
    sv_note_launch();
    *q = EvalReq{b->U, b->fu, half, nullptr};
    return cudaGetLastError();
  }
  if (fused) {  // the evaluation's producers move the particles
    fill_op(b);
    *q = EvalReq{b->X, b->fx, b->NP, &b->gop};
    return cudaGetLastError();
  }
  const int tk12 = sv_trace_begin(SEVO_TK_PSO_MOVE, st);
  pso_move_kernel<<<grid_for(rows * b->D, T), T, 0, st>>>(b->X, b->V, b->P, b->guide, b->seeds,
                                                         b->ctl, take_ctl(b), b->R, b->NP, b->D, b->ld, b->w,
                                                         b->c1, b->c2, b->lb, b->ub,
                                                         make_fastdiv(b->D), make_fastdiv(b->NP),
                                                         b->Ad, b->apitch, b->Osp);
  sv_trace_end(tk12, st);
  *q = EvalReq{b->X, b->fx, b->NP, nullptr, b->Ad ? &b->amap : nullptr};
  return cudaGetLastError();
}

cudaError_t sv_batch_post_eval(Batch* b) {
  cudaStream_t st = b->stream;
  const int64_t rows = (int64_t)b->R * b->NP;
  const int nq = (b->D + 3) >> 2;
  const int T = 256;
  cudaError_t e;
  if (sv_is_de(b->alg)) {
    if ((e = de_post_applies(b) ? de_post(b) : de_select(b, 0)) != cudaSuccess) return e;
    const int tk11 = sv_trace_begin(SEVO_TK_DE_APPLY, st);
    de_apply_kernel<<<grid_for(rows * nq, T), T, 0, st>>>(b->X, b->U, b->A, b->action, b->R, b->NP,
                                                         b->D, b->ld, make_fastdiv(nq),
                                                         make_fastdiv(b->NP));
    sv_trace_end(tk11, st);
    return cudaGetLastError();
  }
  if (b->alg == SEVO_CSO) {
    const int tks = sv_trace_begin(SEVO_TK_PSO_UPDATE, st);
    cso_scatter_kernel<<<b->R, SEL_THREADS, 0, st>>>(b->fx, b->fu, b->order, b->best, b->ctl,
                                                     b->NP);
    sv_trace_end(tks, st);
    return cudaGetLastError();
  }
  if ((e = pso_post(b)) != cudaSuccess) return e;
  const int tk14 = sv_trace_begin(SEVO_TK_PSO_COPY, st);
  pso_copy_kernel<<<grid_for(rows * nq, T), T, 0, st>>>(b->P, b->X, b->action, b->R, b->NP,
                                                       b->D, b->ld, make_fastdiv(nq),
                                                       make_fastdiv(b->NP));
  sv_trace_end(tk14, st);
  return cudaGetLastError();
}

// PSODE (two evaluations per generation): the PSO component's offspring and
// personal bests, then SHADE on the population, then pairwise/3
static cudaError_t psode_generation(Batch* b) {
  cudaStream_t st = b->stream;
  const int64_t rows = (int64_t)b->R * b->NP;
  const int nq = (b->D + 3) >> 2;
  const int T = 256;
  cudaError_t e;
  // PSO component: offspring Y from the population, personal bests, guides
  const int tkm = sv_trace_begin(SEVO_TK_PSO_MOVE, st);
  psode_move_kernel<<<grid_for(rows * b->D, T), T, 0, st>>>(
      b->X, b->V, b->P, b->guide, b->Y, b->seeds, b->ctl, take_ctl(b), b->R, b->NP, b->D, b->ld,
      b->w, b->c1,
      b->c2, b->lb, b->ub, make_fastdiv(b->D), make_fastdiv(b->NP));
  sv_trace_end(tkm, st);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if ((e = eval_rows(b, b->Y, b->fy)) != cudaSuccess) return e;
  const int tku = sv_trace_begin(SEVO_TK_PSO_UPDATE, st);
  pso_update_kernel<<<b->R, SEL_THREADS, (size_t)b->NP * 8, st>>>(
      b->fy, b->fp, b->action, b->guide, b->best, b->ctl, b->NP, 1, 1, 1);
  sv_trace_end(tku, st);
  const int tkc = sv_trace_begin(SEVO_TK_PSO_COPY, st);
  pso_copy_kernel<<<grid_for(rows * nq, T), T, 0, st>>>(b->P, b->Y, b->action, b->R, b->NP,
                                                       b->D, b->ld, make_fastdiv(nq),
                                                       make_fastdiv(b->NP));
  sv_trace_end(tkc, st);
  // SHADE component on the population; its trials count after the NP
  // PSO rows
  if ((e = de_trials_and_select(b, b->NP)) != cudaSuccess) return e;
  // pairwise/3 selection and the DE displacement as the next velocity
  const int tkp = sv_trace_begin(SEVO_TK_DE_APPLY, st);
  psode_pick_kernel<<<grid_for(rows, T), T, 0, st>>>(b->fx, b->fy, b->action, rows);
  psode_combine_kernel<<<grid_for(rows * nq, T), T, 0, st>>>(
      b->X, b->U, b->Y, b->V, b->action, b->R, b->NP, b->D, b->ld, make_fastdiv(nq),
      make_fastdiv(b->NP));
  sv_trace_end(tkp, st);
  sv_note_launch();
  return cudaGetLastError();
}

cudaError_t sv_batch_generation(Batch* b) {
  if (b->small) {
    const int tk = sv_trace_begin(SEVO_TK_SMALL_RUN, b->stream);
    const cudaError_t es = srk_launch(b, 1, 0);
    sv_trace_end(tk, b->stream);
    return es;
  }
  if (b->alg == SEVO_PSODE) return psode_generation(b);
  EvalReq q;
  cudaError_t e;
  if ((e = sv_batch_pre_eval(b, &q)) != cudaSuccess) return e;
  if ((e = eval_rows(b, q.M, q.f, q.rpr, q.op, q.amap)) != cudaSuccess) return e;
  return sv_batch_post_eval(b);
}

// guides only (after the host overwrote pbest fitness)
cudaError_t sv_batch_guides(Batch* b) {
  const int tk15 = sv_trace_begin(SEVO_TK_PSO_UPDATE, b->stream);
  pso_update_kernel<<<b->R, SEL_THREADS, (size_t)b->NP * 8, b->stream>>>(b->fp, b->fp, b->action, b->guide,
                                                         b->best, b->ctl, b->NP,
                                                         sv_topology(b->alg), 0, 0);
  sv_trace_end(tk15, b->stream);
  return cudaGetLastError();
}

int32_t sv_batch_status(Batch* b) {
  uint32_t e = 0;
  SV_CUDA(cudaMemcpyAsync(&e, b->err, 4, cudaMemcpyDeviceToHost, b->stream));
  SV_CUDA(cudaStreamSynchronize(b->stream));
  if (e) {
    SV_CUDA(cudaMemsetAsync(b->err, 0, 4, b->stream));
    if (e & SV_DEVERR_TIMEOUT) return SEVO_ERR_TIMEOUT;
    return SEVO_ERR_CUDA;
  }
  return SEVO_OK;
}
