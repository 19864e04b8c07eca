// post.cuh -- the per-run decisions between one generation's evaluation and
// the row copies that follow it, one launch per batch, one thread-block
// cluster per run: post_cluster(NP) CTAs (a power of two, at most 8) each own
// a contiguous block of at most POST_ROWS rows of the run and exchange their
// partial results (counts, minima, histograms, neighbour values, p-best
// candidates) through distributed shared memory.  One CTA per run would
// leave all but R SMs idle and stretch each run's latency chain.
//
//   de_post_kernel<ARCHIVE>   DE one-to-one selection (f(u) <= f(x)), the
//                             best-so-far, the fitness update, archive slots
//                             (row order; a random slot once the archive is
//                             full; the last row that targets a slot wins),
//                             and with the archive (current-to-pbest) the k
//                             best rows of the new population sorted by
//                             (fitness, index): the next generation's p-best
//                             pool, ranked here instead of in a launch of its
//                             own;
//   pso_post_kernel           PSO personal-best fitness (strict improvement)
//                             and flags, the best-so-far, guides (gbest: the
//                             lowest (key, index); ring: the best of
//                             {i-1, i, i+1}, the lowest index on ties).
//
// The row copies (x <- u and archive <- old x; p <- x) stay in the grid-wide
// kernels that follow.  The decisions equal those of the one-CTA-per-run
// kernels (evo.cu) bit for bit: every rule is applied per row in the same
// order, the cross-CTA sums are integer counts, and the cross-CTA minima do
// not depend on the order in which they are taken.
#pragma once
#include <cooperative_groups.h>

namespace {

namespace cg = cooperative_groups;

constexpr int POST_THREADS = 256;
constexpr int POST_ROWS = 512;  // rows per CTA at most (SV_MAX_NP / 8)
constexpr int POST_MAX_C = 8;

__host__ __device__ inline int post_cluster(int NP) {
  int c = 1;
  while (c * POST_ROWS < NP) c <<= 1;
  return c;
}

// dynamic shared memory: the candidate buffer of the p-best sort (CTA 0):
// cap = (k rounded up to a power of two) keys and indices
__host__ __device__ inline size_t post_cand_bytes(int cap) { return (size_t)cap * 12 + 16; }

// ---------------------------------------------------------------- reductions
// block minimum (dmin_pos) of v; the result in thread 0
__device__ __forceinline__ double post_block_min(double v, double* red) {
  for (int m = 16; m >= 1; m >>= 1) v = dmin_pos(v, __shfl_xor_sync(0xffffffffu, v, m));
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) red[warp] = v;
  __syncthreads();
  double b = red[0];
  if (threadIdx.x == 0)
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) b = dmin_pos(b, red[w]);
  __syncthreads();
  return b;
}

// exclusive row-order prefix of per-row flags fl[0..n) within the block:
// thread t owns rows [t*per, (t+1)*per); returns the count before the
// thread's first row, and the block total in *total
__device__ __forceinline__ int post_block_scan(const unsigned char* fl, int n, int* wsum,
                                               int* total) {
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int per = (n + (int)blockDim.x - 1) / (int)blockDim.x;
  const int j0 = min(n, tid * per), j1 = min(n, j0 + per);
  int cnt = 0;
  for (int i = j0; i < j1; ++i) cnt += fl[i];
  int incl = cnt;
  for (int o = 1; o < 32; o <<= 1) {
    const int v = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += v;
  }
  if (lane == 31) wsum[warp] = incl;
  __syncthreads();
  int woff = 0, tot = 0;
  for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
    if (w < warp) woff += wsum[w];
    tot += wsum[w];
  }
  __syncthreads();
  *total = tot;
  return woff + incl - cnt;
}

// ---------------------------------------------------------------- DE
template <bool ARCHIVE>
__global__ void __launch_bounds__(POST_THREADS)
    de_post_kernel(double* __restrict__ fx, const double* __restrict__ fu,
                   int32_t* __restrict__ asize, int32_t* __restrict__ action,
                   int32_t* __restrict__ order, double* __restrict__ best,
                   const uint64_t* __restrict__ seeds, const GenCtl* __restrict__ ctl, int NP,
                   int k, int cap) {
  extern __shared__ __align__(16) unsigned char pc_sm[];  // CTA 0: p-best candidates
  __shared__ double sf[POST_ROWS], sg[POST_ROWS];
  __shared__ unsigned long long sk[POST_ROWS];
  __shared__ int owner[POST_ROWS], sact[POST_ROWS];
  __shared__ unsigned char sfl[POST_ROWS];
  __shared__ unsigned int hist[2][256];
  __shared__ double red[POST_THREADS / 32];
  __shared__ unsigned long long klo[POST_THREADS / 32], khi[POST_THREADS / 32];
  __shared__ int wsum[POST_THREADS / 32];
  __shared__ double s_min;
  __shared__ unsigned long long s_lo, s_hi, s_prefix;
  __shared__ int s_cnt, s_rem, s_below, s_bin, s_tie, s_ncand;
  cg::cluster_group cl = cg::this_cluster();
  const int C = (int)cl.num_blocks(), c = (int)cl.block_rank();
  const int r = (int)blockIdx.x / C;
  const int L = (NP + C - 1) / C;  // rows per CTA; slot s lives in CTA s / L
  const int i0 = min(NP, c * L), n = min(NP, i0 + L) - i0;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int count = max(0, min(ctl->count, NP));
  const unsigned long long gen = ctl->gen;
  double* f = fx + (int64_t)r * NP + i0;
  const double* g = fu + (int64_t)r * NP + i0;
  for (int i = tid; i < n; i += blockDim.x) {
    const double a = f[i], b = g[i];
    sf[i] = a;
    sg[i] = b;
    sfl[i] = b <= a;  // accepted
  }
  for (int i = tid; i < L; i += blockDim.x) owner[i] = -1;
  if (tid == 0) s_ncand = 0;
  __syncthreads();
  // best-so-far over the trials that count toward the budget
  double m = INFINITY;
  for (int i = tid; i < n && i0 + i < count; i += blockDim.x) m = dmin_pos(m, sg[i]);
  m = post_block_min(m, red);
  int ctot;
  const int kpre = post_block_scan(sfl, n, wsum, &ctot);
  if (tid == 0) {
    s_min = m;
    s_cnt = ctot;
  }
  cl.sync();  // every CTA's accepted count and minimum; owner tables cleared
  int off = 0, tot = 0;
  for (int q = 0; q < C; ++q) {
    const int v = *cl.map_shared_rank(&s_cnt, q);
    if (q < c) off += v;
    tot += v;
  }
  if (c == 0 && tid == 0) {
    double b = best[r];
    for (int q = 0; q < C; ++q) b = dmin_pos(b, *cl.map_shared_rank(&s_min, q));
    best[r] = b;
  }
  // actions in row order: the accepted row of global accepted index kk
  // targets archive slot as0 + kk while the archive has room, else a random
  // slot; every targeted slot keeps its last row
  const int as0 = ARCHIVE ? asize[r] : 0;
  {
    const int per = (n + (int)blockDim.x - 1) / (int)blockDim.x;
    const int j0 = min(n, tid * per), j1 = min(n, j0 + per);
    int kk = off + kpre;
    for (int i = j0; i < j1; ++i) {
      int a = -2;
      if (sfl[i]) {
        a = -1;
        if (ARCHIVE) {
          int slot;
          if (as0 + kk < NP) {
            slot = as0 + kk;
          } else {
            const uint4 w = sv_draw(seeds[r], 0u, (uint32_t)(i0 + i), (uint32_t)gen, SV_P_ARCH);
            slot = (int)sv_below(w.x, (uint32_t)NP);
          }
          atomicMax(cl.map_shared_rank(&owner[slot % L], slot / L), i0 + i);
          a = slot;
        }
        ++kk;
      }
      sact[i] = a;
    }
  }
  cl.sync();  // slot owners final
  int32_t* act = action + (int64_t)r * NP + i0;
  for (int i = tid; i < n; i += blockDim.x) {
    int a = sact[i];
    if (ARCHIVE && a >= 0 && *cl.map_shared_rank(&owner[a % L], a / L) != i0 + i) a = -1;
    act[i] = a;
    if (a != -2) {
      f[i] = sg[i];
      sf[i] = sg[i];
    }
  }
  if (ARCHIVE && c == 0 && tid == 0) asize[r] = min(NP, as0 + tot);
  if (!ARCHIVE) return;  // no later access to another CTA's shared memory

  // ---- the k best of the new population, sorted by (fitness, index)
  // Radix select over the cluster's keys (8-bit digits, MSB first, starting
  // at the highest bit where the smallest and largest keys differ) until the
  // keys up to the selected digit's bin fit the sort (at most cap of them);
  // if they never do (a run of keys equal to the k-th), the candidates are
  // the keys below the k-th one plus the first ties in row order.
  __syncthreads();
  unsigned long long lo = ~0ull, hi = 0ull;
  for (int i = tid; i < n; i += blockDim.x) {
    const unsigned long long v = (unsigned long long)fkey(sf[i]) ^ 0x8000000000000000ull;
    sk[i] = v;
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
    klo[warp] = lo;
    khi[warp] = hi;
  }
  __syncthreads();
  if (tid == 0) {
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) {
      lo = klo[w] < lo ? klo[w] : lo;
      hi = khi[w] > hi ? khi[w] : hi;
    }
    s_lo = lo;
    s_hi = hi;
  }
  cl.sync();  // every CTA's key range
  lo = ~0ull;
  hi = 0ull;
  for (int q = 0; q < C; ++q) {
    const unsigned long long a = *cl.map_shared_rank(&s_lo, q), b = *cl.map_shared_rank(&s_hi, q);
    lo = a < lo ? a : lo;
    hi = b > hi ? b : hi;
  }
  unsigned long long thresh = lo;
  int rem = k;
  bool exact = NP > cap;  // all keys equal: ties only
  if (lo != hi) {
    int shift = ((63 - __clzll((long long)(lo ^ hi))) >> 3) << 3;
    unsigned long long pmask = shift == 56 ? 0ull : ~((1ull << (shift + 8)) - 1ull);
    unsigned long long prefix = lo & pmask;
    int below = 0;  // keys below the prefix's range: all among the k best
    for (int pass = 0;; ++pass) {
      unsigned int* h = hist[pass & 1];
      for (int b = tid; b < 256; b += blockDim.x) h[b] = 0u;
      __syncthreads();
      for (int i = tid; i < n; i += blockDim.x) {
        const unsigned long long v = sk[i];
        if ((v & pmask) == prefix) atomicAdd(&h[(unsigned)((v >> shift) & 255u)], 1u);
      }
      cl.sync();  // every CTA's histogram of this pass
      if (tid < 32) {  // lane owns bins 8*lane .. 8*lane+7, summed over the cluster
        unsigned cb[8], sum = 0u;
#pragma unroll
        for (int q = 0; q < 8; ++q) cb[q] = 0u;
        for (int t = 0; t < C; ++t) {
          const unsigned int* ht = cl.map_shared_rank(h, t);
#pragma unroll
          for (int q = 0; q < 8; ++q) cb[q] += ht[lane * 8 + q];
        }
#pragma unroll
        for (int q = 0; q < 8; ++q) sum += cb[q];
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
            if (acc + cb[q] >= (unsigned)rem) {
              b = lane * 8 + q;
              break;
            }
            acc += cb[q];
          }
          s_prefix = prefix | ((unsigned long long)b << shift);
          s_rem = rem - (int)acc;
          s_below = below + (int)acc;
          s_bin = (int)cb[b - lane * 8];
        }
      }
      __syncthreads();
      prefix = s_prefix;
      rem = s_rem;
      below = s_below;
      const int cnt = s_bin;
      if (below + cnt <= cap) {
        thresh = prefix | (shift == 0 ? 0ull : (1ull << shift) - 1ull);
        exact = false;
        break;
      }
      if (shift == 0) {
        thresh = prefix;
        exact = true;
        break;
      }
      pmask |= 255ull << shift;
      shift -= 8;
    }
  }
  // gather the candidates into CTA 0's buffer (their order there does not
  // matter: the sort orders them by (key, index))
  unsigned long long* ck0 = cl.map_shared_rank(reinterpret_cast<unsigned long long*>(pc_sm), 0);
  int* ci0 = cl.map_shared_rank(reinterpret_cast<int*>(pc_sm + (size_t)cap * 8), 0);
  int* nc0 = cl.map_shared_rank(&s_ncand, 0);
  if (!exact) {
    for (int i = tid; i < n; i += blockDim.x) {
      if (sk[i] <= thresh) {
        const int s = atomicAdd(nc0, 1);
        ck0[s] = sk[i];
        ci0[s] = i0 + i;
      }
    }
  } else {
    // ties with the k-th key: the first rem of them in row order
    for (int i = tid; i < n; i += blockDim.x) sfl[i] = sk[i] == thresh;
    __syncthreads();
    int ttot;
    const int tpre = post_block_scan(sfl, n, wsum, &ttot);
    if (tid == 0) s_tie = ttot;
    cl.sync();  // every CTA's tie count
    int t = tpre;
    for (int q = 0; q < c; ++q) t += *cl.map_shared_rank(&s_tie, q);
    const int per = (n + (int)blockDim.x - 1) / (int)blockDim.x;
    const int j0 = min(n, tid * per), j1 = min(n, j0 + per);
    for (int i = j0; i < j1; ++i) {
      const unsigned long long v = sk[i];
      bool take = v < thresh;
      if (v == thresh) take = t++ < rem;
      if (take) {
        const int s = atomicAdd(nc0, 1);
        ck0[s] = v;
        ci0[s] = i0 + i;
      }
    }
  }
  cl.sync();  // every candidate is in CTA 0; no shared memory is read remotely after this
  if (c != 0) return;
  unsigned long long* ck = reinterpret_cast<unsigned long long*>(pc_sm);
  int* ci = reinterpret_cast<int*>(pc_sm + (size_t)cap * 8);
  const int nc = s_ncand;  // k <= nc <= cap
  const int mm = pow2_at_least(nc);
  for (int i = nc + tid; i < mm; i += blockDim.x) {
    ck[i] = ~0ull;
    ci[i] = 0x7FFFFFFF;
  }
  __syncthreads();
  for (int size = 2; size <= mm; size <<= 1) {
    for (int stride = size >> 1; stride > 0; stride >>= 1) {
      for (int t = tid; t < mm / 2; t += blockDim.x) {
        const int a = 2 * t - (t & (stride - 1)), b = a + stride;
        const bool up = (a & size) == 0;
        const unsigned long long ka = ck[a], kb = ck[b];
        const int ia = ci[a], ib = ci[b];
        const bool a_gt_b = (ka > kb) || (ka == kb && ia > ib);
        if (a_gt_b == up) {
          ck[a] = kb;
          ck[b] = ka;
          ci[a] = ib;
          ci[b] = ia;
        }
      }
      __syncthreads();
    }
  }
  for (int q = tid; q < k; q += blockDim.x) order[(int64_t)r * NP + q] = ci[q];
}

// ---------------------------------------------------------------- PSO
__global__ void __launch_bounds__(POST_THREADS)
    pso_post_kernel(const double* __restrict__ fx, double* __restrict__ fp,
                    int32_t* __restrict__ flag, int32_t* __restrict__ guide,
                    double* __restrict__ best, const GenCtl* __restrict__ ctl, int NP,
                    int topology) {
  __shared__ double sp[POST_ROWS];  // personal-best fitness of this CTA's rows
  __shared__ double red[POST_THREADS / 32];
  __shared__ long long kbw[POST_THREADS / 32];
  __shared__ int ibw[POST_THREADS / 32];
  __shared__ double s_min;
  __shared__ long long s_kb;
  __shared__ int s_ib;
  cg::cluster_group cl = cg::this_cluster();
  const int C = (int)cl.num_blocks(), c = (int)cl.block_rank();
  const int r = (int)blockIdx.x / C;
  const int L = (NP + C - 1) / C;
  const int i0 = min(NP, c * L), n = min(NP, i0 + L) - i0;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int count = max(0, min(ctl->count, NP));
  const double* f = fx + (int64_t)r * NP + i0;
  double* p = fp + (int64_t)r * NP + i0;
  int32_t* fl = flag + (int64_t)r * NP + i0;
  int32_t* gd = guide + (int64_t)r * NP + i0;
  double m = INFINITY;
  long long kb = 0x7FFFFFFFFFFFFFFFll;
  int ib = 0x7FFFFFFF;
  for (int i = tid; i < n; i += blockDim.x) {
    const double fi = f[i];
    double pi = p[i];
    const bool up = fi < pi;  // strict improvement
    fl[i] = up;
    if (up) {
      p[i] = fi;
      pi = fi;
    }
    sp[i] = pi;
    if (i0 + i < count) m = dmin_pos(m, fi);
    const long long kk = fkey(pi);
    if (kk < kb || (kk == kb && i0 + i < ib)) {
      kb = kk;
      ib = i0 + i;
    }
  }
  m = post_block_min(m, red);
  for (int o = 16; o >= 1; o >>= 1) {
    const long long k2 = __shfl_xor_sync(0xffffffffu, kb, o);
    const int i2 = __shfl_xor_sync(0xffffffffu, ib, o);
    if (k2 < kb || (k2 == kb && i2 < ib)) {
      kb = k2;
      ib = i2;
    }
  }
  if (lane == 0) {
    kbw[warp] = kb;
    ibw[warp] = ib;
  }
  __syncthreads();
  if (tid == 0) {
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w)
      if (kbw[w] < kb || (kbw[w] == kb && ibw[w] < ib)) {
        kb = kbw[w];
        ib = ibw[w];
      }
    s_kb = kb;
    s_ib = ib;
    s_min = m;
  }
  cl.sync();  // every CTA's personal bests, minimum and best (key, index)
  if (c == 0 && tid == 0) {
    double b = best[r];
    for (int q = 0; q < C; ++q) b = dmin_pos(b, *cl.map_shared_rank(&s_min, q));
    best[r] = b;
  }
  if (topology == 0) {
    kb = 0x7FFFFFFFFFFFFFFFll;
    ib = 0x7FFFFFFF;
    for (int q = 0; q < C; ++q) {
      const long long k2 = *cl.map_shared_rank(&s_kb, q);
      const int i2 = *cl.map_shared_rank(&s_ib, q);
      if (k2 < kb || (k2 == kb && i2 < ib)) {
        kb = k2;
        ib = i2;
      }
    }
    for (int i = tid; i < n; i += blockDim.x) gd[i] = ib;
  } else {
    for (int i = tid; i < n; i += blockDim.x) {
      const int gi = i0 + i;
      int nb[3] = {(gi + NP - 1) % NP, gi, (gi + 1) % NP};
      // ascending indices, then strict improvement keeps the lowest index
      for (int a = 0; a < 2; ++a)
        for (int t = 0; t < 2 - a; ++t)
          if (nb[t] > nb[t + 1]) {
            const int s = nb[t];
            nb[t] = nb[t + 1];
            nb[t + 1] = s;
          }
      double v[3];
#pragma unroll
      for (int t = 0; t < 3; ++t)
        v[t] = (nb[t] >= i0 && nb[t] < i0 + n) ? sp[nb[t] - i0]
                                               : *cl.map_shared_rank(&sp[nb[t] % L], nb[t] / L);
      int b = 0;
      for (int t = 1; t < 3; ++t)
        if (v[t] < v[b]) b = t;
      gd[i] = nb[b];
    }
  }
  cl.sync();  // no CTA leaves while another may still read its shared memory
}

}  // namespace
