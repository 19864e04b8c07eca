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

// dynamic shared memory: every CTA's copy of the p-best candidates, cap =
// (k rounded up to a power of two) keys and indices
__host__ __device__ inline size_t post_cand_bytes(int cap) { return (size_t)cap * 12 + 16; }

// Cross-CTA exchange is pushed, not pulled: before a cluster barrier each CTA
// writes (or reduces with a remote atomic) its partial results into the
// shared memory of every CTA of the cluster, so that after the barrier every
// CTA reads them locally.  Remote stores do not stall the writer; a remote
// load costs a round trip to another SM.
//
// A CTA's shared memory may be accessed remotely only once the CTA runs and
// has initialised what others write into: each CTA arrives at a cluster
// barrier (release) right after its initialisation and waits on it (acquire)
// just before its first remote access, so the wait usually costs nothing.
__device__ __forceinline__ void cluster_arrive() {
  asm volatile("barrier.cluster.arrive.release.aligned;" ::: "memory");
}
__device__ __forceinline__ void cluster_wait() {
  asm volatile("barrier.cluster.wait.acquire.aligned;" ::: "memory");
}

// ---------------------------------------------------------------- reductions
// block minimum (dmin_pos) of v, returned to every thread
__device__ __forceinline__ double post_block_min(double v, double* red) {
  for (int m = 16; m >= 1; m >>= 1) v = dmin_pos(v, __shfl_xor_sync(0xffffffffu, v, m));
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) red[warp] = v;
  __syncthreads();
  double b = red[0];
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
  constexpr int HB = ARCHIVE ? 256 : 1;  // histogram bins (current-to-pbest only)
  extern __shared__ __align__(16) unsigned char pc_sm[];  // the p-best candidates
  __shared__ double sf[POST_ROWS];
  __shared__ union {
    double g[POST_ROWS];              // trial fitness (selection)
    unsigned long long k[POST_ROWS];  // keys of the new fitness (ranking)
  } su;
  __shared__ int owner[POST_ROWS], sact[POST_ROWS];
  __shared__ unsigned char sfl[POST_ROWS];
  __shared__ unsigned int hloc[HB], htot[2][HB];  // this CTA's / the cluster's histogram
  __shared__ double red[POST_THREADS / 32];
  __shared__ unsigned long long klo[POST_THREADS / 32], khi[POST_THREADS / 32];
  __shared__ int wsum[POST_THREADS / 32];
  // pushed by CTA q into entry q of every CTA
  __shared__ int x_cnt[POST_MAX_C], x_tie[POST_MAX_C];
  __shared__ double x_min[POST_MAX_C];
  __shared__ unsigned long long x_lo[POST_MAX_C], x_hi[POST_MAX_C];
  __shared__ int x_nc;     // candidates in the buffer (max over CTAs of base + count)
  __shared__ int s_alloc;  // CTA 0: buffer allocation counter
  __shared__ unsigned long long s_prefix;
  __shared__ int s_rem, s_below, s_bin, s_base;
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
    su.g[i] = b;
    sfl[i] = b <= a;  // accepted
  }
  for (int i = tid; i < L; i += blockDim.x) owner[i] = -1;
  if (ARCHIVE)
    for (int b = tid; b < HB; b += blockDim.x) htot[0][b] = htot[1][b] = 0u;
  if (tid == 0) {
    x_nc = 0;
    s_alloc = 0;
  }
  __syncthreads();
  cluster_arrive();  // initialised: the tables may be written remotely
  // best-so-far over the trials that count toward the budget
  double m = INFINITY;
  for (int i = tid; i < n && i0 + i < count; i += blockDim.x) m = dmin_pos(m, su.g[i]);
  m = post_block_min(m, red);
  int ctot;
  const int kpre = post_block_scan(sfl, n, wsum, &ctot);
  cluster_wait();  // every CTA initialised
  if (tid < C) {
    *cl.map_shared_rank(&x_cnt[c], tid) = ctot;
    *cl.map_shared_rank(&x_min[c], tid) = m;
  }
  cl.sync();  // every CTA's accepted count and minimum, here
  int off = 0, tot = 0;
  for (int q = 0; q < C; ++q) {
    if (q < c) off += x_cnt[q];
    tot += x_cnt[q];
  }
  if (c == 0 && tid == 0) {
    double b = best[r];
    for (int q = 0; q < C; ++q) b = dmin_pos(b, x_min[q]);
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
  if (ARCHIVE)
    cl.sync();  // slot owners final (and this CTA's actions)
  else
    __syncthreads();  // this CTA's actions (written in row chunks, read strided)
  int32_t* act = action + (int64_t)r * NP + i0;
  for (int i = tid; i < n; i += blockDim.x) {
    int a = sact[i];
    if (ARCHIVE && a >= 0 && *cl.map_shared_rank(&owner[a % L], a / L) != i0 + i) a = -1;
    act[i] = a;
    if (a != -2) {
      f[i] = su.g[i];
      sf[i] = su.g[i];
    }
  }
  if (ARCHIVE && c == 0 && tid == 0) asize[r] = min(NP, as0 + tot);
  if (!ARCHIVE) return;  // nothing of another CTA is read after the last barrier

  // ---- the k best of the new population, sorted by (fitness, index)
  // Radix select over the cluster's keys (8-bit digits, MSB first, starting
  // at the highest bit where the smallest and largest keys differ) until the
  // keys up to the selected digit's bin fit the candidate buffer (at most cap
  // of them); if they never do (a run of keys equal to the k-th), the
  // candidates are the keys below the k-th one plus the first ties in row
  // order.  Every CTA then ranks a share of the candidates by counting.
  __syncthreads();
  unsigned long long lo = ~0ull, hi = 0ull;
  for (int i = tid; i < n; i += blockDim.x) {
    const unsigned long long v = (unsigned long long)fkey(sf[i]) ^ 0x8000000000000000ull;
    su.k[i] = v;
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
  for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
    lo = klo[w] < lo ? klo[w] : lo;
    hi = khi[w] > hi ? khi[w] : hi;
  }
  if (tid < C) {
    *cl.map_shared_rank(&x_lo[c], tid) = lo;
    *cl.map_shared_rank(&x_hi[c], tid) = hi;
  }
  cl.sync();  // every CTA's key range, here
  for (int q = 0; q < C; ++q) {
    lo = x_lo[q] < lo ? x_lo[q] : lo;
    hi = x_hi[q] > hi ? x_hi[q] : hi;
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
      unsigned int* ht = htot[pass & 1];
      for (int b = tid; b < 256; b += blockDim.x) hloc[b] = 0u;
      __syncthreads();
      for (int i = tid; i < n; i += blockDim.x) {
        const unsigned long long v = su.k[i];
        if ((v & pmask) == prefix) atomicAdd(&hloc[(unsigned)((v >> shift) & 255u)], 1u);
      }
      __syncthreads();
      // add this CTA's bins into every CTA's cluster histogram of this pass
      for (int b = tid; b < 256; b += blockDim.x) {
        const unsigned v = hloc[b];
        if (v)
          for (int q = 0; q < C; ++q) atomicAdd(cl.map_shared_rank(&ht[b], q), v);
      }
      cl.sync();  // the cluster histogram of this pass, here
      if (tid < 32) {  // lane owns bins 8*lane .. 8*lane+7
        unsigned cb[8], sum = 0u;
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          cb[q] = ht[lane * 8 + q];
          sum += cb[q];
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
      // this pass's cluster histogram is read: clear it for pass + 2 (no CTA
      // adds into it before every CTA has passed the next pass's barrier)
      for (int b = tid; b < 256; b += blockDim.x) ht[b] = 0u;
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
  // the candidates of this CTA, flagged
  if (!exact) {
    for (int i = tid; i < n; i += blockDim.x) sfl[i] = su.k[i] <= thresh;
  } else {
    // ties with the k-th key: the first rem of them in row order
    for (int i = tid; i < n; i += blockDim.x) sfl[i] = su.k[i] == thresh;
    __syncthreads();
    int ttot;
    const int tpre = post_block_scan(sfl, n, wsum, &ttot);
    if (tid < C) *cl.map_shared_rank(&x_tie[c], tid) = ttot;
    cl.sync();  // every CTA's tie count, here
    int t = tpre;
    for (int q = 0; q < c; ++q) t += x_tie[q];
    const int per = (n + (int)blockDim.x - 1) / (int)blockDim.x;
    const int j0 = min(n, tid * per), j1 = min(n, j0 + per);
    for (int i = j0; i < j1; ++i) {
      const unsigned long long v = su.k[i];
      bool take = v < thresh;
      if (v == thresh) take = t++ < rem;
      sfl[i] = take;
    }
  }
  __syncthreads();
  // one remote atomic reserves this CTA's block of the buffer; the
  // candidates are written into every CTA's copy of it
  unsigned long long* ck = reinterpret_cast<unsigned long long*>(pc_sm);
  int* ci = reinterpret_cast<int*>(pc_sm + (size_t)cap * 8);
  {
    int ntake;
    const int pre = post_block_scan(sfl, n, wsum, &ntake);
    if (tid == 0) {
      const int base = ntake > 0 ? atomicAdd(cl.map_shared_rank(&s_alloc, 0), ntake) : 0;
      s_base = base;
      for (int q = 0; q < C; ++q) atomicMax(cl.map_shared_rank(&x_nc, q), base + ntake);
    }
    __syncthreads();
    int slot = s_base + pre;
    const int per = (n + (int)blockDim.x - 1) / (int)blockDim.x;
    const int j0 = min(n, tid * per), j1 = min(n, j0 + per);
    for (int i = j0; i < j1; ++i) {
      if (!sfl[i] || slot >= cap) continue;  // (never past cap: the select bounds the count)
      for (int q = 0; q < C; ++q) {
        *cl.map_shared_rank(&ck[slot], q) = su.k[i];
        *cl.map_shared_rank(&ci[slot], q) = i0 + i;
      }
      ++slot;
    }
  }
  cl.sync();  // every candidate in every CTA's buffer; no remote access follows
  // rank by counting: candidate j's position among all candidates by (key,
  // index).  CTA c takes candidates c, c + C, c + 2C, ...; eight lanes share
  // one candidate, four candidates per warp (the loop bound is per warp, so
  // that every lane reaches the shuffles)
  const int nc = min(x_nc, cap);  // k <= nc <= cap
  const int gl = lane & 7;
  const int nw = (int)(blockDim.x >> 5);
  for (int mb = warp * 4; c + mb * C < nc; mb += nw * 4) {
    const int j = c + (mb + (lane >> 3)) * C;
    const bool valid = j < nc;
    const unsigned long long kj = valid ? ck[j] : 0ull;
    const int ij = valid ? ci[j] : 0;
    int lower = 0;
    if (valid)
      for (int t = gl; t < nc; t += 8) {
        const unsigned long long kt = ck[t];
        lower += (kt < kj) || (kt == kj && ci[t] < ij);
      }
    lower += __shfl_xor_sync(0xffffffffu, lower, 1);
    lower += __shfl_xor_sync(0xffffffffu, lower, 2);
    lower += __shfl_xor_sync(0xffffffffu, lower, 4);
    if (valid && gl == 0 && lower < k) order[(int64_t)r * NP + lower] = ij;
  }
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
  // pushed by CTA q into entry q of every CTA
  __shared__ double x_min[POST_MAX_C];
  __shared__ long long x_kb[POST_MAX_C];
  __shared__ int x_ib[POST_MAX_C];
  // ring: personal bests of the rows just before and just after this CTA's
  // rows (cyclically), pushed by the neighbouring CTAs
  __shared__ double x_edge[2];
  cluster_arrive();  // nothing to initialise: every pushed entry is overwritten
  cg::cluster_group cl = cg::this_cluster();
  const int C = (int)cl.num_blocks(), c = (int)cl.block_rank();
  const int r = (int)blockIdx.x / C;
  const int L = (NP + C - 1) / C;
  const int i0 = min(NP, c * L), n = min(NP, i0 + L) - i0;  // n >= 1
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
  cluster_wait();  // every CTA runs
  if (tid < C) {
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w)
      if (kbw[w] < kb || (kbw[w] == kb && ibw[w] < ib)) {
        kb = kbw[w];
        ib = ibw[w];
      }
    *cl.map_shared_rank(&x_kb[c], tid) = kb;
    *cl.map_shared_rank(&x_ib[c], tid) = ib;
    *cl.map_shared_rank(&x_min[c], tid) = m;
    if (tid == 0) {
      *cl.map_shared_rank(&x_edge[1], (c + C - 1) % C) = sp[0];  // row i0: after CTA c-1's rows
      *cl.map_shared_rank(&x_edge[0], (c + 1) % C) = sp[n - 1];  // row i0+n-1: before CTA c+1's
    }
  }
  cl.sync();  // every pushed entry, here; no remote access follows
  if (c == 0 && tid == 0) {
    double b = best[r];
    for (int q = 0; q < C; ++q) b = dmin_pos(b, x_min[q]);
    best[r] = b;
  }
  if (topology == 0) {
    kb = 0x7FFFFFFFFFFFFFFFll;
    ib = 0x7FFFFFFF;
    for (int q = 0; q < C; ++q)
      if (x_kb[q] < kb || (x_kb[q] == kb && x_ib[q] < ib)) {
        kb = x_kb[q];
        ib = x_ib[q];
      }
    for (int i = tid; i < n; i += blockDim.x) gd[i] = ib;
  } else {
    const int before = (i0 + NP - 1) % NP;  // the other row outside is (i0 + n) % NP
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
      for (int t = 0; t < 3; ++t) {
        const int j = nb[t];
        v[t] = (j >= i0 && j < i0 + n) ? sp[j - i0] : (j == before ? x_edge[0] : x_edge[1]);
      }
      int b = 0;
      for (int t = 1; t < 3; ++t)
        if (v[t] < v[b]) b = t;
      gd[i] = nb[b];
    }
  }
}

}  // namespace
