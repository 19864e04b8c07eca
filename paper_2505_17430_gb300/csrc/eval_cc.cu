// eval_cc.cu -- CUDA-core evaluation kernels.
//
//   T = double : the plain FP64 GPU path (DFMA rotation, FP64 bodies); also
//                the FP64 refinement of rows listed by a mixed pass.
//   T = float  : FP32 CUDA-core rotation with FP32 bodies (the small-D mixed
//                path); rows below the refinement threshold are listed.
//
// Work split: a CTA of 256 threads takes a tile of 8 rows.  For each chunk of
// 256 outputs i, thread i accumulates z_i for the 8 rows over 256-wide input
// chunks of d = x - o staged in shared memory (M read as M^T, coalesced).
// Warp r then reduces the chunk's body terms of row r group by group in a
// fixed shuffle order (deterministic), carrying the Rosenbrock pair across
// chunk borders.
#include "bodies.cuh"
#include <atomic>

#include "kernels.cuh"

namespace {

constexpr int TR = 8;    // rows per tile (one warp each in the epilogue)
constexpr int NT = 256;  // threads
constexpr int CH = 256;  // chunk width (outputs and inputs)

template <typename T>
struct AccT;
template <>
struct AccT<double> {
  using type = Acc64;
};
template <>
struct AccT<float> {
  using type = Acc32;
};

__device__ __forceinline__ void acc_init(int body, Acc64& a) { acc64_init(body, a); }
__device__ __forceinline__ void acc_init(int, Acc32& a) { acc32_init(a); }

__device__ __forceinline__ void term(int body, double z, double aux, bool hn, double zn,
                                     const ProblemDev& P, Acc64& a) {
  term64(body, z, aux, hn, zn, P, a);
}
__device__ __forceinline__ void term(int body, float z, float aux, bool hn, float zn,
                                     const ProblemDev& P, Acc32& a) {
  term32(body, z, aux, hn, zn, P, a);
}

__device__ __forceinline__ void combine(int body, Acc64& a, const Acc64& b) {
  a.a0 += b.a0;
  if (slot1_is_product64(body))
    a.a1 *= b.a1;
  else
    a.a1 += b.a1;
  a.a2 += b.a2;
}
__device__ __forceinline__ void combine(int, Acc32& a, const Acc32& b) {
  a.a0 += b.a0;
  a.a1 += b.a1;
  a.a2 += b.a2;
}

template <typename A>
__device__ __forceinline__ void warp_reduce(int body, A& a) {
#pragma unroll
  for (int m = 16; m >= 1; m >>= 1) {
    A b;
    b.a0 = __shfl_xor_sync(0xffffffffu, a.a0, m);
    b.a1 = __shfl_xor_sync(0xffffffffu, a.a1, m);
    b.a2 = __shfl_xor_sync(0xffffffffu, a.a2, m);
    combine(body, a, b);
  }
}

__device__ __forceinline__ double finalize(int body, const Acc64& a, int n) {
  return finalize64(body, a, n);
}
__device__ __forceinline__ double finalize(int body, const Acc32& a, int n) {
  return (double)finalize32(body, a, n);
}

template <typename T>
__device__ __forceinline__ const T* mt_ptr(const ProblemDev& P, int c);
template <>
__device__ __forceinline__ const double* mt_ptr<double>(const ProblemDev& P, int c) {
  return P.MT64[c];
}
template <>
__device__ __forceinline__ const float* mt_ptr<float>(const ProblemDev& P, int c) {
  return P.MT32[c];
}
__device__ __forceinline__ double aux_of(const ProblemDev& P, int c, int i, double) {
  return P.aux64[c][i];
}
__device__ __forceinline__ float aux_of(const ProblemDev& P, int c, int i, float) {
  return P.aux32[c][i];
}

// LIST = false: rows row0 .. row0 + N - 1 of one problem (Pg).
// LIST = true : the rows listed per segment (RT.P[s], list[RT.list_off[s]
//               + k] for k < counts[s]); a tile never straddles segments.
template <typename T, bool LIST>
__global__ void __launch_bounds__(NT) eval_cc_kernel(const ProblemDev* __restrict__ Pg,
                                                     const __grid_constant__ RefineTable RT,
                                                     const double* __restrict__ X, int64_t ld,
                                                     int64_t row0, int64_t N,
                                                     const int32_t* __restrict__ list,
                                                     const int32_t* __restrict__ counts,
                                                     double* __restrict__ out, EvalAux aux) {
  using Acc = typename AccT<T>::type;
  __shared__ ProblemDev P;
  __shared__ T dS[TR][CH];
  __shared__ T zS[TR][CH + 1];
  __shared__ Acc tot[TR][SV_MAXG];
  __shared__ T prevz[TR];
  __shared__ int64_t rowS[TR];
  __shared__ double gS[TR][SV_MAXC];
  __shared__ double sS[TR][SV_MAXC];
  __shared__ int64_t cumS[SV_MAX_SEG + 1];
  __shared__ int curSeg;

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  // load problem descriptor P (and the Schwefel constant with the device sin,
  // so that the term is exactly 0 at z = 0)
  auto load_problem = [&](const ProblemDev* src_p) {
    __syncthreads();
    const int* src = (const int*)src_p;
    int* dst = (int*)&P;
    for (int k = tid; k < (int)(sizeof(ProblemDev) / 4); k += NT) dst[k] = src[k];
    __syncthreads();
    if (tid == 0) P.sch_c = __dmul_rn(P.sch_s, sin(sqrt(P.sch_s)));
    __syncthreads();
  };
  int64_t total_tiles;
  if (LIST) {
    if (tid == 0) {
      cumS[0] = 0;
      for (int q = 0; q < RT.nseg; ++q) cumS[q + 1] = cumS[q] + (counts[q] + TR - 1) / TR;
      curSeg = -1;
      if (blockIdx.x == 0)
        for (int q = 0; q < RT.nseg; ++q)
          if (RT.total[q] && counts[q]) atomicAdd(RT.total[q], (unsigned long long)counts[q]);
    }
    __syncthreads();
    total_tiles = cumS[RT.nseg];
  } else {
    load_problem(Pg);
    total_tiles = (N + TR - 1) / TR;
  }

  for (int64_t tile = blockIdx.x; tile < total_tiles; tile += gridDim.x) {
    int seg = 0;
    if (LIST) {
      while (seg + 1 < RT.nseg && tile >= cumS[seg + 1]) ++seg;
      if (seg != curSeg) {
        load_problem(RT.P[seg]);
        if (tid == 0) curSeg = seg;
      }
    }
    const int D = P.D;
    const int nchunks = (D + CH - 1) / CH;
    // a listed segment may name its own rows and results
    const double* __restrict__ Xs = (LIST && RT.X[seg]) ? RT.X[seg] : X;
    double* __restrict__ outs = (LIST && RT.out[seg]) ? RT.out[seg] : out;
    __syncthreads();
    if (tid < TR) {
      if (LIST) {
        const int64_t k = (tile - cumS[seg]) * TR + tid;
        rowS[tid] = (k < counts[seg]) ? (int64_t)list[RT.list_off[seg] + k] : -1;
      } else {
        const int64_t k = tile * TR + tid;
        rowS[tid] = (k < N) ? row0 + k : -1;
      }
    }
    __syncthreads();
    for (int c = 0; c < P.ncomp; ++c) {
      const double* __restrict__ o = P.o[c];
      const T* __restrict__ MT = mt_ptr<T>(P, c);
      const int32_t* __restrict__ gid = P.gid[c];
      const int ng = P.ngc[c];
      if (tid < TR * SV_MAXG) {
        int r = tid / SV_MAXG, g = tid % SV_MAXG;
        int body = P.gbody[c][g];
        acc_init(body, tot[r][g]);
      }
      // composition distance s_c = |x - o_c|^2 in FP64 (warp r, row r)
      if (P.weighted) {
        int64_t row = rowS[warp];
        double s = 0.0;
        if (row >= 0)
          for (int j = lane; j < D; j += 32) {
            double dv = Xs[row * ld + j] - o[j];
            s += dv * dv;
          }
#pragma unroll
        for (int m = 16; m >= 1; m >>= 1) s += __shfl_xor_sync(0xffffffffu, s, m);
        if (lane == 0) sS[warp][c] = s;
      }
      for (int ic = 0; ic < nchunks; ++ic) {
        const int i = ic * CH + tid;
        T accz[TR];
#pragma unroll
        for (int r = 0; r < TR; ++r) accz[r] = T(0);
        for (int jc = 0; jc < nchunks; ++jc) {
          __syncthreads();
          const int j = jc * CH + tid;
#pragma unroll
          for (int r = 0; r < TR; ++r) {
            int64_t row = rowS[r];
            double dv = 0.0;
            if (row >= 0 && j < D) dv = Xs[row * ld + j] - o[j];
            dS[r][tid] = (T)dv;
          }
          __syncthreads();
          if (i < D) {
            const int jn = min(CH, D - jc * CH);
            const T* mcol = MT + (size_t)(jc * CH) * D + i;
            for (int jj = 0; jj < jn; ++jj) {
              const T m = mcol[(size_t)jj * D];
#pragma unroll
              for (int r = 0; r < TR; ++r) accz[r] = fma(m, dS[r][jj], accz[r]);
            }
          }
        }
        __syncthreads();
#pragma unroll
        for (int r = 0; r < TR; ++r) zS[r][tid] = accz[r];
        __syncthreads();
        // epilogue: warp r reduces row r's terms of this chunk
        const int r = warp;
        if (rowS[r] >= 0) {
          const int c0 = ic * CH, c1 = min(D, c0 + CH);
          if (ic > 0 && lane == 0) {  // Rosenbrock pair across the chunk border
            const int ip = c0 - 1, g = gid[ip];
            const int body = P.gbody[c][g];
            if (body == SEVO_ROSENBROCK && ip + 1 < P.gstart[c][g + 1]) {
              Acc a;
              acc_init(body, a);
              term(body, prevz[r], T(0), true, zS[r][0], P, a);
              combine(body, tot[r][g], a);
            }
          }
          for (int g = 0; g < ng; ++g) {
            const int lo = max(c0, P.gstart[c][g]), hi = min(c1, P.gstart[c][g + 1]);
            if (lo >= hi) continue;
            const int body = P.gbody[c][g];
            Acc a;
            acc_init(body, a);
            for (int e = lo + lane; e < hi; e += 32) {
              const T z = zS[r][e - c0];
              const bool hn = (e + 1 < P.gstart[c][g + 1]);
              // a Rosenbrock pair that straddles the chunk border is added
              // when the next chunk is in shared memory
              if (body == SEVO_ROSENBROCK && hn && e + 1 >= c1) continue;
              const T zn = hn ? zS[r][e + 1 - c0] : T(0);
              term(body, z, aux_of(P, c, e, T(0)), hn, zn, P, a);
            }
            warp_reduce(body, a);
            if (lane == 0) combine(body, tot[r][g], a);
          }
          if (lane == 0) prevz[r] = zS[r][c1 - 1 - c0];
        }
        __syncwarp();
      }
      __syncthreads();
      if (lane == 0 && rowS[warp] >= 0) {
        double gsum = 0.0;
        for (int g = 0; g < ng; ++g) {
          const int body = P.gbody[c][g];
          gsum += finalize(body, tot[warp][g], P.gstart[c][g + 1] - P.gstart[c][g]);
        }
        gS[warp][c] = gsum;
      }
      __syncthreads();
    }
    if (lane == 0 && rowS[warp] >= 0) {
      const int64_t row = rowS[warp];
      double err = (P.weighted) ? compose(P, sS[warp], gS[warp]) : gS[warp][0];
      if (!isfinite(err)) {
        err = __longlong_as_double(0x7ff8000000000000ll);
        if (aux.nonfinite) atomicAdd(aux.nonfinite, 1u);
      } else if (!std::is_same<T, double>::value && aux.refine_list && err < SEVO_REFINE_THRESHOLD) {
        int k = atomicAdd(aux.refine_count, 1);
        aux.refine_list[k] = (int32_t)row;
      }
      outs[row] = err;
    }
  }
}

}  // namespace

namespace {
constexpr int SV_MAX_DEVICES = 64;
std::atomic<int> g_sms[SV_MAX_DEVICES];                 // 0: not read yet
std::atomic<uint32_t> g_once[SV_MAX_DEVICES];           // bit k: slot k done
int current_device() {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= SV_MAX_DEVICES) dev = 0;
  return dev;
}
}  // namespace

int sv_num_sms() {
  const int dev = current_device();
  int n = g_sms[dev].load(std::memory_order_acquire);
  if (n == 0) {
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0)
      n = 1;
    g_sms[dev].store(n, std::memory_order_release);
  }
  return n;
}

cudaError_t sv_once_per_device(int slot, cudaError_t (*step)()) {
  const int dev = current_device();
  const uint32_t bit = 1u << slot;
  if (g_once[dev].load(std::memory_order_acquire) & bit) return cudaSuccess;
  const cudaError_t e = step();
  if (e == cudaSuccess) g_once[dev].fetch_or(bit, std::memory_order_acq_rel);
  return e;
}

cudaError_t sv_eval_cc(const ProblemDev* Pd, int prec, const double* X, int64_t ld, int64_t row0,
                       int64_t N, double* out, EvalAux aux, cudaStream_t st) {
  if (N <= 0) return cudaSuccess;
  int64_t tiles = (N + TR - 1) / TR;
  int64_t grid = std::min<int64_t>(tiles, (int64_t)sv_num_sms() * 8);
  RefineTable none{};
  const int tk = sv_trace_begin(SEVO_TK_EVAL_CC, st);
  if (prec == SEVO_FP64)
    eval_cc_kernel<double, false><<<(unsigned)grid, NT, 0, st>>>(Pd, none, X, ld, row0, N, nullptr,
                                                                  nullptr, out, aux);
  else
    eval_cc_kernel<float, false><<<(unsigned)grid, NT, 0, st>>>(Pd, none, X, ld, row0, N, nullptr,
                                                                 nullptr, out, aux);
  sv_trace_end(tk, st);
  return cudaGetLastError();
}

cudaError_t sv_eval_refine(const RefineTable& T, const double* X, int64_t ld, int64_t max_rows,
                           const int32_t* list, const int32_t* counts, double* out,
                           cudaStream_t st) {
  if (max_rows <= 0 || T.nseg <= 0) return cudaSuccess;
  // grid-stride over the listed rows: usually few (late in a run) or none
  int64_t tiles = (max_rows + TR - 1) / TR + T.nseg;
  int64_t grid = std::min<int64_t>(tiles, (int64_t)sv_num_sms() * 2);
  EvalAux none{};
  const int tk = sv_trace_begin(SEVO_TK_REFINE, st);
  eval_cc_kernel<double, true><<<(unsigned)grid, NT, 0, st>>>(nullptr, T, X, ld, 0, 0, list,
                                                               counts, out, none);
  sv_trace_end(tk, st);
  return cudaGetLastError();
}
