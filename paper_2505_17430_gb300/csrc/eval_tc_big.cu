// eval_tc_big.cu -- tcgen05 evaluation for D > 128, where the rotation GEMM
// (N x D times D x D, 2 N D^2 flops) is tensor-bound.
//
//   1. convert: d = x - o_c once per element (float hi/lo split, integer and
//      FP32 work), stored as TF32 (or BF16 hi and lo) rows padded to kpad;
//      for compositions also s_c = |x - o_c|^2 per row;
//   2. gemm: persistent CTAs over jobs (128-row tile, 128-column chunk of z),
//      full K per job: one thread issues TMA loads of A and B K-blocks into a
//      multi-stage shared-memory ring (128B swizzle), one thread issues
//      tcgen05.mma into one of four TMEM accumulators (the whole 512-column
//      TMEM, so the MMA runs up to three jobs ahead of the epilogue), sixteen
//      epilogue warps walk the chunk (four per TMEM lane quarter, 32 columns
//      each; thread = row = TMEM lane) and store, per 32-column slice, the
//      per-group FP32 accumulators plus the slice's first and last z, row
//      index fastest so that a warp's stores are coalesced;
//   3. combine: per row, the slice records are merged in column order (the
//      Rosenbrock pair across a slice border is added here), the groups are
//      finished, the FP64 error is written and rows below the refinement
//      threshold are listed.
// Splitting z into 128-column chunks gives tiles x chunks independent jobs,
// enough to fill the GPU even for N = 1024.  Waits are bounded as in the
// fused kernel.
#include "kernels.cuh"
#include "tc_walk.cuh"

namespace {

constexpr int BM = 128;
constexpr int WPQ = 4;               // epilogue warps per TMEM lane quarter
constexpr int NEPI = 4 * WPQ;
constexpr int SUB = 32;              // columns of z per record slice, for every N tile
constexpr int MAX_NBUF = 8;
constexpr int MAX_STAGES = 8;
// N tile of one job (64, 128 or 256 columns of z): NBUF TMEM accumulators of
// BN columns fill the 512-column TMEM; a job has NSL record slices of SUB
// columns, walked by the epilogue warps of each lane quarter in turn; the B
// operand of a stage is NB boxes of 128 rotation rows (a 64-column tile uses
// the first 64 rows of its box).  The slices, hence the per-row sums and
// every result bit, are the same for every BN.
template <int BN>
struct Tile {
  static constexpr int NBUF = 512 / BN, NSL = BN / SUB, NB = BN >= 128 ? BN / 128 : 1;
  static constexpr int BBOX = BN >= 128 ? 128 : 64;  // rotation rows per B box
  static constexpr int B_BYTES = NB * BBOX * 128;   // one operand copy's B per stage
};
constexpr int WARP_TMA = NEPI, WARP_MMA = NEPI + 1;
constexpr int NTHREADS = (NEPI + 2) * 32;
constexpr int KB_BYTES = 128 * 128;  // one 128-row x 128-byte K block (A or B)
constexpr int REC = 3 * SV_MAXG + 2;  // float slots per (row, slice) record
constexpr long long WAIT_BUDGET = 4000000000LL;

struct BigGeom {
  int D, kpad, nkb, nchunks, nsub, ntiles, stages, stage_bytes;
  int64_t N;
  uint32_t idesc;
};

struct __align__(8) BigBars {
  uint64_t full[MAX_STAGES], empty[MAX_STAGES], t_full[MAX_NBUF], t_empty[MAX_NBUF];
  uint32_t tmem_base;
  int abort;
};

__device__ __forceinline__ void big_abort(BigBars* b, uint32_t* dev_err) {
  b->abort = 1;
  if (dev_err) atomicOr(dev_err, SV_DEVERR_TIMEOUT);
}

// ---------------------------------------------------------------- convert
// One block per row (grid-stride over rows), thread t = quads t, t + 256, ...
// of 4 consecutive columns: 16-byte FP64 loads when rows are 16-byte
// aligned, 16-byte (TF32) or 8-byte (BF16 hi and lo) stores, every quad of
// the row in flight at once; s_c = |x - o_c|^2 in FP32 by a block reduction
// in a fixed order (warp shuffles, then the warps' partial sums in index
// order), so the result does not depend on scheduling.
constexpr int CVT_THREADS = 256;

template <bool BF16>
__global__ void __launch_bounds__(CVT_THREADS)
    convert_kernel(const ProblemDev* __restrict__ P, int c, const double* __restrict__ X,
                   int64_t ld, int64_t row0, int64_t N, int D, int kpad, bool vec,
                   float* __restrict__ A32, __nv_bfloat16* __restrict__ Ahi,
                   __nv_bfloat16* __restrict__ Alo, double* __restrict__ s_out) {
  __shared__ float wsum[CVT_THREADS / 32];
  const float* __restrict__ oh = P->oh32[c];
  const float* __restrict__ ol = P->ol32[c];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  for (int64_t r = blockIdx.x; r < N; r += gridDim.x) {
    const double* xr = X + (row0 + r) * ld;
    float sq = 0.f;
    for (int k0 = tid * 4; k0 < kpad; k0 += CVT_THREADS * 4) {
      double xv[4] = {0.0, 0.0, 0.0, 0.0};
      if (vec && k0 + 3 < D) {
        const double2 p0 = __ldg(reinterpret_cast<const double2*>(xr + k0));
        const double2 p1 = __ldg(reinterpret_cast<const double2*>(xr + k0 + 2));
        xv[0] = p0.x;
        xv[1] = p0.y;
        xv[2] = p1.x;
        xv[3] = p1.y;
      } else {
#pragma unroll
        for (int q = 0; q < 4; ++q)
          if (k0 + q < D) xv[q] = __ldg(xr + k0 + q);
      }
      float d[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int k = k0 + q;
        d[q] = 0.f;
        if (k < D) {
          float xh, xl;
          sv_split_hi_lo(xv[q], xh, xl);
          d[q] = (xh - __ldg(oh + k)) + (xl - __ldg(ol + k));
          sq += d[q] * d[q];
        }
      }
      if (BF16) {
        __nv_bfloat16 h[4], l[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          h[q] = __float2bfloat16_rn(d[q]);
          l[q] = __float2bfloat16_rn(d[q] - __bfloat162float(h[q]));
        }
        uint2 hv, lv;
        hv.x = (uint32_t)__bfloat16_as_ushort(h[0]) | ((uint32_t)__bfloat16_as_ushort(h[1]) << 16);
        hv.y = (uint32_t)__bfloat16_as_ushort(h[2]) | ((uint32_t)__bfloat16_as_ushort(h[3]) << 16);
        lv.x = (uint32_t)__bfloat16_as_ushort(l[0]) | ((uint32_t)__bfloat16_as_ushort(l[1]) << 16);
        lv.y = (uint32_t)__bfloat16_as_ushort(l[2]) | ((uint32_t)__bfloat16_as_ushort(l[3]) << 16);
        *reinterpret_cast<uint2*>(Ahi + r * kpad + k0) = hv;
        *reinterpret_cast<uint2*>(Alo + r * kpad + k0) = lv;
      } else {
        *reinterpret_cast<float4*>(A32 + r * kpad + k0) =
            make_float4(tc::to_tf32(d[0]), tc::to_tf32(d[1]), tc::to_tf32(d[2]), tc::to_tf32(d[3]));
      }
    }
    if (s_out) {
#pragma unroll
      for (int m = 16; m >= 1; m >>= 1) sq += __shfl_xor_sync(0xffffffffu, sq, m);
      if (lane == 0) wsum[warp] = sq;
      __syncthreads();
      if (tid == 0) {
        float t = 0.f;
        for (int w = 0; w < CVT_THREADS / 32; ++w) t += wsum[w];
        s_out[(row0 + r) * SV_MAXC + c] = (double)t;
      }
      __syncthreads();
    }
  }
}

// ---------------------------------------------------------------- gemm
template <bool BF16, int BN>
__global__ void __launch_bounds__(NTHREADS, 1)
    gemm_big_kernel(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapAlo,
                    const ProblemDev* __restrict__ P, const BigGeom geo, int c, bool comp,
                    float* __restrict__ part, uint32_t* dev_err) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  __shared__ BigBars bars;
  unsigned char* base = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int S = geo.stages;
  constexpr int NBUF = Tile<BN>::NBUF, NSL = Tile<BN>::NSL, NB = Tile<BN>::NB;
  constexpr int BBOX = Tile<BN>::BBOX, B_BYTES = Tile<BN>::B_BYTES;
  if (tid == 0) {
    for (int s = 0; s < S; ++s) {
      tc::mbar_init(&bars.full[s], 1);
      tc::mbar_init(&bars.empty[s], 1);
    }
    for (int b = 0; b < NBUF; ++b) {
      tc::mbar_init(&bars.t_full[b], 1);
      tc::mbar_init(&bars.t_empty[b], NEPI);
    }
    bars.abort = 0;
    tc::fence_mbar_init();
  }
  if (warp == WARP_MMA) {
    tc::tmem_alloc(&bars.tmem_base, 512);
    tc::tmem_relinquish();
  }
  tc::tc_fence_before();
  __syncthreads();
  tc::tc_fence_after();
  const uint32_t tmem = bars.tmem_base;
  const int njobs_total = geo.ntiles * geo.nchunks;
  const int KBLK = BF16 ? 64 : 32;  // elements per 128-byte K block

  if (warp == WARP_TMA) {
    if (lane == 0) {
      const CUtensorMap* mB = BBOX == 64 ? (BF16 ? P->tmaphih[c] : P->tmap32h[c])
                                         : (BF16 ? P->tmaphi[c] : P->tmap32[c]);
      const CUtensorMap* mBlo = BBOX == 64 ? P->tmaploh[c] : P->tmaplo[c];
      uint32_t it = 0;
      bool ok = true;
      for (int job = blockIdx.x; job < njobs_total && ok; job += gridDim.x) {
        const int tile = job / geo.nchunks, nb = job % geo.nchunks;
        for (int kb = 0; kb < geo.nkb; ++kb, ++it) {
          const int s = (int)(it % (uint32_t)S);
          const uint32_t ph = (it / (uint32_t)S) & 1u;
          if (!tc::mbar_wait(&bars.empty[s], ph ^ 1u, &bars.abort, WAIT_BUDGET)) {
            big_abort(&bars, dev_err);
            ok = false;
            break;
          }
          unsigned char* st = base + (size_t)s * geo.stage_bytes;
          tc::mbar_arrive_expect_tx(&bars.full[s], (uint32_t)geo.stage_bytes);
          // stage: [A][B x NB] (+ [A_lo][B_lo x NB] for BF16); B boxes past
          // the padded rotation read zeros
          tc::tma_load_2d(st, &mapA, &bars.full[s], kb * KBLK, tile * BM);
#pragma unroll
          for (int q = 0; q < NB; ++q)
            tc::tma_load_2d(st + KB_BYTES + q * BBOX * 128, mB, &bars.full[s], kb * KBLK,
                            nb * BN + q * 128);
          if (BF16) {
            unsigned char* lo = st + KB_BYTES + B_BYTES;
            tc::tma_load_2d(lo, &mapAlo, &bars.full[s], kb * KBLK, tile * BM);
#pragma unroll
            for (int q = 0; q < NB; ++q)
              tc::tma_load_2d(lo + KB_BYTES + q * BBOX * 128, mBlo, &bars.full[s], kb * KBLK,
                              nb * BN + q * 128);
          }
        }
      }
    }
    __syncwarp();
  } else if (warp == WARP_MMA) {
    if (lane == 0) {
      uint32_t it = 0;
      int jl = 0;
      bool ok = true;
      for (int job = blockIdx.x; job < njobs_total && ok; job += gridDim.x, ++jl) {
        const int a = jl % NBUF;
        const uint32_t u = (uint32_t)(jl / NBUF);
        if (!tc::mbar_wait(&bars.t_empty[a], (u & 1u) ^ 1u, &bars.abort, WAIT_BUDGET)) {
          big_abort(&bars, dev_err);
          break;
        }
        tc::tc_fence_after();
        const uint32_t d_tmem = tmem + (uint32_t)(a * BN);
        for (int kb = 0; kb < geo.nkb; ++kb, ++it) {
          const int s = (int)(it % (uint32_t)S);
          const uint32_t ph = (it / (uint32_t)S) & 1u;
          if (!tc::mbar_wait(&bars.full[s], ph, &bars.abort, WAIT_BUDGET)) {
            big_abort(&bars, dev_err);
            ok = false;
            break;
          }
          tc::tc_fence_after();
          const uint32_t aS = tc::smem_u32(base + (size_t)s * geo.stage_bytes);
          const uint32_t bS = aS + KB_BYTES;
#pragma unroll
          for (int ks = 0; ks < 4; ++ks) {
            const uint32_t acc = (kb > 0 || ks > 0) ? 1u : 0u;
            if (BF16) {
              const uint32_t aLo = aS + KB_BYTES + B_BYTES, bLo = aLo + KB_BYTES;
              tc::mma_f16(d_tmem, tc::sdesc_sw128(aS + ks * 32), tc::sdesc_sw128(bS + ks * 32),
                          geo.idesc, acc);
              tc::mma_f16(d_tmem, tc::sdesc_sw128(aS + ks * 32), tc::sdesc_sw128(bLo + ks * 32),
                          geo.idesc, 1u);
              tc::mma_f16(d_tmem, tc::sdesc_sw128(aLo + ks * 32), tc::sdesc_sw128(bS + ks * 32),
                          geo.idesc, 1u);
            } else {
              tc::mma_tf32(d_tmem, tc::sdesc_sw128(aS + ks * 32), tc::sdesc_sw128(bS + ks * 32),
                           geo.idesc, acc);
            }
          }
          tc::mma_commit(&bars.empty[s]);
        }
        if (!ok) break;
        tc::mma_commit(&bars.t_full[a]);
      }
    }
    __syncwarp();
  } else {
    // epilogue: warp w reads TMEM lane quarter w % 4 (thread = row of the
    // tile) and the job's slices w / 4, w / 4 + 4, ... (SUB columns each)
    const int r = (warp & 3) * 32 + lane;
    const int sl = warp >> 2;
    const int64_t N = geo.N;
    int jl = 0;
    for (int job = blockIdx.x; job < njobs_total; job += gridDim.x, ++jl) {
      const int tile = job / geo.nchunks, nb = job % geo.nchunks;
      const int a = jl % NBUF;
      const uint32_t u = (uint32_t)(jl / NBUF);
      if (!tc::mbar_wait(&bars.t_full[a], u & 1u, &bars.abort, WAIT_BUDGET)) {
        big_abort(&bars, dev_err);
        break;
      }
      tc::tc_fence_after();
      const int64_t row = (int64_t)tile * BM + r;
      const bool live = row < N;
      for (int ls = sl; ls < NSL; ls += WPQ) {
        const int sb = nb * NSL + ls;  // slice index within the row
        if (sb >= geo.nsub) break;     // a wide tile past the padded rotation: no record
        const int c0 = sb * SUB, c1 = min(geo.D, c0 + SUB);
        float* rec = part + (int64_t)sb * REC * N + row;  // slot k at rec[k * N]
        float zf = 0.f, zl = 0.f;
        const uint32_t taddr =
            tmem + ((uint32_t)((warp & 3) * 32) << 16) + (uint32_t)(a * BN + ls * SUB);
        if (c0 < c1) {
          walk_cols<!BF16>(taddr, c0, c1, c, comp, *P, zf, zl, [&](int g, const Acc32& acc) {
            if (live) {
              rec[(3 * g) * N] = acc.a0;
              rec[(3 * g + 1) * N] = acc.a1;
              rec[(3 * g + 2) * N] = acc.a2;
            }
          });
        }
        if (live) {
          rec[(3 * SV_MAXG) * N] = zf;
          rec[(3 * SV_MAXG + 1) * N] = zl;
        }
      }
      tc::tc_fence_before();
      __syncwarp();
      if (lane == 0) tc::mbar_arrive(&bars.t_empty[a]);
    }
  }
  tc::tc_fence_before();
  __syncthreads();
  if (warp == WARP_MMA) {
    if (bars.abort) {
      for (int k = 0; k < 1000; ++k) __nanosleep(1000);
    }
    tc::tc_fence_after();
    tc::tmem_dealloc(tmem, 512);
  }
}

// ---------------------------------------------------------------- combine
struct ListOutB {
  int32_t* list;
  int32_t* count;
  uint32_t* nonfinite;
  int64_t list_off;
};

__device__ __forceinline__ int group_of(const ProblemDev& P, int c, bool comp, int i) {
  (void)comp;
  return P.gid[c][i];
}

// one warp per row: lane l merges slices l, l + 32, ... into per-group
// accumulators (adding the Rosenbrock pair across a slice border from the
// previous slice's last z), then the groups are summed across the warp
constexpr int CMB_WARPS = 4;

__global__ void __launch_bounds__(CMB_WARPS * 32)
    combine_kernel(const ProblemDev* __restrict__ Pp, int c, bool comp, int D, int nsub, int SUB,
                   const float* __restrict__ part, int64_t row0, int64_t N,
                   double* __restrict__ out, double* __restrict__ comp_g, ListOutB lo) {
  const ProblemDev& P = *Pp;
  const int lane = threadIdx.x & 31;
  const int ng = P.ngc[c];
  const int64_t nw = (int64_t)gridDim.x * CMB_WARPS;
  for (int64_t lr = (int64_t)blockIdx.x * CMB_WARPS + (threadIdx.x >> 5); lr < N; lr += nw) {
    Acc32 acc[SV_MAXG];
#pragma unroll
    for (int g = 0; g < SV_MAXG; ++g) acc32_init(acc[g]);
    for (int sb = lane; sb < nsub; sb += 32) {
      const int c0 = sb * SUB, c1 = min(D, c0 + SUB);
      if (c0 >= c1) break;
      const float* rec = part + (int64_t)sb * REC * N + lr;  // slot k at rec[k * N]
      const int g0 = group_of(P, c, comp, c0), g1 = group_of(P, c, comp, c1 - 1);
#pragma unroll
      for (int g = 0; g < SV_MAXG; ++g) {
        if (g >= g0 && g <= g1) {
          acc[g].a0 += rec[(3 * g) * N];
          acc[g].a1 += rec[(3 * g + 1) * N];
          acc[g].a2 += rec[(3 * g + 2) * N];
        }
      }
      if (sb > 0) {  // Rosenbrock pair (c0 - 1, c0) inside one group
        const int gp = group_of(P, c, comp, c0 - 1);
        const int body = P.gbody[c][gp];
        if (gp == g0 && body == SEVO_ROSENBROCK) {
          const float zprev = part[((int64_t)(sb - 1) * REC + 3 * SV_MAXG + 1) * N + lr];
#pragma unroll
          for (int g = 0; g < SV_MAXG; ++g)
            if (g == gp) term32(SEVO_ROSENBROCK, zprev, 0.f, true, rec[(3 * SV_MAXG) * N], P, acc[g]);
        }
      }
    }
    double gsum = 0.0;
#pragma unroll
    for (int g = 0; g < SV_MAXG; ++g) {
      if (g < ng) {
        float a0 = acc[g].a0, a1 = acc[g].a1, a2 = acc[g].a2;
#pragma unroll
        for (int m = 16; m >= 1; m >>= 1) {
          a0 += __shfl_xor_sync(0xffffffffu, a0, m);
          a1 += __shfl_xor_sync(0xffffffffu, a1, m);
          a2 += __shfl_xor_sync(0xffffffffu, a2, m);
        }
        Acc32 t;
        t.a0 = a0;
        t.a1 = a1;
        t.a2 = a2;
        const int body = P.gbody[c][g];
        const int n = P.gstart[c][g + 1] - P.gstart[c][g];
        gsum += (double)finalize32(body, t, n);
      }
    }
    if (lane != 0) continue;
    const int64_t row = row0 + lr;
    if (comp) {
      comp_g[row * SV_MAXC + c] = gsum;
      continue;
    }
    double err = gsum;
    if (!isfinite(err)) {
      err = __longlong_as_double(0x7ff8000000000000ll);
      if (lo.nonfinite) atomicAdd(lo.nonfinite, 1u);
    } else if (lo.list && err < SEVO_REFINE_THRESHOLD) {
      int k = atomicAdd(lo.count, 1);
      lo.list[lo.list_off + k] = (int32_t)row;
    }
    out[row] = err;
  }
}

__global__ void compose_big_kernel(const ProblemDev* __restrict__ Pp, const double* comp_g,
                                   const double* comp_s, int64_t row0, int64_t N, double* out,
                                   ListOutB lo) {
  const ProblemDev& P = *Pp;
  for (int64_t lr = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; lr < N;
       lr += (int64_t)gridDim.x * blockDim.x) {
    const int64_t row = row0 + lr;
    double err = compose(P, comp_s + row * SV_MAXC, comp_g + row * SV_MAXC);
    if (!isfinite(err)) {
      err = __longlong_as_double(0x7ff8000000000000ll);
      if (lo.nonfinite) atomicAdd(lo.nonfinite, 1u);
    } else if (lo.list && err < SEVO_REFINE_THRESHOLD) {
      int k = atomicAdd(lo.count, 1);
      lo.list[lo.list_off + k] = (int32_t)row;
    }
    out[row] = err;
  }
}

typedef CUresult (*EncodeTiledFnB)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                   const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                   const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                   CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

bool make_a_map(CUtensorMap* m, const void* ptr, bool bf16, int kpad, int64_t rows) {
  static EncodeTiledFnB fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
      return false;
    fn = (EncodeTiledFnB)p;
  }
  const int es = bf16 ? 2 : 4;
  cuuint64_t dims[2] = {(cuuint64_t)kpad, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)kpad * es};
  cuuint32_t box[2] = {(cuuint32_t)(bf16 ? 64 : 32), (cuuint32_t)BM};
  cuuint32_t estr[2] = {1, 1};
  return fn(m, bf16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2,
            const_cast<void*>(ptr), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
            CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

size_t al256b(size_t b) { return (b + 255) & ~(size_t)255; }

}  // namespace

// scratch of one segment of `rows` rows: converted operand, chunk records,
// composition staging (per row SV_MAXC slots of g_c and of s_c)
size_t sv_eval_big_scratch_bytes(int D, bool any_comp, int prec, int64_t rows) {
  (void)prec;
  const int kpad = (D + 63) / 64 * 64;
  const int nsub = ((D + 127) / 128 * 128) / SUB;
  size_t b = al256b((size_t)rows * kpad * 4) + al256b((size_t)rows * nsub * REC * 4);
  if (any_comp) b += al256b((size_t)rows * SV_MAXC * 16);
  return b;
}

// the GEMM's dynamic shared memory above the default 48 KB (once per device)
static cudaError_t set_big_smem() {
  const int lim = 200 * 1024;
  const cudaFuncAttribute a = cudaFuncAttributeMaxDynamicSharedMemorySize;
  cudaError_t e = cudaFuncSetAttribute(gemm_big_kernel<true, 64>, a, lim);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(gemm_big_kernel<true, 128>, a, lim);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(gemm_big_kernel<true, 256>, a, lim);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(gemm_big_kernel<false, 64>, a, lim);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(gemm_big_kernel<false, 128>, a, lim);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(gemm_big_kernel<false, 256>, a, lim);
  return e;
}

cudaError_t sv_eval_tc_big(const TcSegment& seg, int prec, const double* X, int64_t ld,
                           double* out, int32_t* list, int64_t list_off, int32_t* count,
                           uint32_t* nonfinite, void* scratch, size_t scratch_bytes,
                           uint32_t* dev_err, cudaStream_t st) {
  const sevo_problem* p = seg.p;
  const ProblemDev& h = p->host_desc;
  const int64_t N = seg.nrows;
  if (N <= 0) return cudaSuccess;
  const bool bf16 = (prec == SEVO_BF16X3);
  const bool comp = sv_weighted_family(p->family);
  if (h.npad % 128 != 0 || p->tmap_rows != 128) return cudaErrorNotSupported;
  if (!scratch || scratch_bytes < sv_eval_big_scratch_bytes(h.D, comp, prec, N))
    return cudaErrorInvalidValue;
  // N tile of a job: 64, 128 or 256 columns of z, all giving the same bits.
  // Measured (SEVO_POLICY_AUTOTUNE) the first time a (D, row bucket,
  // precision) is seen outside stream capture, else a rule: the width whose
  // whole waves of persistent jobs, ceil(jobs / SMs) x the cost of one job,
  // finish first (a 256-column job measured 1.7x the flop rate of a
  // 128-column one in TF32, 1.2x in BF16X3; a 64-column job half the flops
  // for about 0.6 of the time).
  const int64_t tiles = (N + BM - 1) / BM;
  const int64_t sms = sv_num_sms();
  auto waves = [&](int bn) { return (double)((tiles * ((h.npad + bn - 1) / bn) + sms - 1) / sms); };
  const double t256 = waves(256) * (2.0 / (bf16 ? 1.2 : 1.7));
  const double t128 = waves(128), t64 = waves(64) * 0.6;
  int BN = (t256 < t128) ? 256 : 128;
  if (t64 < std::min(t128, t256)) BN = 64;
  bool tune = false;
  if (sv_policy_autotune()) {
    // a cached width that is not a candidate (an edited or foreign cache
    // file) is ignored and measured again
    int cached = sv_tune_lookup(SV_TUNE_BIG_NTILE, h.D, N, prec);
    if (cached != 64 && cached != 128 && cached != 256) cached = 0;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cached)
      BN = cached;
    else if (cudaStreamIsCapturing(st, &cs) == cudaSuccess && cs == cudaStreamCaptureStatusNone)
      tune = true;
  }
  auto geom = [&](int bn) {
    BigGeom g;
    g.D = h.D;
    g.kpad = h.kpad;
    g.nkb = h.kpad / (bf16 ? 64 : 32);
    g.nchunks = (h.npad + bn - 1) / bn;
    g.nsub = h.npad / SUB;
    g.ntiles = (int)tiles;
    g.N = N;
    const int nb = bn >= 128 ? bn / 128 : 1, bbox = bn >= 128 ? 128 : 64;
    g.stage_bytes = (bf16 ? 2 : 1) * (KB_BYTES + nb * bbox * 128);
    g.stages = std::min(MAX_STAGES, (192 * 1024) / g.stage_bytes);
    g.idesc = tc::idesc_make(bf16 ? 1 : 2, BM, bn);
    return g;
  };
  BigGeom g = geom(BN);
  // scratch: A (N x kpad fp32, or hi then lo bf16), chunk records, composition
  char* cp = (char*)scratch;
  void* Abase = cp;
  cp += al256b((size_t)N * h.kpad * 4);
  float* part = (float*)cp;
  cp += al256b((size_t)N * g.nsub * REC * 4);
  // composition staging: g_c in the first N x SV_MAXC doubles, s_c in the
  // next; both indexed by global row (row0 + local row)
  double* comp_g = nullptr;
  double* comp_s = nullptr;
  if (comp) {
    double* comp_base = (double*)cp;
    comp_g = comp_base - seg.row0 * SV_MAXC;
    comp_s = comp_base + (size_t)N * SV_MAXC - seg.row0 * SV_MAXC;
  }
  float* A32 = (float*)Abase;
  __nv_bfloat16* Ahi = (__nv_bfloat16*)Abase;
  __nv_bfloat16* Alo = Ahi + (size_t)N * h.kpad;
  CUtensorMap mA, mAlo;
  if (bf16) {
    if (!make_a_map(&mA, Ahi, true, h.kpad, N) || !make_a_map(&mAlo, Alo, true, h.kpad, N))
      return cudaErrorInvalidValue;
  } else {
    if (!make_a_map(&mA, A32, false, h.kpad, N)) return cudaErrorInvalidValue;
    mAlo = mA;
  }
  {
    const cudaError_t e = sv_once_per_device(SV_ONCE_BIG_SMEM, set_big_smem);
    if (e != cudaSuccess) return e;
  }
  const int cvt_grid = (int)std::min<int64_t>(N, (int64_t)sv_num_sms() * 16);
  const bool vec = ((uintptr_t)X % 16 == 0) && (ld % 2 == 0);
  const int cgrid = (int)std::max<int64_t>(1, std::min<int64_t>((N + 127) / 128, sv_num_sms() * 4));
  const int mgrid = (int)std::max<int64_t>(
      1, std::min<int64_t>((N + CMB_WARPS - 1) / CMB_WARPS, (int64_t)sv_num_sms() * 16));
  const ListOutB lo{list, count, nonfinite, list_off};
  auto gemm = [&](int bn, const BigGeom& gg, int c) {
    const int njobs = gg.ntiles * gg.nchunks;
    const int ggrid = std::min(njobs, sv_num_sms());
    const size_t smem = (size_t)gg.stages * gg.stage_bytes + 1024;
    if (bf16) {
      if (bn == 256)
        gemm_big_kernel<true, 256><<<ggrid, NTHREADS, smem, st>>>(mA, mAlo, p->desc_d, gg, c, comp,
                                                                  part, dev_err);
      else if (bn == 128)
        gemm_big_kernel<true, 128><<<ggrid, NTHREADS, smem, st>>>(mA, mAlo, p->desc_d, gg, c, comp,
                                                                  part, dev_err);
      else
        gemm_big_kernel<true, 64><<<ggrid, NTHREADS, smem, st>>>(mA, mAlo, p->desc_d, gg, c, comp,
                                                                 part, dev_err);
    } else {
      if (bn == 256)
        gemm_big_kernel<false, 256><<<ggrid, NTHREADS, smem, st>>>(mA, mAlo, p->desc_d, gg, c,
                                                                   comp, part, dev_err);
      else if (bn == 128)
        gemm_big_kernel<false, 128><<<ggrid, NTHREADS, smem, st>>>(mA, mAlo, p->desc_d, gg, c,
                                                                   comp, part, dev_err);
      else
        gemm_big_kernel<false, 64><<<ggrid, NTHREADS, smem, st>>>(mA, mAlo, p->desc_d, gg, c, comp,
                                                                  part, dev_err);
    }
    return cudaGetLastError();
  };
  cudaError_t e;
  for (int c = 0; c < h.ncomp; ++c) {
    int tk = sv_trace_begin(SEVO_TK_CONVERT, st);
    if (bf16)
      convert_kernel<true><<<cvt_grid, CVT_THREADS, 0, st>>>(
          p->desc_d, c, X, ld, seg.row0, N, h.D, h.kpad, vec, nullptr, Ahi, Alo,
          comp ? comp_s : nullptr);
    else
      convert_kernel<false><<<cvt_grid, CVT_THREADS, 0, st>>>(
          p->desc_d, c, X, ld, seg.row0, N, h.D, h.kpad, vec, A32, nullptr, nullptr,
          comp ? comp_s : nullptr);
    sv_trace_end(tk, st);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if (tune) {  // time every width on this data (one warm-up, then two runs each)
      tune = false;
      const int cand[3] = {64, 128, 256};
      float ms[3] = {0.f, 0.f, 0.f};
      cudaEvent_t e0 = nullptr, e1 = nullptr;
      e = cudaEventCreate(&e0);
      if (e == cudaSuccess) e = cudaEventCreate(&e1);
      for (int i = 0; i < 3 && e == cudaSuccess; ++i) {
        const BigGeom gi = geom(cand[i]);
        int tkt = sv_trace_begin(SEVO_TK_GEMM_BIG, st);
        e = gemm(cand[i], gi, c);
        sv_trace_end(tkt, st);
        if (e == cudaSuccess) e = cudaEventRecord(e0, st);
        for (int rep = 0; rep < 2 && e == cudaSuccess; ++rep) {
          tkt = sv_trace_begin(SEVO_TK_GEMM_BIG, st);
          e = gemm(cand[i], gi, c);
          sv_trace_end(tkt, st);
        }
        if (e == cudaSuccess) e = cudaEventRecord(e1, st);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms[i], e0, e1);
      }
      if (e0) cudaEventDestroy(e0);
      if (e1) cudaEventDestroy(e1);
      if (e != cudaSuccess) return e;
      int best = 1;
      for (int i = 0; i < 3; ++i)
        if (ms[i] < ms[best]) best = i;
      BN = cand[best];
      g = geom(BN);
      sv_tune_store(SV_TUNE_BIG_NTILE, h.D, N, prec, BN, ms, cand, 3);
    }
    tk = sv_trace_begin(SEVO_TK_GEMM_BIG, st);
    e = gemm(BN, g, c);
    sv_trace_end(tk, st);
    if (e != cudaSuccess) return e;
    tk = sv_trace_begin(SEVO_TK_COMBINE, st);
    combine_kernel<<<mgrid, CMB_WARPS * 32, 0, st>>>(p->desc_d, c, comp, h.D, g.nsub, SUB,
                                                     part, seg.row0, N, out, comp_g, lo);
    sv_trace_end(tk, st);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  if (comp) {
    const int tk = sv_trace_begin(SEVO_TK_COMPOSE, st);
    compose_big_kernel<<<cgrid, 128, 0, st>>>(p->desc_d, comp_g, comp_s, seg.row0, N, out, lo);
    sv_trace_end(tk, st);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  return cudaSuccess;
}
