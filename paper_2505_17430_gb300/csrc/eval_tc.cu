// eval_tc.cu -- tcgen05 evaluation: the rotation z = M (x - o) as a
// tensor-core GEMM (population x D times D x D) with the function bodies and
// per-row sums fused into the epilogue (TMEM -> registers, thread = row).
//
// Fused-producer kernel (D <= 128: the whole K extent of a 128-row tile fits
// in shared memory), persistent over a table of segments (runs of rows that
// share one problem instance), one job = (tile, component):
//   warps 0-7   epilogue: warp group g (warps 4g..4g+3) owns TMEM accumulator
//               buffer g and takes every other job; a thread walks its row's
//               z through TMEM (tcgen05.ld), FP32 bodies with one dispatch per
//               16 columns, FP64 row error, refinement listing;
//   warps 8-15  producers: FP64 rows of x (4 rows of loads in flight per
//               lane), d = x - o formed from a float hi/lo split with integer
//               and FP32 operations only (FP64 throughput on this part is
//               ~1/70 of FP32), rounded to TF32 (or split to BF16 hi/lo),
//               written as the 128B-swizzled K-major A tile;
//   warp 16     TMA loads of the rotation (B operand, reloaded only when the
//               problem or component changes), tcgen05.mma into the job's
//               TMEM buffer, TMEM allocation;
//   warp 17     row loader: TMA of the FP64 rows into a shared ring when the
//               producers convert from shared memory (idle otherwise).
// When the operator that made the rows (a DE trial, a PSO move) already wrote
// their TF32 d = x - o, the producer warps are not launched: warp 8 issues the
// MMAs and warp 9 TMA-loads the A tile straight from that operand (320 threads
// in all).  The three ways of filling A are listed above eval_tc_fused.
// BF16X3 accumulates A_hi B_hi + A_hi B_lo + A_lo B_hi into the same TMEM.
// Composition components are written per row (g_c, s_c) and combined by a
// second small kernel.  Every mbarrier wait is bounded; on a timeout the
// kernel raises an error bit, stops issuing work and still frees its TMEM.
#include <cstring>

#include "bodies.cuh"
#include "kernels.cuh"
#include "ops.cuh"
#include "tc_ptx.cuh"
#include "tc_walk.cuh"

namespace {

constexpr int BM = 128;
constexpr int NEPI = 8, NPROD = 8;
constexpr int WARP_MMA = NEPI + NPROD;
constexpr int WARP_LOAD = NEPI + NPROD + 1;    // TMA loader of FP64 rows (staged mode)
constexpr int NTHREADS = (NEPI + NPROD + 2) * 32;
constexpr int NTHREADS_OPERAND = (NEPI + 2) * 32;  // epilogue, MMA and loader warps only
constexpr int XQ = 32;                        // rows per staged quarter-tile
constexpr int MAX_XB = 4;                     // staged row buffers (ring)
constexpr long long WAIT_BUDGET = 4000000000LL;  // ~2 s of clock64
constexpr int TCOLS = 128;                      // TMEM columns per accumulator buffer
constexpr int A_KB_BYTES = BM * 128;            // one 128-byte-wide K block of A
constexpr int MAX_SEG = 64;
constexpr int MAX_XMAPS = 4;                    // distinct populations per launch (staged mode)
constexpr int MAX_OPS = 8;                      // distinct operators per launch

struct Seg {
  const ProblemDev* P;
  const double* X;   // the segment's population (rows row0 ..)
  double* out;       // its results
  uint32_t* err;     // its device error word
  int64_t row0;      // first row of the segment in X / out
  int64_t list_off;  // start of the segment's refinement sub-list
  int64_t stage0;    // composition staging: first slot row of the segment
  int32_t nrows;
  int32_t tile0;     // tiles of all earlier segments
  int32_t ncomp;
  int32_t comp;      // composition family
  int32_t sidx;      // index of the segment's refinement counter
  int32_t xmap;      // staged mode: index of the tensor map over X
  int32_t op;        // index into the launch's operators (-1: rows are loaded from X)
  int32_t pad;
};

// tensor maps over the launch's distinct populations (staged mode)
struct XMaps {
  CUtensorMap m[MAX_XMAPS];
};

// the launch's operators (segments whose rows the producers make)
struct GenOps {
  int n;
  GenOp op[MAX_OPS];
};

struct SegTable {
  int nseg, ntiles, D;
  Seg seg[MAX_SEG];
};


struct FusedGeom {
  int D, kpad, npad;
  int nkb;         // K blocks per operand copy (tf32: kpad/32, bf16: kpad/64)
  int ksteps;      // MMA K steps per product
  int b_kb_bytes;  // npad * 128
  int a_bytes;     // one A stage (both copies for bf16)
  int b_bytes;     // resident B (both copies for bf16)
  uint32_t idesc;
  int vec_ok;      // rows 16-byte aligned (X aligned, ld even): vector loads
  int dbox;        // staged mode: columns per staged row (D rounded up to even)
  int xb_bytes;    // staged mode: bytes of one quarter-tile buffer
  int nxb;         // staged mode: number of quarter-tile buffers
  long long probe_wait;  // > 0: test of the timeout path (SEVO_POLICY_TEST_WAIT)
};

struct __align__(8) Bars {
  uint64_t a_full[2], a_empty[2], t_full[2], t_empty[2], s_full[2];
  uint64_t x_full[MAX_XB], x_empty[MAX_XB];
  uint64_t b_full, mma_done;
  uint64_t probe;  // never arrived on: the timeout test waits on it
  uint32_t tmem_base;
  int abort;
};

// a wait gave up: stop this CTA and flag every segment (its remaining jobs,
// whichever segments they belong to, are not done)
__device__ void raise_abort(Bars* bars, const SegTable& T) {
  bars->abort = 1;
  for (int s = 0; s < T.nseg; ++s)
    if (T.seg[s].err) atomicOr(T.seg[s].err, SV_DEVERR_TIMEOUT);
}

// The job sequence of one CTA: tiles blockIdx.x, +gridDim.x, ...; each tile
// has ncomp(segment) jobs.  Every role walks the same sequence.
struct JobIter {
  const SegTable* T;
  int tile, s, c;
  __device__ void init(const SegTable* t) {
    T = t;
    tile = blockIdx.x;
    s = 0;
    c = 0;
    while (s + 1 < T->nseg && tile >= T->seg[s + 1].tile0) ++s;
  }
  __device__ bool valid() const { return tile < T->ntiles; }
  __device__ void next() {
    if (++c < T->seg[s].ncomp) return;
    c = 0;
    tile += gridDim.x;
    while (s + 1 < T->nseg && tile >= T->seg[s + 1].tile0) ++s;
  }
  __device__ const Seg& seg() const { return T->seg[s]; }
  __device__ int local_tile() const { return tile - T->seg[s].tile0; }
};

// ------------------------------------------------------------ epilogue walk
// the whole row: every group finalized and summed (FP64)
template <bool FAST>
__device__ __forceinline__ double walk_row(uint32_t taddr, int D, int c, bool comp,
                                           const ProblemDev& P) {
  double gsum = 0.0;
  float zf, zl;
  walk_cols<FAST>(taddr, 0, D, c, comp, P, zf, zl, [&](int g, const Acc32& acc) {
    const int body = P.gbody[c][g];
    gsum += (double)finalize32(body, acc, P.gstart[c][g + 1] - P.gstart[c][g]);
  });
  return gsum;
}

struct ListOut {
  int32_t* list;
  int32_t* counts;
  uint32_t* nonfinite;
};

__device__ __forceinline__ void emit(double err, int64_t row, double* out, const ListOut& lo,
                                     const Seg& sg) {
  if (!isfinite(err)) {
    err = __longlong_as_double(0x7ff8000000000000ll);
    if (lo.nonfinite) atomicAdd(lo.nonfinite, 1u);
  } else if (lo.list && err < SEVO_REFINE_THRESHOLD) {
    int k = atomicAdd(lo.counts + sg.sidx, 1);
    lo.list[sg.list_off + k] = (int32_t)row;
  }
  out[row] = err;
}

// one producer lane: 4 FP64 values of row r (columns k0..k0+3) -> d = x - o
// from the float hi/lo split -> TF32 (or BF16 hi/lo) into the 128B-swizzled
// K-major A tile; for a composition also the row's |d|^2 (warp sum)
template <bool BF16>
__device__ __forceinline__ void convert_store(int r, const double (&x)[4], int k0, int D,
                                              const FusedGeom& geo, const float (&ohv)[4],
                                              const float (&olv)[4], bool comp, int lane,
                                              float* sSa, unsigned char* At) {
  // unconditional: columns past D hold x = 0 and o = 0, so d = 0 there
  float d[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) d[q] = sv_operand_d(x[q], ohv[q], olv[q]);
  if (comp) {
    float sq = d[0] * d[0] + d[1] * d[1] + d[2] * d[2] + d[3] * d[3];
#pragma unroll
    for (int m = 16; m >= 1; m >>= 1) sq += __shfl_xor_sync(0xffffffffu, sq, m);
    if (lane == 0) sSa[r] = sq;
  }
  const int sw = r & 7;
  if (k0 >= geo.kpad) return;
  if (BF16) {
    // 64 bf16 per 128-byte K block: k0 -> block k0/64, chunk (k0%64)/8, half (k0%8)/4
    const int kb = k0 >> 6, ch = (k0 & 63) >> 3, hf = (k0 & 7) >> 2;
    uint32_t hi2[2], lo2[2];
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      __nv_bfloat16 h0 = __float2bfloat16_rn(d[2 * q]), h1 = __float2bfloat16_rn(d[2 * q + 1]);
      __nv_bfloat16 l0 = __float2bfloat16_rn(d[2 * q] - __bfloat162float(h0));
      __nv_bfloat16 l1 = __float2bfloat16_rn(d[2 * q + 1] - __bfloat162float(h1));
      hi2[q] = (uint32_t)__bfloat16_as_ushort(h0) | ((uint32_t)__bfloat16_as_ushort(h1) << 16);
      lo2[q] = (uint32_t)__bfloat16_as_ushort(l0) | ((uint32_t)__bfloat16_as_ushort(l1) << 16);
    }
    const int off = kb * A_KB_BYTES + r * 128 + ((ch ^ sw) << 4) + hf * 8;
    *reinterpret_cast<uint2*>(At + off) = make_uint2(hi2[0], hi2[1]);
    *reinterpret_cast<uint2*>(At + geo.nkb * A_KB_BYTES + off) = make_uint2(lo2[0], lo2[1]);
  } else {
    // 32 tf32 per 128-byte K block: k0 -> block k0/32, chunk (k0%32)/4
    const int kb = k0 >> 5, ch = (k0 & 31) >> 2;
    const int off = kb * A_KB_BYTES + r * 128 + ((ch ^ sw) << 4);
    *reinterpret_cast<float4*>(At + off) =
        make_float4(tc::to_tf32(d[0]), tc::to_tf32(d[1]), tc::to_tf32(d[2]), tc::to_tf32(d[3]));
  }
}

// quad jq of batch row `row` made by the operator: a DE trial quad (written
// to U) or four moved coordinates of a particle (written to X and V in
// place), returned in v
__device__ __forceinline__ void make_row_quad(const GenOp& op, unsigned long long gen,
                                              int64_t row, int jq, double (&v)[4]) {
  const int r = (int)(row / op.NP), i = (int)(row - (int64_t)r * op.NP);
  switch (op.alg) {
    case SEVO_DE_RAND1:
      de_trial_elem<SEVO_DE_RAND1>(op.X, op.U, nullptr, nullptr, nullptr, op.part, op.seeds,
                                   op.NP, op.D, op.ld, op.F, op.cr_thr, op.lb, op.ub, 0, gen, r,
                                   i, jq, nullptr, nullptr, nullptr, v);
      break;
    case SEVO_DE_CTPB:
      de_trial_elem<SEVO_DE_CTPB>(op.X, op.U, op.A, op.asize, op.order, op.part, op.seeds, op.NP,
                                  op.D, op.ld, op.F, op.cr_thr, op.lb, op.ub, op.pk, gen, r, i,
                                  jq, nullptr, nullptr, nullptr, v);
      break;
    case SEVO_DE_SHADE:
      de_trial_elem<SEVO_DE_SHADE>(op.X, op.U, nullptr, nullptr, op.order, op.part, op.seeds,
                                   op.NP, op.D, op.ld, 0.0, 0ull, op.lb, op.ub, op.pk, gen, r, i,
                                   jq, op.Fi, op.CRi, op.kpb, v);
      break;
    default: {  // PSO move, in place
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int j = jq * 4 + q;
        v[q] = 0.0;
        if (j < op.D) {
          const int64_t e = row * op.ld + j;
          double vn;
          const double xn = pso_moved(op.U, op.V, op.P, op.guide, op.seeds, gen, op.NP, op.ld,
                                      op.w, op.c1, op.c2, op.lb, op.ub, r, i, j, row, e, &vn);
          op.U[e] = xn;
          op.V[e] = vn;
          v[q] = xn;
        }
      }
    }
  }
}

// Where the A tile comes from (XM):
//   XM_DIRECT  producers load FP64 rows from global memory and convert them
//              (A double-buffered);
//   XM_STAGED  FP64 rows are streamed by TMA (32-row quarter tiles) into a
//              ring of shared-memory buffers and converted from there (A
//              single-buffered);
//   XM_OPERAND the operator that made the rows also wrote their converted
//              operand (TF32, the same bits sv_operand_d gives here); the
//              loader warp TMA-loads it straight into the 128B-swizzled A tile
//              (double-buffered) and the producers have nothing to do.
constexpr int XM_DIRECT = 0, XM_STAGED = 1, XM_OPERAND = 2;
template <bool BF16, int XM>
__global__ void __launch_bounds__(NTHREADS, 1)
    eval_tc_fused(const __grid_constant__ SegTable T, const FusedGeom geo,
                  const __grid_constant__ XMaps maps, const __grid_constant__ GenOps ops,
                  int64_t ld, double* __restrict__ comp_g, double* __restrict__ comp_s,
                  ListOut lo) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  __shared__ Bars bars;
  __shared__ float sS[2][BM];

  unsigned char* base = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  // staged: [A][B][x ring]; direct: [A0][A1][B]
  constexpr bool XTMA = XM == XM_STAGED;
  unsigned char* sA[2] = {base, XTMA ? base : base + geo.a_bytes};
  unsigned char* sB = base + (XTMA ? 1 : 2) * geo.a_bytes;
  unsigned char* sX = sB + geo.b_bytes;

  // roles: operand mode has no producer warps, and launches without them
  constexpr int W_MMA = XM == XM_OPERAND ? NEPI : WARP_MMA;
  constexpr int W_LOAD = W_MMA + 1;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (tid == 0) {
    for (int b = 0; b < 2; ++b) {
      tc::mbar_init(&bars.a_full[b], XM == XM_OPERAND ? 1 : NPROD);
      tc::mbar_init(&bars.a_empty[b], 1);
      tc::mbar_init(&bars.t_full[b], 1);
      tc::mbar_init(&bars.t_empty[b], NEPI / 2);
      tc::mbar_init(&bars.s_full[b], NPROD);
    }
    for (int b = 0; b < MAX_XB; ++b) {
      tc::mbar_init(&bars.x_full[b], 1);
      tc::mbar_init(&bars.x_empty[b], NPROD);
    }
    tc::mbar_init(&bars.b_full, 1);
    tc::mbar_init(&bars.mma_done, 1);
    tc::mbar_init(&bars.probe, 1);
    bars.abort = 0;
    tc::fence_mbar_init();
  }
  if (blockIdx.x == 0 && tid == 0) {  // the operators' counters, for the later kernels
    for (int k = 0; k < ops.n; ++k)
      if (ops.op[k].cs.on) {
        ops.op[k].ctl->gen = ops.op[k].cs.gen;
        ops.op[k].ctl->count = ops.op[k].cs.count;
      }
  }
  if (geo.probe_wait > 0) {
    // the timeout path under test: one bounded wait on a barrier nothing
    // arrives on, before any TMEM allocation, TMA copy or MMA is issued, so
    // that the CTA can leave with nothing in flight
    __syncthreads();
    if (tid == 0 && !tc::mbar_wait(&bars.probe, 0, &bars.abort, geo.probe_wait))
      raise_abort(&bars, T);
    __syncthreads();
    if (bars.abort) return;
  }
  if (warp == W_MMA) {
    tc::tmem_alloc(&bars.tmem_base, 2 * TCOLS);
    tc::tmem_relinquish();
  }
  tc::tc_fence_before();
  __syncthreads();
  tc::tc_fence_after();
  const uint32_t tmem = bars.tmem_base;
  const int D = geo.D;

  if (warp == W_MMA) {
    // ------------------------------------------------------------ MMA warp
    if (lane == 0) {
      JobIter it;
      it.init(&T);
      const ProblemDev* curP = nullptr;
      int cur_c = -1;
      uint32_t b_phase = 0, done_phase = 0;
      bool pending_done = false;
      for (int64_t j = 0; it.valid(); ++j, it.next()) {
        const Seg& sg = it.seg();
        const int c = it.c;
        const int a = (int)(j & 1);
        const uint32_t u = (uint32_t)(j >> 1);
        if (sg.P != curP || c != cur_c) {
          if (pending_done) {  // the previous job's MMAs must finish reading B
            if (!tc::mbar_wait(&bars.mma_done, done_phase, &bars.abort, WAIT_BUDGET)) {
              raise_abort(&bars, T);
              break;
            }
            done_phase ^= 1u;
            pending_done = false;
          }
          const CUtensorMap* m0 = BF16 ? sg.P->tmaphi[c] : sg.P->tmap32[c];
          const CUtensorMap* m1 = sg.P->tmaplo[c];
          tc::mbar_arrive_expect_tx(&bars.b_full, (uint32_t)geo.b_bytes);
          for (int kb = 0; kb < geo.nkb; ++kb) {
            if (BF16) {
              tc::tma_load_2d(sB + kb * geo.b_kb_bytes, m0, &bars.b_full, kb * 64, 0);
              tc::tma_load_2d(sB + (geo.nkb + kb) * geo.b_kb_bytes, m1, &bars.b_full, kb * 64, 0);
            } else {
              tc::tma_load_2d(sB + kb * geo.b_kb_bytes, m0, &bars.b_full, kb * 32, 0);
            }
          }
          if (!tc::mbar_wait(&bars.b_full, b_phase, &bars.abort, WAIT_BUDGET)) {
            raise_abort(&bars, T);
            break;
          }
          b_phase ^= 1u;
          curP = sg.P;
          cur_c = c;
        }
        const int ab = XTMA ? 0 : a;                        // A buffer
        const uint32_t apar = XTMA ? (uint32_t)(j & 1) : (u & 1u);
        if (!tc::mbar_wait(&bars.a_full[ab], apar, &bars.abort, WAIT_BUDGET) ||
            !tc::mbar_wait(&bars.t_empty[a], (u & 1u) ^ 1u, &bars.abort, WAIT_BUDGET)) {
          raise_abort(&bars, T);
          break;
        }
        tc::tc_fence_after();
        const uint32_t d_tmem = tmem + (uint32_t)(a * TCOLS);
        const uint32_t aS = tc::smem_u32(sA[ab]);
        const uint32_t bS = tc::smem_u32(sB);
        if (BF16) {
          const uint32_t a_lo = aS + (uint32_t)(geo.nkb * A_KB_BYTES);
          const uint32_t b_lo = bS + (uint32_t)(geo.nkb * geo.b_kb_bytes);
          for (int ks = 0; ks < geo.ksteps; ++ks) {
            const uint32_t ka = (uint32_t)((ks >> 2) * A_KB_BYTES + (ks & 3) * 32);
            const uint32_t kbb = (uint32_t)((ks >> 2) * geo.b_kb_bytes + (ks & 3) * 32);
            tc::mma_f16(d_tmem, tc::sdesc_sw128(aS + ka), tc::sdesc_sw128(bS + kbb), geo.idesc,
                        ks > 0 ? 1u : 0u);
            tc::mma_f16(d_tmem, tc::sdesc_sw128(aS + ka), tc::sdesc_sw128(b_lo + kbb), geo.idesc, 1);
            tc::mma_f16(d_tmem, tc::sdesc_sw128(a_lo + ka), tc::sdesc_sw128(bS + kbb), geo.idesc, 1);
          }
        } else {
          for (int ks = 0; ks < geo.ksteps; ++ks) {
            const uint32_t ka = (uint32_t)((ks >> 2) * A_KB_BYTES + (ks & 3) * 32);
            const uint32_t kbb = (uint32_t)((ks >> 2) * geo.b_kb_bytes + (ks & 3) * 32);
            tc::mma_tf32(d_tmem, tc::sdesc_sw128(aS + ka), tc::sdesc_sw128(bS + kbb), geo.idesc,
                         ks > 0 ? 1u : 0u);
          }
        }
        tc::mma_commit(&bars.a_empty[ab]);
        tc::mma_commit(&bars.t_full[a]);
        // if the next job needs another B, track when these MMAs are done
        JobIter nx = it;
        nx.next();
        if (nx.valid() && (nx.seg().P != curP || nx.c != cur_c)) {
          tc::mma_commit(&bars.mma_done);
          pending_done = true;
        }
      }
    }
    __syncwarp();
  } else if (warp == W_LOAD) {
    // ------------------------------------------------------------ row loader
    if (XM == XM_OPERAND && lane == 0) {
      // the operand tiles: buffer j & 1, free again once job j - 2's MMAs
      // have read it
      JobIter it;
      it.init(&T);
      for (int64_t j = 0; it.valid(); ++j, it.next()) {
        const Seg& sg = it.seg();
        const int a = (int)(j & 1);
        const uint32_t u = (uint32_t)(j >> 1);
        if (!tc::mbar_wait(&bars.a_empty[a], (u & 1u) ^ 1u, &bars.abort, WAIT_BUDGET)) {
          raise_abort(&bars, T);
          break;
        }
        const int32_t row0 = (int32_t)(sg.row0 + (int64_t)it.local_tile() * BM);
        tc::mbar_arrive_expect_tx(&bars.a_full[a], (uint32_t)geo.a_bytes);
        for (int kb = 0; kb < geo.nkb; ++kb)
          tc::tma_load_2d(sA[a] + kb * A_KB_BYTES, &maps.m[sg.xmap], &bars.a_full[a], kb * 32,
                          row0);
      }
    }
    if (XTMA && lane == 0) {
      JobIter it;
      it.init(&T);
      uint32_t q = 0;  // quarter-tiles issued
      bool ok = true;
      for (int64_t j = 0; it.valid() && ok; ++j, it.next()) {
        const Seg& sg = it.seg();
        const int64_t row0 = sg.row0 + (int64_t)it.local_tile() * BM;
        for (int h = 0; h < BM / XQ; ++h, ++q) {
          const int b = (int)(q % (uint32_t)geo.nxb);
          const uint32_t use = q / (uint32_t)geo.nxb;
          if (!tc::mbar_wait(&bars.x_empty[b], (use & 1u) ^ 1u, &bars.abort, WAIT_BUDGET)) {
            raise_abort(&bars, T);
            ok = false;
            break;
          }
          tc::mbar_arrive_expect_tx(&bars.x_full[b], (uint32_t)geo.xb_bytes);
          tc::tma_load_2d(sX + (size_t)b * geo.xb_bytes, &maps.m[sg.xmap], &bars.x_full[b], 0,
                          (int32_t)(row0 + h * XQ));
        }
      }
    }
    __syncwarp();
  } else if (warp >= NEPI && warp < W_MMA) {
    // ------------------------------------------------------------ producers
    // (idle when the loader brings the operand: the role is compiled out)
    if (XM != XM_OPERAND) {
      const int pw = warp - NEPI;
      constexpr int RPW = BM / NPROD;  // rows per producer warp
      const int k0 = lane * 4;         // lane owns columns k0..k0+3 (kpad <= 128)
      const bool full4 = (k0 + 3 < D) && geo.vec_ok;
      JobIter it;
      it.init(&T);
      for (int64_t j = 0; it.valid(); ++j, it.next()) {
        const Seg& sg = it.seg();
        const int c = it.c;
        const bool comp = sg.comp;
        const int a = (int)(j & 1);
        const uint32_t u = (uint32_t)(j >> 1);
        const int ab = XTMA ? 0 : a;
        const uint32_t apar = XTMA ? (uint32_t)((j & 1) ^ 1) : ((u & 1u) ^ 1u);
        if (!tc::mbar_wait(&bars.a_empty[ab], apar, &bars.abort, WAIT_BUDGET) ||
            (comp && !tc::mbar_wait(&bars.t_empty[a], (u & 1u) ^ 1u, &bars.abort, WAIT_BUDGET))) {
          if (lane == 0) raise_abort(&bars, T);
          break;
        }
        const float* __restrict__ oh = sg.P->oh32[c];
        const float* __restrict__ ol = sg.P->ol32[c];
        float ohv[4], olv[4];
#pragma unroll
        for (int t = 0; t < 4; ++t) {
          const int k = k0 + t;
          ohv[t] = (k < D) ? __ldg(oh + k) : 0.f;
          olv[t] = (k < D) ? __ldg(ol + k) : 0.f;
        }
        const int64_t lrow0 = (int64_t)it.local_tile() * BM;
        unsigned char* At = sA[ab];
        if (XTMA) {
          // quarter-tiles of 32 rows from the staged ring: warp pw converts 4 rows
          bool okq = true;
          for (int h = 0; h < BM / XQ; ++h) {
            const uint32_t qi = (uint32_t)j * (BM / XQ) + (uint32_t)h;
            const int b = (int)(qi % (uint32_t)geo.nxb);
            const uint32_t use = qi / (uint32_t)geo.nxb;
            if (!tc::mbar_wait(&bars.x_full[b], use & 1u, &bars.abort, WAIT_BUDGET)) {
              if (lane == 0) raise_abort(&bars, T);
              okq = false;
              break;
            }
            const double* xs = reinterpret_cast<const double*>(sX + (size_t)b * geo.xb_bytes);
#pragma unroll
            for (int t = 0; t < XQ / NPROD; ++t) {
              const int rq = pw * (XQ / NPROD) + t;  // row within the quarter
              const int r = h * XQ + rq;             // row within the tile
              double xv[4] = {0.0, 0.0, 0.0, 0.0};
              if (lrow0 + r < sg.nrows) {
                const double* xr = xs + rq * geo.dbox;
                if (k0 + 3 < D) {
                  const double2 p0 = *reinterpret_cast<const double2*>(xr + k0);
                  const double2 p1 = *reinterpret_cast<const double2*>(xr + k0 + 2);
                  xv[0] = p0.x;
                  xv[1] = p0.y;
                  xv[2] = p1.x;
                  xv[3] = p1.y;
                } else {
#pragma unroll
                  for (int qq = 0; qq < 4; ++qq)
                    if (k0 + qq < D) xv[qq] = xr[k0 + qq];
                }
              }
              convert_store<BF16>(r, xv, k0, D, geo, ohv, olv, comp, lane, sS[a], At);
            }
            __syncwarp();
            if (lane == 0) tc::mbar_arrive(&bars.x_empty[b]);
          }
          if (!okq) break;
        } else if (sg.op >= 0) {
          // rows made here: DE trials or moved particles (component 0), read
          // back from the segment's rows by later components of a composition
          const GenOp& op = ops.op[sg.op];
          const unsigned long long gen = op.cs.on ? op.cs.gen : op.ctl->gen;
          for (int rb = 0; rb < RPW; rb += 4) {
            double xv[4][4];
#pragma unroll
            for (int t = 0; t < 4; ++t) {
              const int r = pw * RPW + rb + t;
              const int64_t lr = lrow0 + r;
#pragma unroll
              for (int q = 0; q < 4; ++q) xv[t][q] = 0.0;
              if (lr < sg.nrows && k0 < D) {
                const int64_t row = sg.row0 + lr;
                if (c == 0)
                  make_row_quad(op, gen, row, lane, xv[t]);
                else
                  load_quad(sg.X + row * ld, k0, D, xv[t]);
              }
            }
#pragma unroll
            for (int t = 0; t < 4; ++t)
              convert_store<BF16>(pw * RPW + rb + t, xv[t], k0, D, geo, ohv, olv, comp, lane, sS[a], At);
          }
        } else
        for (int rb = 0; rb < RPW; rb += 4) {
          double xv[4][4];
#pragma unroll
          for (int t = 0; t < 4; ++t) {
            const int r = pw * RPW + rb + t;
            const int64_t lr = lrow0 + r;
#pragma unroll
            for (int q = 0; q < 4; ++q) xv[t][q] = 0.0;
            if (lr < sg.nrows) {
              const double* xr = sg.X + (sg.row0 + lr) * ld;
              if (full4) {
                const double2 p0 = __ldg(reinterpret_cast<const double2*>(xr + k0));
                const double2 p1 = __ldg(reinterpret_cast<const double2*>(xr + k0 + 2));
                xv[t][0] = p0.x;
                xv[t][1] = p0.y;
                xv[t][2] = p1.x;
                xv[t][3] = p1.y;
              } else {
#pragma unroll
                for (int q = 0; q < 4; ++q)
                  if (k0 + q < D) xv[t][q] = __ldg(xr + k0 + q);
              }
            }
          }
#pragma unroll
          for (int t = 0; t < 4; ++t)
            convert_store<BF16>(pw * RPW + rb + t, xv[t], k0, D, geo, ohv, olv, comp, lane, sS[a], At);
        }
        __syncwarp();
        tc::fence_proxy_async_smem();
        __syncwarp();
        if (lane == 0) {
          tc::mbar_arrive(&bars.a_full[XTMA ? 0 : a]);
          if (comp) tc::mbar_arrive(&bars.s_full[a]);
        }
      }
    }
  } else {
    // ------------------------------------------------------------ epilogue
    // group g = warp / 4 takes the jobs of parity g (TMEM buffer g); thread
    // = row 32 * (warp % 4) + lane = TMEM lane.
    const int g = warp >> 2;
    const int r = (warp & 3) * 32 + lane;
    const uint32_t taddr = tmem + ((uint32_t)((warp & 3) * 32) << 16) + (uint32_t)(g * TCOLS);
    JobIter it;
    it.init(&T);
    // s_full[g] completes only on composition jobs of parity g: its phase is
    // counted separately from t_full[g], which completes on every job
    uint32_t comp_uses = 0;
    for (int64_t j = 0; it.valid(); ++j, it.next()) {
      if ((int)(j & 1) != g) continue;
      const Seg& sg = it.seg();
      const int c = it.c;
      const bool comp = sg.comp;
      const uint32_t u = (uint32_t)(j >> 1);
      const uint32_t sp = comp_uses & 1u;
      if (comp) ++comp_uses;
      if (!tc::mbar_wait(&bars.t_full[g], u & 1u, &bars.abort, WAIT_BUDGET) ||
          (comp && !tc::mbar_wait(&bars.s_full[g], sp, &bars.abort, WAIT_BUDGET))) {
        raise_abort(&bars, T);
        break;
      }
      tc::tc_fence_after();
      const float s_c = comp ? sS[g][r] : 0.f;
      const double gsum = walk_row<!BF16>(taddr, D, c, comp, *sg.P);
      tc::tc_fence_before();
      __syncwarp();
      if (lane == 0) tc::mbar_arrive(&bars.t_empty[g]);
      const int64_t lr = (int64_t)it.local_tile() * BM + r;
      if (lr < sg.nrows) {
        if (comp) {
          const int64_t slot = (sg.stage0 + lr) * SV_MAXC + c;
          comp_g[slot] = gsum;
          comp_s[slot] = (double)s_c;
        } else {
          emit(gsum, sg.row0 + lr, sg.out, lo, sg);
        }
      }
    }
  }
  tc::tc_fence_before();
  __syncthreads();
  if (warp == W_MMA) {
    if (bars.abort) {  // let any MMA still in flight finish before freeing TMEM
      for (int k = 0; k < 1000; ++k) __nanosleep(1000);
    }
    tc::tc_fence_after();
    tc::tmem_dealloc(tmem, 2 * TCOLS);
  }
}

// composition rows: weights from the FP32 distances of the tensor-core pass
// (exactly 0 at x = o_c, where the weight collapses onto component c)
__global__ void compose_rows_kernel(const __grid_constant__ SegTable T, const double* comp_g,
                                    const double* comp_s, ListOut lo) {
  for (int s = 0; s < T.nseg; ++s) {
    const Seg& sg = T.seg[s];
    if (!sg.comp) continue;
    const ProblemDev& P = *sg.P;
    for (int64_t lr = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; lr < sg.nrows;
         lr += (int64_t)gridDim.x * blockDim.x) {
      const int64_t slot = (sg.stage0 + lr) * SV_MAXC;
      emit(compose(P, comp_s + slot, comp_g + slot), sg.row0 + lr, sg.out, lo, sg);
    }
  }
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                  const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                  const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
  static EncodeTiledFn fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (EncodeTiledFn)p;
  }
  return fn;
}

// 2D map over a row-major rows x cols matrix (cols contiguous), box
// (box_cols, box_rows), 128-byte swizzle
bool make_map(CUtensorMap* m, const void* ptr, CUtensorMapDataType dt, int esize, int cols,
              int rows, int box_cols, int box_rows) {
  EncodeTiledFn enc = encode_fn();
  if (!enc) return false;
  cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)cols * esize};
  cuuint32_t box[2] = {(cuuint32_t)box_cols, (cuuint32_t)box_rows};
  cuuint32_t estr[2] = {1, 1};
  return enc(m, dt, 2, const_cast<void*>(ptr), dims, strides, box, estr,
             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
             CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// FP64 rows of X as a 2D tensor (D columns, rows_total rows, pitch ld),
// box = dbox columns x 32 rows, no swizzle (row-major in shared memory);
// columns D..dbox-1 and rows past the end read as zeros
bool make_x_map(CUtensorMap* m, const double* X, int D, int dbox, int64_t rows_total, int64_t ld) {
  EncodeTiledFn enc = encode_fn();
  if (!enc || rows_total <= 0) return false;
  cuuint64_t dims[2] = {(cuuint64_t)D, (cuuint64_t)rows_total};
  cuuint64_t strides[1] = {(cuuint64_t)ld * 8};
  cuuint32_t box[2] = {(cuuint32_t)dbox, (cuuint32_t)XQ};
  cuuint32_t estr[2] = {1, 1};
  return enc(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 2, const_cast<double*>(X), dims, strides, box,
             estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
             CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace

// The operators' TF32 operand of a batch: rows x D floats with a pitch of
// `pitch` floats (a multiple of 4), box = one 128-byte K block (32 floats) x
// BM rows, 128-byte swizzle (the layout the A tile wants); columns D..kpad-1
// and rows past the end read as zeros
bool sv_make_operand_map(CUtensorMap* m, const float* A, int D, int64_t rows, int pitch) {
  EncodeTiledFn enc = encode_fn();
  if (!enc || rows <= 0 || (pitch & 3) || ((uintptr_t)A & 15)) return false;
  cuuint64_t dims[2] = {(cuuint64_t)D, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)pitch * 4};
  cuuint32_t box[2] = {32u, (cuuint32_t)BM};
  cuuint32_t estr[2] = {1, 1};
  return enc(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float*>(A), dims, strides, box,
             estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
             CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

namespace {

FusedGeom fused_geom(const ProblemDev& h, bool bf16) {
  FusedGeom g;
  g.D = h.D;
  g.kpad = h.kpad;
  g.npad = h.npad;
  g.b_kb_bytes = h.npad * 128;
  if (bf16) {
    g.nkb = h.kpad / 64;
    g.a_bytes = 2 * g.nkb * A_KB_BYTES;
    g.b_bytes = 2 * g.nkb * g.b_kb_bytes;
    g.ksteps = (h.D + 15) / 16;
    g.idesc = tc::idesc_make(1, BM, h.npad);
  } else {
    g.nkb = h.kpad / 32;
    g.a_bytes = g.nkb * A_KB_BYTES;
    g.b_bytes = g.nkb * g.b_kb_bytes;
    g.ksteps = (h.D + 7) / 8;
    g.idesc = tc::idesc_make(2, BM, h.npad);
  }
  return g;
}

}  // namespace

// rows of the B box: the whole padded N extent for the fused kernel
static int b_box_rows(const ProblemDev& h) { return h.D <= 128 ? h.npad : 128; }

int32_t sv_build_tmaps(sevo_problem* p) {
  const ProblemDev& h = p->host_desc;
  const int rows = b_box_rows(h);
  for (int c = 0; c < h.ncomp; ++c) {
    if (!make_map(&p->tmap_f32[c], h.M32[c], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, h.kpad, h.npad,
                  32, rows) ||
        !make_map(&p->tmap_hi[c], h.Mhi[c], CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, h.kpad, h.npad,
                  64, rows) ||
        !make_map(&p->tmap_lo[c], h.Mlo[c], CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, h.kpad, h.npad,
                  64, rows))
      return SEVO_ERR_CUDA;
    // 64-row boxes for the large-D GEMM's 64-column tiles
    if (h.D > 128 &&
        (!make_map(&p->tmap_f32h[c], h.M32[c], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, h.kpad, h.npad,
                   32, 64) ||
         !make_map(&p->tmap_hih[c], h.Mhi[c], CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, h.kpad, h.npad,
                   64, 64) ||
         !make_map(&p->tmap_loh[c], h.Mlo[c], CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, h.kpad,
                   h.npad, 64, 64)))
      return SEVO_ERR_CUDA;
  }
  p->tmap_rows = rows;
  p->tmaps_ready = true;
  return SEVO_OK;
}

// composition scratch: per row, SV_MAXC slots of g_c and of s_c (FP64)
size_t sv_eval_tc_scratch_bytes(bool any_comp, int, int64_t rows) {
  return any_comp ? (size_t)rows * SV_MAXC * 16 : 0;
}

// the fused kernel's dynamic shared memory above the default 48 KB (once per device)
static cudaError_t set_fused_smem() {
  const int lim = 224 * 1024;  // opt-in maximum minus this kernel's static shared memory
  const cudaFuncAttribute a = cudaFuncAttributeMaxDynamicSharedMemorySize;
  cudaError_t e = cudaFuncSetAttribute(eval_tc_fused<true, XM_STAGED>, a, lim);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(eval_tc_fused<true, XM_DIRECT>, a, lim);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(eval_tc_fused<false, XM_STAGED>, a, lim);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(eval_tc_fused<false, XM_DIRECT>, a, lim);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(eval_tc_fused<false, XM_OPERAND>, a, lim);
  return e;
}

cudaError_t sv_eval_tc_segments(const TcSegment* segs, int nseg, int prec, int64_t ld,
                                int32_t* list, const int64_t* list_off, int32_t* counts,
                                uint32_t* nonfinite, void* scratch, size_t scratch_bytes,
                                cudaStream_t st) {
  if (nseg <= 0) return cudaSuccess;
  if (nseg > SV_MAX_SEG) return cudaErrorInvalidValue;
  const ProblemDev& h0 = segs[0].p->host_desc;
  if (h0.D > 128) return cudaErrorNotSupported;
  const bool bf16 = (prec == SEVO_BF16X3);
  FusedGeom g = fused_geom(h0, bf16);
  // the populations of the segments: vector loads and TMA staging need every
  // one 16-byte aligned with an even pitch; staging takes one tensor map per
  // distinct population (at most MAX_XMAPS)
  const double* xs[MAX_XMAPS];
  int64_t xrows[MAX_XMAPS];
  int nx = 0;
  bool aligned = (ld & 1) == 0, few = true;
  int xmap_of[SV_MAX_SEG];
  for (int k = 0; k < nseg; ++k) {
    const TcSegment& s = segs[k];
    aligned = aligned && (((uintptr_t)s.X & 15) == 0);
    int m = 0;
    while (m < nx && xs[m] != s.X) ++m;
    if (m == nx) {
      if (nx == MAX_XMAPS) {
        few = false;
        m = 0;
      } else {
        xs[nx] = s.X;
        xrows[nx] = 0;
        ++nx;
      }
    }
    if (xs[m] == s.X) xrows[m] = std::max<int64_t>(xrows[m], s.row0 + s.nrows);
    xmap_of[k] = m;
  }
  // operators: rows made by the producers (DE trials, PSO moves)
  GenOps ops;
  std::memset(&ops, 0, sizeof(ops));
  int op_of[SV_MAX_SEG];
  const GenOp* op_src[MAX_OPS];
  for (int k = 0; k < nseg; ++k) {
    op_of[k] = -1;
    if (!segs[k].op) continue;
    int m = 0;
    while (m < ops.n && op_src[m] != segs[k].op) ++m;
    if (m == ops.n) {
      if (ops.n == MAX_OPS) return cudaErrorInvalidValue;
      op_src[m] = segs[k].op;
      ops.op[ops.n++] = *segs[k].op;
    }
    op_of[k] = m;
  }
  g.vec_ok = aligned;
  g.probe_wait = sv_policy_test_wait();
  g.dbox = (h0.D + 1) & ~1;
  g.xb_bytes = XQ * g.dbox * 8;
  const size_t budget = 220 * 1024;
  const size_t fixed = (size_t)g.a_bytes + g.b_bytes + 1024;
  g.nxb = (int)std::min<size_t>(MAX_XB, (budget - fixed) / (size_t)g.xb_bytes);
  // operand mode: every segment's rows come with their converted operand,
  // written by the operator that made them (TF32, one component, no weights)
  int amap_of[SV_MAX_SEG];
  const CUtensorMap* am[MAX_XMAPS];
  int na = 0;
  bool operand = !bf16 && ops.n == 0;
  for (int k = 0; k < nseg && operand; ++k) {
    const TcSegment& s = segs[k];
    if (!s.amap || s.p->ncomp != 1 || sv_weighted_family(s.p->family)) {
      operand = false;
      break;
    }
    int m = 0;
    while (m < na && am[m] != s.amap) ++m;
    if (m == na) {
      if (na == MAX_XMAPS) {
        operand = false;
        break;
      }
      am[na++] = s.amap;
    }
    amap_of[k] = m;
  }
  // staged rows come from TMA loads of X, which an operator's rows do not have yet
  bool staged = !operand && aligned && few && g.nxb >= 2 && ops.n == 0;
  const size_t smem = staged ? fixed + (size_t)g.nxb * g.xb_bytes
                             : (size_t)2 * g.a_bytes + g.b_bytes + 1024;
  {
    const cudaError_t e = sv_once_per_device(SV_ONCE_FUSED_SMEM, set_fused_smem);
    if (e != cudaSuccess) return e;
  }
  SegTable T;
  T.nseg = nseg;
  T.D = h0.D;
  int tiles = 0;
  int64_t stage_rows = 0;
  for (int k = 0; k < nseg; ++k) {
    const TcSegment& s = segs[k];
    Seg& d = T.seg[k];
    d.P = s.p->desc_d;
    d.X = s.X;
    d.out = s.out;
    d.err = s.err;
    d.row0 = s.row0;
    d.list_off = list_off ? list_off[k] : 0;
    d.nrows = (int32_t)s.nrows;
    d.tile0 = tiles;
    d.comp = sv_weighted_family(s.p->family);
    d.ncomp = s.p->ncomp;
    d.sidx = k;
    d.xmap = operand ? amap_of[k] : xmap_of[k];
    d.op = op_of[k];
    d.pad = 0;
    d.stage0 = stage_rows;
    tiles += (int)((s.nrows + BM - 1) / BM);
    if (d.comp) stage_rows += s.nrows;
  }
  T.ntiles = tiles;
  if (tiles == 0) return cudaSuccess;
  // composition staging: SV_MAXC slots of g_c and of s_c per composition row
  double* comp_g = nullptr;
  double* comp_s = nullptr;
  if (stage_rows > 0) {
    const size_t need = (size_t)stage_rows * SV_MAXC * 16;
    if (!scratch || scratch_bytes < need) return cudaErrorInvalidValue;
    comp_g = (double*)scratch;
    comp_s = (double*)scratch + (size_t)stage_rows * SV_MAXC;
  }
  const ListOut lo{list, counts, nonfinite};
  const int grid = std::min(tiles, sv_num_sms());
  XMaps maps;
  std::memset(&maps, 0, sizeof(maps));
  for (int m = 0; m < na && operand; ++m) maps.m[m] = *am[m];
  for (int m = 0; m < nx && staged; ++m)
    staged = make_x_map(&maps.m[m], xs[m], h0.D, g.dbox, xrows[m], ld);
  const size_t smem_direct = (size_t)2 * g.a_bytes + g.b_bytes + 1024;
  const int tk = sv_trace_begin(SEVO_TK_EVAL_TC_FUSED, st);
  if (operand) {
    eval_tc_fused<false, XM_OPERAND><<<grid, NTHREADS_OPERAND, smem_direct, st>>>(T, g, maps, ops, ld,
                                                                          comp_g, comp_s, lo);
  } else if (!staged) {
    if (bf16)
      eval_tc_fused<true, XM_DIRECT><<<grid, NTHREADS, smem_direct, st>>>(T, g, maps, ops, ld,
                                                                          comp_g, comp_s, lo);
    else
      eval_tc_fused<false, XM_DIRECT><<<grid, NTHREADS, smem_direct, st>>>(T, g, maps, ops, ld,
                                                                           comp_g, comp_s, lo);
  } else {
    if (bf16)
      eval_tc_fused<true, XM_STAGED><<<grid, NTHREADS, smem, st>>>(T, g, maps, ops, ld, comp_g,
                                                                   comp_s, lo);
    else
      eval_tc_fused<false, XM_STAGED><<<grid, NTHREADS, smem, st>>>(T, g, maps, ops, ld, comp_g,
                                                                    comp_s, lo);
  }
  sv_trace_end(tk, st);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  if (stage_rows > 0) {
    const int cgrid = std::max(1, std::min(sv_num_sms() * 4, (int)((stage_rows + 255) / 256)));
    const int tkc = sv_trace_begin(SEVO_TK_COMPOSE, st);
    compose_rows_kernel<<<cgrid, 256, 0, st>>>(T, comp_g, comp_s, lo);
    sv_trace_end(tkc, st);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  return cudaSuccess;
}
