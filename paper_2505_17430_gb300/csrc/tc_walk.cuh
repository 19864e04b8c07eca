// tc_walk.cuh -- epilogue walk over one row's z held in TMEM (thread = row =
// TMEM lane): FP32 body terms with one body dispatch per 16 columns inside a
// group, a per-element path where a chunk crosses a group border.
#pragma once
#include "bodies.cuh"
#include "tc_ptx.cuh"

template <int BODY, bool FAST>
__device__ __forceinline__ void chunk16(const float* v, const float* aux, int col0, bool pair0,
                                        float& zprev, const ProblemDev& P, Acc32& acc) {
  if (BODY == SEVO_ROSENBROCK) {
    if (pair0) term32t<FAST>(SEVO_ROSENBROCK, zprev, 0.f, true, v[0], P, acc);
#pragma unroll
    for (int k = 0; k + 1 < 16; ++k) term32t<FAST>(SEVO_ROSENBROCK, v[k], 0.f, true, v[k + 1], P, acc);
  } else if (BODY == SEVO_ELLIPSOID || BODY == SEVO_GRIEWANK) {
    float a[16];
    const float4* a4 = reinterpret_cast<const float4*>(aux + col0);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const float4 t = __ldg(a4 + q);
      a[4 * q] = t.x;
      a[4 * q + 1] = t.y;
      a[4 * q + 2] = t.z;
      a[4 * q + 3] = t.w;
    }
#pragma unroll
    for (int k = 0; k < 16; ++k) term32t<FAST>(BODY, v[k], a[k], false, 0.f, P, acc);
  } else {
#pragma unroll
    for (int k = 0; k < 16; ++k) term32t<FAST>(BODY, v[k], 0.f, false, 0.f, P, acc);
  }
  zprev = v[15];
}

// Walk columns [c0, c1) (c0 a multiple of 16; column c0 sits at TMEM address
// taddr) of component c.  Rosenbrock pairs are formed only inside [c0, c1)
// and inside a group.  close(g, acc) is called for every group the walk
// leaves and for the group it ends in.  zfirst/zlast receive z_{c0} and
// z_{c1-1} (used to join Rosenbrock pairs across walks).
template <bool FAST, class Close>
__device__ __forceinline__ void walk_cols(uint32_t taddr, int c0, int c1, int c, bool comp,
                                          const ProblemDev& P, float& zfirst, float& zlast,
                                          Close&& close) {
  (void)comp;  // groups are per component for every family
  const float* __restrict__ aux32 = P.aux32[c];
  int g = P.gid[c][c0];
  int gend = P.gstart[c][g + 1];
  int body = P.gbody[c][g];
  Acc32 acc;
  acc32_init(acc);
  float zprev = 0.f;
  zfirst = 0.f;
  // software pipeline: the next chunk's TMEM load is in flight while this
  // chunk's bodies are computed
  uint32_t cur[16], nxt[16];
  if (c0 < c1) {
    tc::tmem_ld16_issue(taddr, cur);
    tc::tmem_wait16(cur);
  }
  for (int col0 = c0; col0 < c1; col0 += 16) {
    const bool more = col0 + 16 < c1;
    if (more) tc::tmem_ld16_issue(taddr + (uint32_t)(col0 + 16 - c0), nxt);
    float v[16];
#pragma unroll
    for (int k = 0; k < 16; ++k) v[k] = __uint_as_float(cur[k]);
    if (col0 == c0) zfirst = v[0];
    while (col0 >= gend) {  // close groups that ended before this chunk
      close(g, acc);
      ++g;
      gend = P.gstart[c][g + 1];
      body = P.gbody[c][g];
      acc32_init(acc);
    }
    if (col0 + 16 <= gend && col0 + 16 <= c1) {
      const bool pair0 = col0 > P.gstart[c][g] && col0 > c0;
      switch (body) {
        case SEVO_ELLIPSOID: chunk16<SEVO_ELLIPSOID, FAST>(v, aux32, col0, pair0, zprev, P, acc); break;
        case SEVO_ROSENBROCK: chunk16<SEVO_ROSENBROCK, FAST>(v, aux32, col0, pair0, zprev, P, acc); break;
        case SEVO_RASTRIGIN: chunk16<SEVO_RASTRIGIN, FAST>(v, aux32, col0, pair0, zprev, P, acc); break;
        case SEVO_SCHWEFEL: chunk16<SEVO_SCHWEFEL, FAST>(v, aux32, col0, pair0, zprev, P, acc); break;
        case SEVO_ACKLEY: chunk16<SEVO_ACKLEY, FAST>(v, aux32, col0, pair0, zprev, P, acc); break;
        default: chunk16<SEVO_GRIEWANK, FAST>(v, aux32, col0, pair0, zprev, P, acc); break;
      }
      if (col0 + 16 == c1) zlast = v[15];
    } else {
#pragma unroll
      for (int k = 0; k < 16; ++k) {
        const int i = col0 + k;
        if (i < c1) {
          while (i == gend) {
            close(g, acc);
            ++g;
            gend = P.gstart[c][g + 1];
            body = P.gbody[c][g];
            acc32_init(acc);
          }
          const float z = v[k];
          if (body == SEVO_ROSENBROCK) {
            if (i > P.gstart[c][g] && i > c0) term32t<FAST>(SEVO_ROSENBROCK, zprev, 0.f, true, z, P, acc);
          } else {
            term32t<FAST>(body, z, aux32[i], false, 0.f, P, acc);
          }
          zprev = z;
          if (i == c1 - 1) zlast = z;
        }
      }
    }
    if (more) {
      tc::tmem_wait16(nxt);
#pragma unroll
      for (int k = 0; k < 16; ++k) cur[k] = nxt[k];
    }
  }
  close(g, acc);
}
