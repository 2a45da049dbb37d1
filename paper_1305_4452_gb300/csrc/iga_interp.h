// FP32 reaction coefficient of the reduced-precision Jacobians: u~ = sum_a w_a U_a M_a
// at every Gauss point, then Q00 = cs gSg - cr jw/W^2 lambda e^(u~/W) (+ cr shift jw/W^2).
// A block of 128 threads takes EB = 128 / NQ elements (one thread per Gauss point):
// the elements' weighted coefficients and 1D value tables are staged in shared memory
// once, and each thread sums its point directly over the (p+1)^DIM functions.
#pragma once
#include "iga_internal.h"

namespace {

template <int DIM, int P>
struct InterpF32 {
  static constexpr int N1 = P + 1, Q = P + 1;
  static constexpr int NEN = DIM == 3 ? N1 * N1 * N1 : N1 * N1, NQ = DIM == 3 ? Q * Q * Q : Q * Q;
  static constexpr int EB = 128 / NQ > 0 ? 128 / NQ : 1;  // elements per block
  static constexpr int THREADS = 128 > NQ ? 128 : NQ;
};

// Stage the EB elements' data; returns this thread's u~ (0 when the thread has no point).
// ue: [EB][NEN] floats, tb: [EB][DIM][Q][N1] floats of shared memory.
template <int DIM, int P>
__device__ __forceinline__ float interp_u_block(const DirArgs &d0, const DirArgs &d1, const DirArgs &d2,
                                                const double *__restrict__ U, const double *__restrict__ wts, int64_t e_first,
                                                int64_t nelem, float *ue, float *tb) {
  using S = InterpF32<DIM, P>;
  constexpr int N1 = S::N1, Q = S::Q, NEN = S::NEN, NQ = S::NQ, EB = S::EB;
  for (int k = threadIdx.x; k < EB * NEN; k += blockDim.x) {
    const int le = k / NEN, a = k - le * NEN;
    const int64_t e = e_first + le;
    float v = 0.f;
    if (e < nelem && U) {
      const int e0 = (int)(e % d0.nel), e1 = (int)((e / d0.nel) % d1.nel), e2 = DIM == 3 ? (int)(e / ((int64_t)d0.nel * d1.nel)) : 0;
      const int a0 = a % N1, a1 = (a / N1) % N1, a2 = DIM == 3 ? a / (N1 * N1) : 0;
      const int64_t G = (d0.first[e0] + a0) + (int64_t)d0.n * ((d1.first[e1] + a1) + (int64_t)d1.n * ((DIM == 3 ? d2.first[e2] : 0) + a2));
      v = (float)(U[G] * (wts ? wts[G] : 1.0));
    }
    ue[k] = v;
  }
  for (int k = threadIdx.x; k < EB * DIM * Q * N1; k += blockDim.x) {
    const int le = k / (DIM * Q * N1), r = k - le * (DIM * Q * N1);
    const int ax = r / (Q * N1), ga = r - ax * (Q * N1);  // ga = g * N1 + a
    const int64_t e = e_first + le;
    float v = 0.f;
    if (e < nelem) {
      const int ee = ax == 0 ? (int)(e % d0.nel) : (ax == 1 ? (int)((e / d0.nel) % d1.nel) : (int)(e / ((int64_t)d0.nel * d1.nel)));
      const DirArgs &d = ax == 0 ? d0 : (ax == 1 ? d1 : d2);
      v = (float)d.tab[((size_t)ee * Q * N1 + ga) * 2];
    }
    tb[k] = v;
  }
  __syncthreads();
  const int le = threadIdx.x / NQ, qp = threadIdx.x - le * NQ;
  if (le >= EB || e_first + le >= nelem) return 0.f;
  const int g0 = qp % Q, g1 = (qp / Q) % Q, g2 = DIM == 3 ? qp / (Q * Q) : 0;
  const float *T = tb + le * DIM * Q * N1;
  const float *u = ue + le * NEN;
  float ut = 0.f;
#pragma unroll
  for (int a2 = 0; a2 < (DIM == 3 ? N1 : 1); a2++) {
    float s1 = 0.f;
#pragma unroll
    for (int a1 = 0; a1 < N1; a1++) {
      float s0 = 0.f;
#pragma unroll
      for (int a0 = 0; a0 < N1; a0++) s0 = fmaf(T[(0 * Q + g0) * N1 + a0], u[(a2 * N1 + a1) * N1 + a0], s0);
      s1 = fmaf(T[(1 * Q + g1) * N1 + a1], s0, s1);
    }
    ut = DIM == 3 ? fmaf(T[(2 * Q + g2) * N1 + a2], s1, ut) : s1;
  }
  return ut;
}

// u~ at the Gauss points of element e (NQ values, point index g0 + Q (g1 + Q g2)) by
// one thread: the weighted coefficients and FP32 1D tables in registers and the nested
// sums of interp_u_block (axis 0 innermost, then axis 1, then axis 2, each in function
// order) with the partial sums shared between points, so every point gets the same
// operations as there.  For elements of at most 27 points (2D, or 3D with p <= 2).
template <int DIM, int P>
__device__ __forceinline__ void interp_u_elem(const DirArgs &d0, const DirArgs &d1, const DirArgs &d2, const double *__restrict__ U,
                                              const double *__restrict__ wts, int64_t e, float *out) {
  constexpr int N1 = P + 1, Q = P + 1;
  constexpr int N2 = DIM == 3 ? N1 : 1, Q2 = DIM == 3 ? Q : 1;
  const int e0 = (int)(e % d0.nel), e1 = (int)((e / d0.nel) % d1.nel), e2 = DIM == 3 ? (int)(e / ((int64_t)d0.nel * d1.nel)) : 0;
  if (!U) {
#pragma unroll
    for (int k = 0; k < Q * Q * Q2; k++) out[k] = 0.f;
    return;
  }
  float B0[Q][N1], B1[Q][N1], B2[Q2][N2];
#pragma unroll
  for (int g = 0; g < Q; g++)
#pragma unroll
    for (int a = 0; a < N1; a++) {
      B0[g][a] = (float)d0.tab[(((size_t)e0 * Q + g) * N1 + a) * 2];
      B1[g][a] = (float)d1.tab[(((size_t)e1 * Q + g) * N1 + a) * 2];
      if (DIM == 3) B2[g < Q2 ? g : 0][a < N2 ? a : 0] = (float)d2.tab[(((size_t)e2 * Q + g) * N1 + a) * 2];
    }
  const int64_t f0 = d0.first[e0], f1 = d1.first[e1], f2 = DIM == 3 ? d2.first[e2] : 0;
  float t1[N2][Q][Q];  // [a2][g1][g0]
#pragma unroll
  for (int a2 = 0; a2 < N2; a2++) {
    float t0[N1][Q];  // [a1][g0]
#pragma unroll
    for (int a1 = 0; a1 < N1; a1++) {
      float uw[N1];
#pragma unroll
      for (int a0 = 0; a0 < N1; a0++) {
        const int64_t G = (f0 + a0) + (int64_t)d0.n * ((f1 + a1) + (int64_t)d1.n * (f2 + a2));
        uw[a0] = (float)(U[G] * (wts ? wts[G] : 1.0));
      }
#pragma unroll
      for (int g0 = 0; g0 < Q; g0++) {
        float s0 = 0.f;
#pragma unroll
        for (int a0 = 0; a0 < N1; a0++) s0 = fmaf(B0[g0][a0], uw[a0], s0);
        t0[a1][g0] = s0;
      }
    }
#pragma unroll
    for (int g1 = 0; g1 < Q; g1++)
#pragma unroll
      for (int g0 = 0; g0 < Q; g0++) {
        float s1 = 0.f;
#pragma unroll
        for (int a1 = 0; a1 < N1; a1++) s1 = fmaf(B1[g1][a1], t0[a1][g0], s1);
        t1[a2][g1][g0] = s1;
      }
  }
#pragma unroll
  for (int g2 = 0; g2 < Q2; g2++)
#pragma unroll
    for (int g1 = 0; g1 < Q; g1++)
#pragma unroll
      for (int g0 = 0; g0 < Q; g0++) {
        float u = 0.f;
        if (DIM == 3) {
#pragma unroll
          for (int a2 = 0; a2 < N2; a2++) u = fmaf(B2[g2][a2], t1[a2][g1][g0], u);
        } else {
          u = t1[0][g1][g0];
        }
        out[(g2 * Q + g1) * Q + g0] = u;
      }
}

}  // namespace
