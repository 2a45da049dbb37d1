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

}  // namespace
