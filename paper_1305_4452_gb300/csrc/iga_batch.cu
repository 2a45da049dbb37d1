// Batched Newton-Krylov for many independent 2D Bratu problems in one persistent,
// graph-captured launch.
//
// Each problem ("instance") is a 2D scalar Bratu problem on the identity map
// (x = xi) with its own knot vectors, degree p <= 3, lambda and optional log-kappa
// field, and homogeneous Dirichlet values on all four sides.  One kernel is
// launched with a fixed number of CTAs per SM; each CTA takes the next instance
// from an integer work counter (instances are ordered largest first) and runs the
// whole solve for it with block-level synchronisation only:
//   residual  (FP64; Algorithm 3 with Eq. residual): one element per thread with
//             sum factorisation, then a fixed-order gather per control variable;
//   Jacobian  (FP32; Eq. jacobian): global sum factorisation over the instance's
//             mesh, axis 0 then axis 1, each entry written once, into a layout
//             sliced by 32 rows for the operator products (see jslot); axis 0 runs
//             on tiles of Gauss lines staged in shared memory (see b_stage1);
//   GMRES(m)  with right Jacobi preconditioning; FP64 Krylov vectors and
//             classical Gram-Schmidt, once or twice as gmres_cgs_refine says (one
//             warp per dot product, fixed-order warp reductions), FP32 operator
//             products; or Jacobi CG;
//   Newton    with backtracking, as in iga_solve_newton.
// There are no spin-waits: every loop is bounded by the Newton and Krylov caps.
// The launch, the copy of its arguments and the read-back of the per-instance
// reports are captured once into a CUDA graph and replayed on later solves.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <map>
#include <numeric>
#include <string>
#include <vector>

#include "iga_exp.h"
#include "iga_internal.h"

namespace {

constexpr int BMAXM = 64;  // largest GMRES restart in the batched solver
constexpr int BDOT_MAX = 16;  // largest number of row chunks per Gram-Schmidt dot

struct BMesh {  // device data shared by instances with the same knots (square meshes: both axes identical)
  int p, q, nel, n, np, N;
  int64_t nnz;
  const double *tab;   // [nel][q][p+1][2]
  const double *wq;    // [nel][q]
  const int *first, *node_e0, *node_ne, *l, *r;
  const int *pair_off, *pair_i, *pair_x0, *pair_np, *pair_po;
  const float *pair_val;  // [pts][5]
};

struct BInst {
  BMesh m;
  double lambda;
  int64_t uoff;          // offset of this instance's U in the caller's array
  const double *ck;      // [nelem][nq] kappa * jw
  const double *cr;      // [nelem][nq] jw
  const float *ck32, *cr32;  // kappa jw, line-major [x1][x0]; jw, element-major [e][qp]
  double *F, *dU, *Ut, *Ft, *dinv, *w, *V;  // V: (mmax+1) x N
  double *Fe;            // [nelem][nen]
  float *J;              // Jacobian values, sliced by 32 rows (see jslot)
  float *T1;             // stage-1 groups G0, G2: [2][x1][slot s0 < 2p+1][i0]
  float *q00, *z32;      // q00: [x1][x0], line-major (x = e q + g)
};

// The batch Jacobian is stored by slices of 32 consecutive rows, slot-major within a
// slice: slot s = (j1 - l(i1)) (2p+1) + (j0 - l(i0)) of row A = (i0, i1) is at
// J[(A / 32) 32 (2p+1)^2 + 32 s + A % 32], so that a warp's loads of one slot for its 32
// rows are one 128-byte access.  Slots outside a row's stencil stay zero.
__host__ __device__ __forceinline__ int64_t jslot(int A, int s, int wf) {
  return (int64_t)(A >> 5) * 32 * wf * wf + 32 * s + (A & 31);
}
__host__ __device__ __forceinline__ int64_t jsize(int N, int p) {
  return (int64_t)((N + 31) / 32) * 32 * (2 * p + 1) * (2 * p + 1);
}

struct BArgs {
  double *U;
  iga_newton_opts opts;
  int dot_chunks;  // work unit of the Gram-Schmidt dots: row chunks per dot (0: as many as keep every warp busy)
  int jac_lines;   // element tile of the Jacobian's first stage: Gauss lines per shared-memory tile (1, 2, 4, 8)
};

struct BRep {
  int newton_its, krylov_its, status, pad;
  double fnorm0, fnorm;
  uint64_t t0, t1;  // %globaltimer (ns) at the start and the end of the instance's solve
};

__device__ __forceinline__ uint64_t gtimer() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

struct Cta {
  int tid, nt, lane, warp, nw;
  double *red;  // shared, >= 38 doubles (cta_sum: 0..33; scalars shared by thread 0: 35..37)
  float *zs;    // shared FP32 operand vector of the operator products (N floats), or null
  float *tile;  // the same dynamic shared memory (tile_cap floats), for the Jacobian's line tiles
  int tile_cap;
  int dot_chunks;  // row chunks per Gram-Schmidt dot (BArgs::dot_chunks)
  int jac_lines;   // Gauss lines per stage-1 tile (BArgs::jac_lines)
};

__device__ __forceinline__ double warp_sum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return __shfl_sync(0xffffffffu, v, 0);
}

// block sum in a fixed order, returned to every thread
__device__ double cta_sum(const Cta &c, double v) {
  v = warp_sum(v);
  if (c.lane == 0) c.red[c.warp] = v;
  __syncthreads();
  if (c.warp == 0) {
    double r = (c.lane < c.nw) ? c.red[c.lane] : 0.0;
    r = warp_sum(r);
    if (c.lane == 0) c.red[33] = r;
  }
  __syncthreads();
  double r = c.red[33];
  __syncthreads();
  return r;
}

// two block sums at once (one pair of barriers fewer), each in the order of cta_sum
__device__ void cta_sum2(const Cta &c, double &a, double &b) {
  a = warp_sum(a);
  b = warp_sum(b);
  if (c.lane == 0) {
    c.red[c.warp] = a;
    c.red[16 + c.warp] = b;
  }
  __syncthreads();
  if (c.warp == 0) {
    double r = (c.lane < c.nw) ? c.red[c.lane] : 0.0;
    double t = (c.lane < c.nw) ? c.red[16 + c.lane] : 0.0;
    r = warp_sum(r);
    t = warp_sum(t);
    if (c.lane == 0) {
      c.red[34] = r;
      c.red[35] = t;
    }
  }
  __syncthreads();
  a = c.red[34];
  b = c.red[35];
  __syncthreads();
}

// slot of the diagonal entry of row A
__device__ __forceinline__ int diag_slot(const BMesh &M, int A, int wf) {
  const int i0 = A % M.n, i1 = A / M.n;
  return (i1 - M.l[i1]) * wf + (i0 - M.l[i0]);
}

__device__ __forceinline__ bool on_bnd(int i0, int i1, int n) { return i0 == 0 || i1 == 0 || i0 == n - 1 || i1 == n - 1; }

// ---------------------------------------------------------------- residual --
template <int P>
__device__ void b_residual(const BInst &I, const double *__restrict__ U, double *__restrict__ F, const Cta &c) {
  constexpr int N1 = P + 1, Q = P + 1, NEN = N1 * N1, NQ = Q * Q;
  const BMesh &M = I.m;
  const int nel = M.nel;
  const double lam = I.lambda;
  for (int e = c.tid; e < nel * nel; e += c.nt) {
    const int e0 = e % nel, e1 = e / nel;
    const double *B0 = M.tab + (size_t)e0 * Q * N1 * 2, *B1 = M.tab + (size_t)e1 * Q * N1 * 2;
    const int f0 = M.first[e0], f1 = M.first[e1];
    double Ue[NEN];
#pragma unroll
    for (int a1 = 0; a1 < N1; a1++)
#pragma unroll
      for (int a0 = 0; a0 < N1; a0++) Ue[a1 * N1 + a0] = U[(f0 + a0) + (size_t)M.n * (f1 + a1)];
    double T[2][N1][Q];
#pragma unroll
    for (int s = 0; s < 2; s++)
#pragma unroll
      for (int a1 = 0; a1 < N1; a1++)
#pragma unroll
        for (int g0 = 0; g0 < Q; g0++) {
          double acc = 0.0;
#pragma unroll
          for (int a0 = 0; a0 < N1; a0++) acc = fma(B0[(g0 * N1 + a0) * 2 + s], Ue[a1 * N1 + a0], acc);
          T[s][a1][g0] = acc;
        }
    double vs[NQ], v0[NQ], v1[NQ];
#pragma unroll
    for (int g1 = 0; g1 < Q; g1++)
#pragma unroll
      for (int g0 = 0; g0 < Q; g0++) {
        double u = 0.0, d0 = 0.0, d1 = 0.0;
#pragma unroll
        for (int a1 = 0; a1 < N1; a1++) {
          const double b = B1[(g1 * N1 + a1) * 2], db = B1[(g1 * N1 + a1) * 2 + 1];
          u = fma(b, T[0][a1][g0], u);
          d0 = fma(b, T[1][a1][g0], d0);
          d1 = fma(db, T[0][a1][g0], d1);
        }
        const int qp = g1 * Q + g0;
        const double ck = I.ck[(size_t)e * NQ + qp], cr = I.cr[(size_t)e * NQ + qp];
        vs[qp] = -cr * lam * iga_exp(u);
        v0[qp] = ck * d0;
        v1[qp] = ck * d1;
      }
    double Z[2][N1][Q];
#pragma unroll
    for (int a1 = 0; a1 < N1; a1++)
#pragma unroll
      for (int g0 = 0; g0 < Q; g0++) {
        double z0 = 0.0, z1 = 0.0;
#pragma unroll
        for (int g1 = 0; g1 < Q; g1++) {
          const double b = B1[(g1 * N1 + a1) * 2], db = B1[(g1 * N1 + a1) * 2 + 1];
          const int qp = g1 * Q + g0;
          z0 = fma(b, vs[qp], z0);
          z0 = fma(db, v1[qp], z0);
          z1 = fma(b, v0[qp], z1);
        }
        Z[0][a1][g0] = z0;
        Z[1][a1][g0] = z1;
      }
#pragma unroll
    for (int a1 = 0; a1 < N1; a1++)
#pragma unroll
      for (int a0 = 0; a0 < N1; a0++) {
        double acc = 0.0;
#pragma unroll
        for (int g0 = 0; g0 < Q; g0++) {
          acc = fma(B0[(g0 * N1 + a0) * 2], Z[0][a1][g0], acc);
          acc = fma(B0[(g0 * N1 + a0) * 2 + 1], Z[1][a1][g0], acc);
        }
        I.Fe[(size_t)e * NEN + a1 * N1 + a0] = acc;
      }
  }
  __syncthreads();
  for (int A = c.tid; A < M.N; A += c.nt) {
    const int i0 = A % M.n, i1 = A / M.n;
    if (on_bnd(i0, i1, M.n)) {
      F[A] = U[A];
      continue;
    }
    double acc = 0.0;
    for (int e1 = M.node_e0[i1]; e1 < M.node_e0[i1] + M.node_ne[i1]; e1++)
      for (int e0 = M.node_e0[i0]; e0 < M.node_e0[i0] + M.node_ne[i0]; e0++)
        acc += I.Fe[(size_t)(e1 * nel + e0) * NEN + (i1 - M.first[e1]) * N1 + (i0 - M.first[e0])];
    F[A] = acc;
  }
  __syncthreads();
}

// ---------------------------------------------------------------- Jacobian --
// Stage 1 (axis 0) on tiles of L Gauss lines x1: the tile's Q00 and kappa jw lines are
// copied to shared memory (contiguous, line-major), then each work item, a 1D pair
// (i0, slot s0) of axis 0, forms G0 = sum P00 Q00 + P11 kappa jw and G2 = sum P00 kappa jw
// over the pair's common Gauss points for all L lines at once, so that each pair-table
// value serves L lines.  L is the element-tile shape the autotuner chooses (Cta::jac_lines);
// it changes neither the terms nor their order, only the reuse.
template <int P, int L>
__device__ void b_stage1(const BInst &I, const Cta &c) {
  constexpr int Q = P + 1, WF = 2 * P + 1;
  const BMesh &M = I.m;
  const int X = M.nel * Q, n = M.n;
  const size_t plane = (size_t)X * WF * n;
  float *lq = c.tile, *lk = c.tile + L * X;  // [L][X] each
  for (int x1a = 0; x1a < X; x1a += L) {
    const int nl = min(L, X - x1a);
    for (int idx = c.tid; idx < nl * X; idx += c.nt) {
      lq[idx] = I.q00[(size_t)x1a * X + idx];
      lk[idx] = I.ck32[(size_t)x1a * X + idx];
    }
    __syncthreads();
    for (int it = c.tid; it < WF * n; it += c.nt) {
      const int s0 = it / n, i0 = it - s0 * n;
      if (s0 > M.r[i0] - M.l[i0]) continue;
      const int pi = M.pair_off[i0] + s0;
      const int xs = M.pair_x0[pi], cnt = M.pair_np[pi];
      const float *pv = M.pair_val + (size_t)M.pair_po[pi] * IGA_PVS;
      float g0[L], g2[L];
#pragma unroll
      for (int l = 0; l < L; l++) g0[l] = g2[l] = 0.f;
      for (int k = 0; k < cnt; k++) {
        const float p00 = pv[IGA_PVS * k + 0], p11 = pv[IGA_PVS * k + 3];
#pragma unroll
        for (int l = 0; l < L; l++) {
          const float q = lq[l * X + xs + k], ck = lk[l * X + xs + k];
          g0[l] = fmaf(p00, q, g0[l]);
          g0[l] = fmaf(p11, ck, g0[l]);
          g2[l] = fmaf(p00, ck, g2[l]);
        }
      }
#pragma unroll
      for (int l = 0; l < L; l++)
        if (l < nl) {
          const size_t o = ((size_t)(x1a + l) * WF + s0) * n + i0;
          I.T1[o] = g0[l];
          I.T1[plane + o] = g2[l];
        }
    }
    __syncthreads();
  }
}

template <int P>
__device__ void b_jacobian(const BInst &I, const double *__restrict__ U, float *__restrict__ J, const Cta &c) {
  constexpr int N1 = P + 1, Q = P + 1, NQ = Q * Q, WF = 2 * P + 1;
  const BMesh &M = I.m;
  const int nel = M.nel, X = nel * Q, np = M.np, n = M.n;
  const float lam = (float)I.lambda;
  // Q00 = -jw lambda e^u at every Gauss point (u interpolated in FP32), line-major
  for (int e = c.tid; e < nel * nel; e += c.nt) {
    const int e0 = e % nel, e1 = e / nel;
    const double *B0 = M.tab + (size_t)e0 * Q * N1 * 2, *B1 = M.tab + (size_t)e1 * Q * N1 * 2;
    const int f0 = M.first[e0], f1 = M.first[e1];
    float T[N1][Q];
#pragma unroll
    for (int a1 = 0; a1 < N1; a1++)
#pragma unroll
      for (int g0 = 0; g0 < Q; g0++) {
        float acc = 0.f;
#pragma unroll
        for (int a0 = 0; a0 < N1; a0++) acc = fmaf((float)B0[(g0 * N1 + a0) * 2], (float)U[(f0 + a0) + (size_t)M.n * (f1 + a1)], acc);
        T[a1][g0] = acc;
      }
#pragma unroll
    for (int g1 = 0; g1 < Q; g1++)
#pragma unroll
      for (int g0 = 0; g0 < Q; g0++) {
        float u = 0.f;
#pragma unroll
        for (int a1 = 0; a1 < N1; a1++) u = fmaf((float)B1[(g1 * N1 + a1) * 2], T[a1][g0], u);
        const int qp = g1 * Q + g0;
        I.q00[(size_t)(e1 * Q + g1) * X + e0 * Q + g0] = -I.cr32[(size_t)e * NQ + qp] * lam * expf(u);
      }
  }
  __syncthreads();
  // stage 1 (axis 0), on tiles of L lines that fit the shared memory
  int L = c.jac_lines;
  while (L > 1 && 2 * L * X > c.tile_cap) L >>= 1;
  switch (L) {
    case 8: b_stage1<P, 8>(I, c); break;
    case 4: b_stage1<P, 4>(I, c); break;
    case 2: b_stage1<P, 2>(I, c); break;
    default: b_stage1<P, 1>(I, c); break;
  }
  // final stage (axis 1): J = sum P1^00 G0 + P1^11 G2, one entry per work item; items
  // (axis-1 pair, slot s0, i0) with i0 fastest, so that a warp reads consecutive G values
  // and writes consecutive rows of one slot of the sliced layout
  const size_t plane = (size_t)X * WF * n;
  for (int wi = c.tid; wi < np * WF * n; wi += c.nt) {
    const int p1 = wi / (WF * n), rem = wi - p1 * (WF * n);
    const int s0 = rem / n, i0 = rem - s0 * n;
    if (s0 > M.r[i0] - M.l[i0]) continue;
    const int i1 = M.pair_i[p1], s1 = p1 - M.pair_off[i1];
    const int xs = M.pair_x0[p1], cnt = M.pair_np[p1];
    const float *pv = M.pair_val + (size_t)M.pair_po[p1] * IGA_PVS;
    float acc = 0.f;
    for (int k = 0; k < cnt; k++) {
      const size_t o = ((size_t)(xs + k) * WF + s0) * n + i0;
      acc = fmaf(pv[IGA_PVS * k + 0], I.T1[o], acc);
      acc = fmaf(pv[IGA_PVS * k + 3], I.T1[plane + o], acc);
    }
    const int j0 = M.l[i0] + s0, j1 = M.l[i1] + s1;
    const int A = i0 + n * i1, B = j0 + n * j1;
    if (on_bnd(i0, i1, n) || on_bnd(j0, j1, n)) acc = (A == B) ? 1.f : 0.f;
    J[jslot(A, s1 * WF + s0, WF)] = acc;
  }
  __syncthreads();
}

// ------------------------------------------------------------------- GMRES --
// y = J (dinv .* v) (scaled) or y = J v, with FP32 products.  The FP32 operand goes to
// shared memory (c.zs; the global z32 when it does not fit).  Row A = (i0, i1) holds the
// columns (j0, j1), j1 in [l(i1), r(i1)] outer and j0 in [l(i0), r(i0)] inner, so the
// column indices follow from the 1D stencils and no index is loaded.  Every row runs the
// same unrolled (2P+1)^2 slots: the thread of row A is lane A % 32 of the warp that owns
// A's slice, so each slot is one coalesced load; a slot outside the row's stencil holds
// zero and reads a column of the row (clamped), so it adds nothing and the sum is the one
// over the row's own columns in their order.
template <int P>
__device__ void b_apply(const BInst &I, const double *__restrict__ v, double *__restrict__ y, bool scaled, const Cta &c) {
  constexpr int WF = 2 * P + 1;
  const BMesh &M = I.m;
  const int n = M.n, N = M.N;
  float *z = c.zs ? c.zs : I.z32;
  for (int r = c.tid; r < N; r += c.nt) z[r] = (float)(scaled ? I.dinv[r] * v[r] : v[r]);
  __syncthreads();
  for (int r = c.tid; r < N; r += c.nt) {
    const int i0 = r % n, i1 = r / n;
    const int l0 = M.l[i0], m0 = M.r[i0] - l0, l1 = M.l[i1], m1 = M.r[i1] - l1;
    const float *Jr = I.J + jslot(r, 0, WF);
    float acc = 0.f;
#pragma unroll
    for (int b = 0; b < WF; b++) {
      const float *zr = z + l0 + (int64_t)n * (l1 + min(b, m1));
#pragma unroll
      for (int a = 0; a < WF; a++) acc = fmaf(Jr[32 * (b * WF + a)], zr[min(a, m0)], acc);
    }
    y[r] = (double)acc;
  }
  __syncthreads();
}

struct GmShared {
  double H[BMAXM + 1][BMAXM];
  double part[BMAXM + 1][BDOT_MAX];  // chunk sums of the Gram-Schmidt dots
  double cs[BMAXM], sn[BMAXM], g[BMAXM + 1], y[BMAXM], h[BMAXM + 1];
  double scal[8];
  int flag[4];
};

// CGS pass: h_i = <V_i, w>, then w -= sum h_i V_i; adds h into H[:, j].  Work unit of
// the dots: (column i, row chunk) with R chunks of about N / R rows per column (R =
// c.dot_chunks, or as many as keep every warp busy when it is 0), one warp per unit; the
// chunk sums are added in chunk order, so the result depends on R but not on scheduling.
__device__ void b_cgs_pass(const BInst &I, double *__restrict__ w, int jp1, GmShared &s, int j, bool first, const Cta &c) {
  const int N = I.m.N;
  int R = c.dot_chunks > 0 ? c.dot_chunks : max(1, c.nw / jp1);
  R = min(R, BDOT_MAX);
  const int items = jp1 * R, clen = (N + R - 1) / R;
  for (int it = c.warp; it < items; it += c.nw) {
    const int i = it / R, ch = it - i * R;
    const int r0 = ch * clen, r1 = min(N, r0 + clen);
    const double *v = I.V + (size_t)i * N;
    double acc = 0.0;
    for (int r = r0 + c.lane; r < r1; r += 32) acc = fma(v[r], w[r], acc);
    acc = warp_sum(acc);
    if (c.lane == 0) s.part[i][ch] = acc;
  }
  __syncthreads();
  if (c.tid < jp1) {
    double h = s.part[c.tid][0];
    for (int ch = 1; ch < R; ch++) h += s.part[c.tid][ch];
    s.h[c.tid] = h;
  }
  __syncthreads();
  for (int r = c.tid; r < N; r += c.nt) {
    double acc = w[r];
    for (int i = 0; i < jp1; i++) acc = fma(-s.h[i], I.V[(size_t)i * N + r], acc);
    w[r] = acc;
  }
  if (c.tid < jp1) s.H[c.tid][j] = first ? s.h[c.tid] : s.H[c.tid][j] + s.h[c.tid];
  __syncthreads();
}

// returns 0 converged, 1 cap reached, 2 breakdown/NaN
template <int P>
__device__ int b_gmres(const BInst &I, const double *__restrict__ b, double *__restrict__ x, double tol, int m, int maxit,
                       int refine, GmShared &s, const Cta &c, int *its) {
  const BMesh &M = I.m;
  const int N = M.N;
  // Jacobi scaling from the diagonal
  for (int r = c.tid; r < N; r += c.nt) {
    const double d = (double)I.J[jslot(r, diag_slot(M, r, 2 * P + 1), 2 * P + 1)];
    I.dinv[r] = (d != 0.0) ? 1.0 / d : 1.0;
    x[r] = 0.0;
  }
  __syncthreads();
  int total = 0, rc = 1;
  bool first_cycle = true;
  while (total < maxit) {
    // r = b - A x  -> V[0]
    double *V0 = I.V;
    if (first_cycle) {
      for (int r = c.tid; r < N; r += c.nt) V0[r] = b[r];
      __syncthreads();
    } else {
      b_apply<P>(I, x, I.w, false, c);  // x is in the unpreconditioned space: apply J itself
      for (int r = c.tid; r < N; r += c.nt) V0[r] = b[r] - I.w[r];
      __syncthreads();
    }
    first_cycle = false;
    double ss = 0.0;
    for (int r = c.tid; r < N; r += c.nt) ss = fma(V0[r], V0[r], ss);
    ss = cta_sum(c, ss);
    if (c.tid == 0) {
      const double bt = sqrt(ss);
      c.red[35] = bt;
      c.red[36] = 1.0 / bt;
    }
    __syncthreads();
    const double beta = c.red[35], binv = c.red[36];
    if (!isfinite(beta)) { rc = 2; break; }
    if (beta <= tol) { rc = 0; break; }
    for (int r = c.tid; r < N; r += c.nt) V0[r] *= binv;
    if (c.tid == 0) {
      s.g[0] = beta;
      for (int i = 1; i <= m; i++) s.g[i] = 0.0;
    }
    __syncthreads();
    int k = 0;
    double res = beta;
    bool brk = false;
    for (int j = 0; j < m && total + j < maxit; j++) {
      double *w = I.w;
      b_apply<P>(I, I.V + (size_t)j * N, w, true, c);
      // classical Gram-Schmidt once, twice, or twice where the first pass removes more than
      // half of ||w||^2 (the modes of gmres_cgs_refine)
      double w0 = 0.0;
      if (refine == IGA_CGS_REFINE_IFNEEDED) {
        for (int r = c.tid; r < N; r += c.nt) w0 = fma(w[r], w[r], w0);
        w0 = cta_sum(c, w0);
      }
      b_cgs_pass(I, w, j + 1, s, j, true, c);
      bool twice = refine == IGA_CGS_REFINE_ALWAYS;
      if (refine == IGA_CGS_REFINE_IFNEEDED) {
        if (c.tid == 0) {
          double t = 0.0;
          for (int i = 0; i <= j; i++) t = fma(s.H[i][j], s.H[i][j], t);
          s.flag[1] = (w0 - t > 0.5 * w0) ? 0 : 1;
        }
        __syncthreads();
        twice = s.flag[1] != 0;
      }
      if (twice) b_cgs_pass(I, w, j + 1, s, j, false, c);
      double ww = 0.0;
      for (int r = c.tid; r < N; r += c.nt) ww = fma(w[r], w[r], ww);
      ww = cta_sum(c, ww);
      if (c.tid == 0) {
        // ||w||, its reciprocal and the Givens step by thread 0, shared after the barrier
        const double hn = sqrt(ww);
        s.scal[1] = hn;
        s.scal[2] = 1.0 / hn;
        s.H[j + 1][j] = hn;
        for (int i = 0; i < j; i++) {
          double a = s.H[i][j], bb = s.H[i + 1][j];
          s.H[i][j] = s.cs[i] * a + s.sn[i] * bb;
          s.H[i + 1][j] = -s.sn[i] * a + s.cs[i] * bb;
        }
        double a = s.H[j][j], bb = s.H[j + 1][j];
        double rr = hypot(a, bb);
        double cc = (rr > 0.0) ? a / rr : 1.0, sn = (rr > 0.0) ? bb / rr : 0.0;
        s.cs[j] = cc;
        s.sn[j] = sn;
        s.H[j][j] = rr;
        s.H[j + 1][j] = 0.0;
        double gj = s.g[j];
        s.g[j] = cc * gj;
        s.g[j + 1] = -sn * gj;
        s.scal[0] = fabs(s.g[j + 1]);
      }
      __syncthreads();
      res = s.scal[0];
      const double hn = s.scal[1];
      k = j + 1;
      if (!(hn > 1e-300) || !isfinite(res)) { brk = true; break; }
      if (res <= tol) break;
      double *vn = I.V + (size_t)(j + 1) * N;
      const double inv = s.scal[2];
      for (int r = c.tid; r < N; r += c.nt) vn[r] = w[r] * inv;
      __syncthreads();
    }
    // y = H^{-1} g (k x k upper triangular), x += dinv .* (V y)
    if (c.tid == 0) {
      for (int i = k - 1; i >= 0; i--) {
        double t = s.g[i];
        for (int q = i + 1; q < k; q++) t -= s.H[i][q] * s.y[q];
        s.y[i] = (s.H[i][i] != 0.0) ? t / s.H[i][i] : 0.0;
      }
    }
    __syncthreads();
    for (int r = c.tid; r < N; r += c.nt) {
      double acc = 0.0;
      for (int i = 0; i < k; i++) acc = fma(s.y[i], I.V[(size_t)i * N + r], acc);
      x[r] += I.dinv[r] * acc;
    }
    __syncthreads();
    total += k;
    if (brk) { rc = (res <= tol) ? 0 : 2; break; }
    if (res <= tol) { rc = 0; break; }
    if (k == 0) break;
  }
  *its = total;
  return rc;
}

// Jacobi-preconditioned conjugate gradients (the -ksp_type cg solve of App. B):
// FP64 vectors and reductions, FP32 operator products.  0 converged, 1 cap, 2 breakdown.
template <int P>
__device__ int b_cg(const BInst &I, const double *__restrict__ b, double *__restrict__ x, double tol, int maxit, const Cta &c,
                    int *its) {
  const BMesh &M = I.m;
  const int N = M.N;
  double *r = I.w;  // residual (the GMRES work vector; p and q use the first two basis slots)
  double *p = I.V, *q = I.V + N;
  for (int i = c.tid; i < N; i += c.nt) {
    const double d = (double)I.J[jslot(i, diag_slot(M, i, 2 * P + 1), 2 * P + 1)];
    I.dinv[i] = (d != 0.0) ? 1.0 / d : 1.0;
  }
  __syncthreads();
  double rz = 0.0, rr = 0.0;
  for (int i = c.tid; i < N; i += c.nt) {
    x[i] = 0.0;
    r[i] = b[i];
    p[i] = I.dinv[i] * b[i];
    rz = fma(b[i], p[i], rz);
    rr = fma(b[i], b[i], rr);
  }
  cta_sum2(c, rz, rr);
  int it = 0, rc = 1;
  if (!isfinite(rr)) rc = 2;
  else if (sqrt(rr) <= tol) rc = 0;
  while (rc == 1 && it < maxit) {
    b_apply<P>(I, p, q, false, c);
    double pq = 0.0;
    for (int i = c.tid; i < N; i += c.nt) pq = fma(p[i], q[i], pq);
    pq = cta_sum(c, pq);
    if (!(pq > 0.0) || !isfinite(pq)) { rc = 2; break; }
    // the iteration's scalars by thread 0, shared: a FP64 division or square root in every
    // thread would cost the SM's narrow FP64 pipe as much as a pass over a vector
    if (c.tid == 0) c.red[35] = rz / pq;
    __syncthreads();
    const double alpha = c.red[35];
    double rr2 = 0.0, rz2 = 0.0;
    for (int i = c.tid; i < N; i += c.nt) {
      x[i] = fma(alpha, p[i], x[i]);
      const double ri = fma(-alpha, q[i], r[i]);
      r[i] = ri;
      rr2 = fma(ri, ri, rr2);
      rz2 = fma(ri, I.dinv[i] * ri, rz2);
    }
    cta_sum2(c, rr2, rz2);
    it++;
    if (!isfinite(rr2)) { rc = 2; break; }
    if (c.tid == 0) {
      c.red[36] = sqrt(rr2) <= tol ? 1.0 : 0.0;
      c.red[37] = rz2 / rz;
    }
    __syncthreads();
    if (c.red[36] != 0.0) { rc = 0; break; }
    const double beta = c.red[37];
    rz = rz2;
    for (int i = c.tid; i < N; i += c.nt) p[i] = fma(beta, p[i], I.dinv[i] * r[i]);
    __syncthreads();
  }
  *its = it;
  return rc;
}

// ------------------------------------------------------------------ Newton --
template <int P>
__device__ void b_solve(const BInst &I, double *__restrict__ U, const iga_newton_opts &o, GmShared &s, BRep *rep, const Cta &c) {
  const int N = I.m.N;
  double *F = I.F, *dU = I.dU, *Ut = I.Ut, *Ft = I.Ft;
  b_residual<P>(I, U, F, c);
  double ss = 0.0;
  for (int r = c.tid; r < N; r += c.nt) ss = fma(F[r], F[r], ss);
  double fn = sqrt(cta_sum(c, ss));
  const double fn0 = fn;
  int k = 0, kry = 0, status = IGA_ENOCONV;
  const int m = o.gmres_restart < BMAXM ? o.gmres_restart : BMAXM;
  for (;;) {
    if (!isfinite(fn)) { status = IGA_ENAN; break; }
    if (fn <= o.atol) { status = IGA_OK; break; }
    if (k >= o.max_newton) { status = IGA_ENOCONV; break; }
    b_jacobian<P>(I, U, I.J, c);
    for (int r = c.tid; r < N; r += c.nt) Ft[r] = -F[r];
    __syncthreads();
    double rtol = o.krylov_rtol < fn ? o.krylov_rtol : fn;
    if (rtol < 1e-4) rtol = 1e-4;  // FP32 operator: no tighter than its own accuracy
    double tol = rtol * fn;
    if (tol < 0.5 * o.atol) tol = 0.5 * o.atol;
    int its = 0;
    if (o.ksp == IGA_KSP_CG) b_cg<P>(I, Ft, dU, tol, o.max_krylov, c, &its);
    else b_gmres<P>(I, Ft, dU, tol, m, o.max_krylov, o.gmres_cgs_refine, s, c, &its);
    kry += its;
    double alpha = 1.0, ft = 0.0;
    bool ok = false;
    for (int ls = 0; ls <= 10; ls++) {
      for (int r = c.tid; r < N; r += c.nt) Ut[r] = U[r] + alpha * dU[r];
      __syncthreads();
      b_residual<P>(I, Ut, Ft, c);
      double s2 = 0.0;
      for (int r = c.tid; r < N; r += c.nt) s2 = fma(Ft[r], Ft[r], s2);
      ft = sqrt(cta_sum(c, s2));
      if (isfinite(ft) && ft < fn) { ok = true; break; }
      alpha *= 0.5;
    }
    k++;
    if (!ok) { status = isfinite(ft) ? IGA_EDIVERGED : IGA_ENAN; break; }
    for (int r = c.tid; r < N; r += c.nt) {
      U[r] = Ut[r];
      F[r] = Ft[r];
    }
    __syncthreads();
    fn = ft;
  }
  if (c.tid == 0) {
    rep->newton_its = k;
    rep->krylov_its = kry;
    rep->status = status;
    rep->fnorm0 = fn0;
    rep->fnorm = fn;
  }
  __syncthreads();
}

constexpr int BZCAP_MAX = 40960;  // floats of dynamic shared memory at most (160 KB)

// Launch shapes: NT threads per CTA, register budget for MINB resident CTAs per SM
// (256 threads: 255 registers with MINB = 1, 128 with MINB = 2; 512: 128).  More
// threads per instance give the memory-bound Krylov phases more loads in flight at the
// price of register spills in the element kernels (at 1024 threads, 64 registers, the
// spills cost more than the extra loads gain).
template <int MINB, int NT>
__global__ void __launch_bounds__(NT, MINB) k_batch(const BInst *__restrict__ insts, const int *__restrict__ order, int count,
                                                const BArgs *__restrict__ args, int *__restrict__ counter, BRep *__restrict__ reps,
                                                int zcap) {
  extern __shared__ float zs_dyn[];  // [zcap]: the operand vector of instances with N <= zcap
  __shared__ double red[40];
  __shared__ GmShared s;
  __shared__ int cur;
  Cta c;
  c.tid = threadIdx.x;
  c.nt = blockDim.x;
  c.lane = threadIdx.x & 31;
  c.warp = threadIdx.x >> 5;
  c.nw = blockDim.x >> 5;
  c.red = red;
  c.zs = nullptr;
  c.tile = zs_dyn;
  c.tile_cap = zcap;
  c.dot_chunks = args->dot_chunks;
  c.jac_lines = args->jac_lines;
  const iga_newton_opts o = args->opts;
  for (;;) {
    if (c.tid == 0) cur = atomicAdd(counter, 1);
    __syncthreads();
    const int k = cur;
    __syncthreads();
    if (k >= count) return;
    const int idx = order[k];
    const BInst I = insts[idx];
    double *U = args->U + I.uoff;
    c.zs = I.m.N <= zcap ? zs_dyn : nullptr;
    if (c.tid == 0) reps[idx].t0 = gtimer();
    switch (I.m.p) {
      case 1: b_solve<1>(I, U, o, s, reps + idx, c); break;
      case 2: b_solve<2>(I, U, o, s, reps + idx, c); break;
      default: b_solve<3>(I, U, o, s, reps + idx, c); break;
    }
    if (c.tid == 0) reps[idx].t1 = gtimer();
  }
}

// kappa * jw and jw at every Gauss point of every instance; log kappa interpolated
// with the tensor-product basis (identity map, unit weights)
__global__ void k_batch_coeffs(const BInst *__restrict__ insts, int count, const int64_t *__restrict__ eoff,
                               const double *const *__restrict__ logk, double *__restrict__ ck_all, double *__restrict__ cr_all,
                               float *__restrict__ ck32_all, float *__restrict__ cr32_all, int64_t total_qp) {
  int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= total_qp) return;
  // find the instance: eoff holds the first Gauss-point index of each instance (ascending)
  int lo = 0, hi = count - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (eoff[mid] <= t) lo = mid; else hi = mid - 1;
  }
  const BInst &I = insts[lo];
  const BMesh &M = I.m;
  const int Q = M.q, N1 = M.p + 1, NQ = Q * Q;
  const int64_t local = t - eoff[lo];
  const int e = (int)(local / NQ), qp = (int)(local % NQ);
  const int e0 = e % M.nel, e1 = e / M.nel, g0 = qp % Q, g1 = qp / Q;
  const double jw = M.wq[e0 * Q + g0] * M.wq[e1 * Q + g1];
  double kappa = 1.0;
  if (logk[lo]) {
    const double *B0 = M.tab + ((size_t)e0 * Q + g0) * N1 * 2, *B1 = M.tab + ((size_t)e1 * Q + g1) * N1 * 2;
    double L = 0.0;
    for (int a1 = 0; a1 < N1; a1++)
      for (int a0 = 0; a0 < N1; a0++)
        L += B0[a0 * 2] * B1[a1 * 2] * logk[lo][(M.first[e0] + a0) + (size_t)M.n * (M.first[e1] + a1)];
    kappa = exp(L);
  }
  ck_all[t] = kappa * jw;
  cr_all[t] = jw;
  // the FP32 kappa jw of the Jacobian's line tiles: line-major [x1][x0], x = e q + g
  const int X = M.nel * Q;
  ck32_all[eoff[lo] + (int64_t)(e1 * Q + g1) * X + e0 * Q + g0] = (float)(kappa * jw);
  cr32_all[t] = (float)jw;
}

}  // namespace

// ------------------------------------------------------------------- host ---
struct MeshHost {
  std::vector<void *> bufs;
  BMesh dev;
};

struct iga_batch_s {
  int count = 0;
  cudaStream_t stream = nullptr;   // internal, non-blocking (graph capture needs a non-default stream)
  std::vector<MeshHost> meshes;
  std::vector<void *> bufs;        // arenas
  BInst *d_insts = nullptr;
  int *d_order = nullptr, *d_counter = nullptr;
  BArgs *d_args = nullptr, *h_args = nullptr;  // pinned host mirror
  BRep *d_reps = nullptr, *h_reps = nullptr;
  std::vector<int64_t> uoff;       // count + 1
  int threads = 512, ctas_per_sm = 1, nsm = 0;
  int dot_chunks = 1;              // work unit of the Gram-Schmidt dots (iga_batch_set_tiles)
  int jac_lines = 4;               // Gauss lines per stage-1 tile of the Jacobian (iga_batch_set_tiles)
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  int graph_threads = 0, graph_ctas = 0;
  int zcap = 0;                    // floats of dynamic shared memory for the operand vector
  std::string err;
  int mmax = 0;
};

static void batch_release(iga_batch_s *b) {
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  for (auto &m : b->meshes)
    for (void *p : m.bufs) cudaFree(p);
  for (void *p : b->bufs) cudaFree(p);
  if (b->h_args) cudaFreeHost(b->h_args);
  if (b->h_reps) cudaFreeHost(b->h_reps);
  if (b->stream) cudaStreamDestroy(b->stream);
}

#define BCK(call)                                                            \
  do {                                                                       \
    cudaError_t ce_ = (call);                                                \
    if (ce_ != cudaSuccess) {                                                \
      b->err = iga_format("%s: %s", #call, cudaGetErrorString(ce_));         \
      return ce_ == cudaErrorMemoryAllocation ? IGA_ENOMEM : IGA_ECUDA;      \
    }                                                                        \
  } while (0)

template <typename T>
static cudaError_t upload_v(std::vector<void *> &keep, const T **dst, const std::vector<T> &src) {
  T *p = nullptr;
  size_t n = src.empty() ? 1 : src.size();
  cudaError_t ce = cudaMalloc((void **)&p, n * sizeof(T));
  if (ce) return ce;
  keep.push_back(p);
  if (!src.empty()) ce = cudaMemcpy(p, src.data(), src.size() * sizeof(T), cudaMemcpyHostToDevice);
  *dst = p;
  return ce;
}

static thread_local std::string g_batch_err;

static iga_status build_mesh(iga_batch_s *b, const iga_desc *d, MeshHost &mh) {
  iga_s tmp;
  iga_status st = iga_build_dirs(&tmp, d);
  if (st != IGA_OK) {
    b->err = tmp.err;
    return st;
  }
  const Dir &D = tmp.dir[0];
  if (tmp.dir[1].knots != D.knots) {
    b->err = "batched instances must use the same knot vector in both directions";
    return IGA_EINVAL;
  }
  std::vector<int64_t> rowptr;
  iga_rowptr(&tmp, rowptr);
  BMesh &M = mh.dev;
  M.p = D.p; M.q = D.q; M.nel = D.nel; M.n = D.n; M.np = D.npairs(); M.N = (int)tmp.N; M.nnz = rowptr.back();
  std::vector<float> pv(D.pair_val.begin(), D.pair_val.end());
  cudaError_t ce;
  if ((ce = upload_v(mh.bufs, &M.tab, D.tab)) || (ce = upload_v(mh.bufs, &M.wq, D.wq)) ||
      (ce = upload_v(mh.bufs, &M.first, D.first)) || (ce = upload_v(mh.bufs, &M.node_e0, D.node_e0)) ||
      (ce = upload_v(mh.bufs, &M.node_ne, D.node_ne)) || (ce = upload_v(mh.bufs, &M.l, D.l)) ||
      (ce = upload_v(mh.bufs, &M.r, D.r)) || (ce = upload_v(mh.bufs, &M.pair_off, D.pair_off)) ||
      (ce = upload_v(mh.bufs, &M.pair_i, D.pair_i)) || (ce = upload_v(mh.bufs, &M.pair_x0, D.pair_x0)) ||
      (ce = upload_v(mh.bufs, &M.pair_np, D.pair_np)) || (ce = upload_v(mh.bufs, &M.pair_po, D.pair_po)) ||
      (ce = upload_v(mh.bufs, &M.pair_val, pv))) {
    b->err = iga_format("mesh upload: %s", cudaGetErrorString(ce));
    return ce == cudaErrorMemoryAllocation ? IGA_ENOMEM : IGA_ECUDA;
  }
  return IGA_OK;
}

static iga_status batch_create_impl(iga_batch_s *b, int count, const iga_desc *descs, const iga_bratu *params, void *stream) {
  (void)stream;
  b->count = count;
  b->mmax = BMAXM;
  BCK(cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking));
  int dev = 0;
  BCK(cudaGetDevice(&dev));
  BCK(cudaDeviceGetAttribute(&b->nsm, cudaDevAttrMultiProcessorCount, dev));
  // meshes, shared by instances with identical descriptions
  std::map<std::vector<double>, int> mesh_of;
  std::vector<int> mi(count);
  for (int i = 0; i < count; i++) {
    const iga_desc &d = descs[i];
    if (d.dim != 2 || d.ctrl || d.weights || d.degree[0] != d.degree[1] || d.degree[0] < 1 || d.degree[0] > 3 ||
        d.periodic[0] || d.periodic[1]) {
      b->err = iga_format("instance %d: batched instances are 2D, identity map, unit weights, p = 1..3, not periodic", i);
      return IGA_EINVAL;
    }
    if (!isfinite(params[i].lambda)) {
      b->err = iga_format("instance %d: lambda must be finite", i);
      return IGA_EINVAL;
    }
    std::vector<double> key = {(double)d.degree[0], (double)d.nel[0], (double)d.nel[1], (double)d.continuity[0],
                               (double)d.continuity[1], (double)d.quad[0], (double)d.quad[1]};
    for (int ax = 0; ax < 2; ax++) {
      key.push_back(d.knots[ax] ? (double)d.nknots[ax] : -1.0);
      if (d.knots[ax]) key.insert(key.end(), d.knots[ax], d.knots[ax] + d.nknots[ax]);
    }
    auto it = mesh_of.find(key);
    if (it == mesh_of.end()) {
      MeshHost mh;
      iga_status st = build_mesh(b, &d, mh);
      if (st != IGA_OK) {
        for (void *p : mh.bufs) cudaFree(p);
        b->err = iga_format("instance %d: %s", i, b->err.c_str());
        return st;
      }
      b->meshes.push_back(mh);
      it = mesh_of.emplace(key, (int)b->meshes.size() - 1).first;
    }
    mi[i] = it->second;
  }
  // sizes and arenas
  b->uoff.assign(count + 1, 0);
  int64_t dbl = 0, flt = 0, qp_total = 0;
  std::vector<int64_t> qpoff(count + 1, 0);
  for (int i = 0; i < count; i++) {
    const BMesh &M = b->meshes[mi[i]].dev;
    int64_t nelem = (int64_t)M.nel * M.nel, nq = (int64_t)M.q * M.q, nen = (int64_t)(M.p + 1) * (M.p + 1);
    // one Gauss line of Q00 and one of kappa jw must fit the shared-memory tile
    if (2 * (int64_t)M.nel * M.q > BZCAP_MAX) {
      b->err = iga_format("instance %d: %d elements per direction exceed the batched solver's line tile", i, M.nel);
      return IGA_EINVAL;
    }
    b->uoff[i + 1] = b->uoff[i] + M.N;
    b->zcap = std::max(b->zcap, M.N);
    dbl += 6 * (int64_t)M.N + (int64_t)(b->mmax + 1) * M.N + nelem * nen + 2 * nelem * nq + 8;
    flt += jsize(M.N, M.p) + 32 + 2 * (int64_t)M.nel * M.q * (2 * M.p + 1) * M.n + nelem * nq + M.N + 2 * nelem * nq + 8;
    qpoff[i + 1] = qpoff[i] + nelem * nq;
  }
  qp_total = qpoff[count];
  // the operand vector of the operator products lives in shared memory (up to 160 KB)
  b->zcap = std::min(b->zcap, BZCAP_MAX);
  for (auto kern : {k_batch<1, 256>, k_batch<2, 256>, k_batch<1, 512>})
    BCK(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)(b->zcap * sizeof(float))));
  double *dar = nullptr;
  float *far = nullptr;
  BCK(cudaMalloc((void **)&dar, dbl * sizeof(double)));
  b->bufs.push_back(dar);
  BCK(cudaMalloc((void **)&far, flt * sizeof(float)));
  b->bufs.push_back(far);
  BCK(cudaMemset(far, 0, flt * sizeof(float)));  // the Jacobian slots outside the stencils stay zero
  std::vector<BInst> insts(count);
  double *dp = dar;
  float *fp = far;
  double *ck_all = nullptr, *cr_all = nullptr;
  float *ck32_all = nullptr, *cr32_all = nullptr;
  // coefficient arrays are contiguous across instances (one set-up launch fills them)
  for (int i = 0; i < count; i++) {
    BInst &I = insts[i];
    I.m = b->meshes[mi[i]].dev;
    const BMesh &M = I.m;
    int64_t nelem = (int64_t)M.nel * M.nel, nq = (int64_t)M.q * M.q, nen = (int64_t)(M.p + 1) * (M.p + 1);
    I.lambda = params[i].lambda;
    I.uoff = b->uoff[i];
    I.F = dp; dp += M.N;
    I.dU = dp; dp += M.N;
    I.Ut = dp; dp += M.N;
    I.Ft = dp; dp += M.N;
    I.dinv = dp; dp += M.N;
    I.w = dp; dp += M.N;
    I.V = dp; dp += (int64_t)(b->mmax + 1) * M.N;
    I.Fe = dp; dp += nelem * nen;
    fp = far + ((fp - far + 31) / 32) * 32;  // slices start on 128 bytes
    I.J = fp; fp += jsize(M.N, M.p);
    I.T1 = fp; fp += 2 * (int64_t)M.nel * M.q * (2 * M.p + 1) * M.n;
    I.q00 = fp; fp += nelem * nq;
    I.z32 = fp; fp += M.N;
  }
  ck_all = dp; dp += qp_total;
  cr_all = dp; dp += qp_total;
  ck32_all = fp; fp += qp_total;
  cr32_all = fp; fp += qp_total;
  for (int i = 0; i < count; i++) {
    insts[i].ck = ck_all + qpoff[i];
    insts[i].cr = cr_all + qpoff[i];
    insts[i].ck32 = ck32_all + qpoff[i];
    insts[i].cr32 = cr32_all + qpoff[i];
  }
  BCK(cudaMalloc((void **)&b->d_insts, count * sizeof(BInst)));
  b->bufs.push_back(b->d_insts);
  BCK(cudaMemcpy(b->d_insts, insts.data(), count * sizeof(BInst), cudaMemcpyHostToDevice));
  // log kappa fields
  std::vector<const double *> lk_ptrs(count, nullptr);
  int64_t lk_total = 0;
  for (int i = 0; i < count; i++)
    if (params[i].log_kappa) lk_total += insts[i].m.N;
  double *lk = nullptr;
  if (lk_total) {
    BCK(cudaMalloc((void **)&lk, lk_total * sizeof(double)));
    b->bufs.push_back(lk);
    int64_t o = 0;
    for (int i = 0; i < count; i++)
      if (params[i].log_kappa) {
        for (int64_t A = 0; A < insts[i].m.N; A++)
          if (!isfinite(params[i].log_kappa[A])) {
            b->err = iga_format("instance %d: log-kappa must be finite", i);
            return IGA_EINVAL;
          }
        BCK(cudaMemcpy(lk + o, params[i].log_kappa, insts[i].m.N * sizeof(double), cudaMemcpyHostToDevice));
        lk_ptrs[i] = lk + o;
        o += insts[i].m.N;
      }
  }
  const double **d_lk = nullptr;
  int64_t *d_qpoff = nullptr;
  BCK(cudaMalloc((void **)&d_lk, count * sizeof(double *)));
  b->bufs.push_back(d_lk);
  BCK(cudaMemcpy(d_lk, lk_ptrs.data(), count * sizeof(double *), cudaMemcpyHostToDevice));
  BCK(cudaMalloc((void **)&d_qpoff, (count + 1) * sizeof(int64_t)));
  b->bufs.push_back(d_qpoff);
  BCK(cudaMemcpy(d_qpoff, qpoff.data(), (count + 1) * sizeof(int64_t), cudaMemcpyHostToDevice));
  k_batch_coeffs<<<(unsigned)((qp_total + 255) / 256), 256, 0, b->stream>>>(b->d_insts, count, d_qpoff, d_lk, ck_all, cr_all,
                                                                          ck32_all, cr32_all, qp_total);
  BCK(cudaGetLastError());
  // largest instances first (their solves are the longest)
  std::vector<int> order(count);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int a, int c) {
    const BMesh &A = insts[a].m, &C = insts[c].m;
    return (double)A.nnz * A.n > (double)C.nnz * C.n;
  });
  BCK(cudaMalloc((void **)&b->d_order, count * sizeof(int)));
  b->bufs.push_back(b->d_order);
  BCK(cudaMemcpy(b->d_order, order.data(), count * sizeof(int), cudaMemcpyHostToDevice));
  BCK(cudaMalloc((void **)&b->d_counter, sizeof(int)));
  b->bufs.push_back(b->d_counter);
  BCK(cudaMalloc((void **)&b->d_args, sizeof(BArgs)));
  b->bufs.push_back(b->d_args);
  BCK(cudaMalloc((void **)&b->d_reps, count * sizeof(BRep)));
  b->bufs.push_back(b->d_reps);
  BCK(cudaMallocHost((void **)&b->h_args, sizeof(BArgs)));
  BCK(cudaMallocHost((void **)&b->h_reps, count * sizeof(BRep)));
  BCK(cudaStreamSynchronize(b->stream));
  return IGA_OK;
}

extern "C" iga_status iga_batch_create(int count, const iga_desc *descs, const iga_bratu *params, void *stream,
                                       iga_batch_t *out) {
  if (!out) return IGA_EINVAL;
  *out = nullptr;
  if (count < 1 || !descs || !params) {
    g_batch_err = "count must be positive and descs/params non-NULL";
    return IGA_EINVAL;
  }
  iga_batch_s *b = new iga_batch_s();
  iga_status st = batch_create_impl(b, count, descs, params, stream);
  if (st != IGA_OK) {
    g_batch_err = b->err;
    batch_release(b);
    delete b;
    return st;
  }
  *out = b;
  return IGA_OK;
}

extern "C" iga_status iga_batch_offsets(iga_batch_t b, int64_t *offsets) {
  if (!b || !offsets) return IGA_EINVAL;
  for (int i = 0; i <= b->count; i++) offsets[i] = b->uoff[i];
  return IGA_OK;
}

extern "C" iga_status iga_batch_set_launch(iga_batch_t b, int ctas_per_sm, int threads_per_cta) {
  if (!b) return IGA_EINVAL;
  if ((threads_per_cta != 256 && threads_per_cta != 512) || ctas_per_sm < 1 || ctas_per_sm * threads_per_cta > 2048) {
    b->err = "threads_per_cta must be 256 or 512 and ctas_per_sm * threads_per_cta at most 2048";
    return IGA_EINVAL;
  }
  b->ctas_per_sm = ctas_per_sm;
  b->threads = threads_per_cta;
  return IGA_OK;
}

extern "C" iga_status iga_batch_set_tiles(iga_batch_t b, int dot_chunks, int jac_lines) {
  if (!b) return IGA_EINVAL;
  if (dot_chunks < 0 || dot_chunks > BDOT_MAX) {
    b->err = iga_format("dot_chunks must be in 0..%d", BDOT_MAX);
    return IGA_EINVAL;
  }
  if (jac_lines != 1 && jac_lines != 2 && jac_lines != 4 && jac_lines != 8) {
    b->err = "jac_lines must be 1, 2, 4 or 8";
    return IGA_EINVAL;
  }
  b->dot_chunks = dot_chunks;
  b->jac_lines = jac_lines;
  return IGA_OK;
}

static cudaError_t batch_enqueue(iga_batch_s *b) {
  cudaMemcpyAsync(b->d_args, b->h_args, sizeof(BArgs), cudaMemcpyHostToDevice, b->stream);
  cudaMemsetAsync(b->d_counter, 0, sizeof(int), b->stream);
  int grid = b->nsm * b->ctas_per_sm;
  const size_t zb = (size_t)b->zcap * sizeof(float);
  auto kern = k_batch<1, 512>;
  if (b->threads == 256) kern = b->ctas_per_sm == 1 ? k_batch<1, 256> : k_batch<2, 256>;
  kern<<<grid, b->threads, zb, b->stream>>>(b->d_insts, b->d_order, b->count, b->d_args, b->d_counter, b->d_reps, b->zcap);
  cudaMemcpyAsync(b->h_reps, b->d_reps, b->count * sizeof(BRep), cudaMemcpyDeviceToHost, b->stream);
  return cudaGetLastError();
}

extern "C" iga_status iga_batch_solve(iga_batch_t b, double *U, const iga_newton_opts *opts_in, iga_batch_report *rep) {
  if (!b) return IGA_EINVAL;
  iga_newton_opts o;
  iga_newton_defaults(&o);
  if (opts_in) o = *opts_in;
  if (!U || o.gmres_restart < 1 || o.max_newton < 0 || !(o.atol >= 0.0) || o.gmres_cgs_refine < IGA_CGS_REFINE_NEVER ||
      o.gmres_cgs_refine > IGA_CGS_REFINE_ALWAYS) {
    b->err = "bad options or NULL U";
    return IGA_EINVAL;
  }
  if (o.gmres_restart > BMAXM) o.gmres_restart = BMAXM;
  b->h_args->U = U;
  b->h_args->opts = o;
  b->h_args->dot_chunks = b->dot_chunks;  // read by the graph's argument copy at every replay
  b->h_args->jac_lines = b->jac_lines;
  // the caller's pending work (any stream) completes before the solve reads U
  BCK(cudaDeviceSynchronize());
  if (!b->exec || b->graph_threads != b->threads || b->graph_ctas != b->ctas_per_sm) {
    if (b->exec) { cudaGraphExecDestroy(b->exec); b->exec = nullptr; }
    if (b->graph) { cudaGraphDestroy(b->graph); b->graph = nullptr; }
    BCK(cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal));
    cudaError_t ce = batch_enqueue(b);
    cudaError_t ce2 = cudaStreamEndCapture(b->stream, &b->graph);
    BCK(ce);
    BCK(ce2);
    BCK(cudaGraphInstantiate(&b->exec, b->graph, 0));
    b->graph_threads = b->threads;
    b->graph_ctas = b->ctas_per_sm;
  }
  BCK(cudaGraphLaunch(b->exec, b->stream));
  BCK(cudaStreamSynchronize(b->stream));
  int solved = 0;
  for (int i = 0; i < b->count; i++) solved += (b->h_reps[i].status == IGA_OK);
  if (rep) {
    rep->solved = solved;
    for (int i = 0; i < b->count; i++) {
      if (rep->newton_its) rep->newton_its[i] = b->h_reps[i].newton_its;
      if (rep->krylov_its) rep->krylov_its[i] = b->h_reps[i].krylov_its;
      if (rep->fnorm) rep->fnorm[i] = b->h_reps[i].fnorm;
      if (rep->status) rep->status[i] = b->h_reps[i].status;
      if (rep->solve_us) rep->solve_us[i] = 1e-3 * (double)(b->h_reps[i].t1 - b->h_reps[i].t0);
    }
  }
  if (solved != b->count) {
    b->err = iga_format("%d of %d instances did not reach the tolerance", b->count - solved, b->count);
    return IGA_ENOCONV;
  }
  return IGA_OK;
}

extern "C" void iga_batch_destroy(iga_batch_t b) {
  if (!b) return;
  if (b->stream) cudaStreamSynchronize(b->stream);
  batch_release(b);
  delete b;
}

extern "C" const char *iga_batch_last_error(iga_batch_t b) { return b ? b->err.c_str() : g_batch_err.c_str(); }
