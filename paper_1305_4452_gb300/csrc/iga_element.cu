// Element-level kernels of libiga for sm_103a: geometry factors, residual, Q00.
//
// Residual (Sec. 2.7 Algorithm 3 with Eq. residual): one fused kernel per
// element tile -- gather U_e, sum-factorised interpolation of u~ and grad u~ to
// the Gauss points, the Bratu integrand with the cached geometry factors, and
// the transposed sum-factorised test-function contraction -- writes F_e; a
// gather kernel adds the element vectors of each control variable in a fixed
// order (no atomics) and applies the Dirichlet rows.
//
// The Gauss-point field Q00 for the Jacobian (u~ interpolated to the Gauss points)
// is formed here too; the Jacobian stages live in iga_jacobian.cu.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <algorithm>

#include "iga_exp.h"
#include "iga_internal.h"
#include "iga_interp.h"

DirArgs dir_args(const DirDev &d) {
  DirArgs a;
  a.p = d.p; a.q = d.q; a.nel = d.nel; a.n = d.n; a.np = d.np; a.X = d.X;
  a.first = d.first; a.tab = d.tab; a.wq = d.wq; a.l = d.l; a.r = d.r;
  a.pair_off = d.pair_off; a.pair_i = d.pair_i; a.pair_j = d.pair_j;
  a.pair_x0 = d.pair_x0; a.pair_np = d.pair_np; a.pair_po = d.pair_po; a.pair_T = d.pair_T;
  a.nc = d.nc; a.pair_c = d.pair_c; a.pair_cs = d.pair_cs;
  a.pair_val = d.pair_val; a.pair_val_f = d.pair_val_f;
  a.node_e0 = d.node_e0; a.node_ne = d.node_ne;
  return a;
}

template <int DIM> __host__ __device__ constexpr int ipow(int b) { return DIM == 2 ? b * b : b * b * b; }

// ---------------------------------------------------------------------------
// Geometry factors (Sec. 2.3 Eqs. 6-7, drational; Appendix A Eqs. identity,
// dspatial).  Run once per iga_create.
//
// The rational map and its derivatives at a Gauss point are sums over the element's
// (p+1)^DIM functions of w_a, w_a X_a (and w_a log kappa_a) times the tensor products of
// the 1D values and first derivatives.  They are formed by sum factorisation, one axis
// at a time, for NE elements per CTA in shared memory:
//   axis 0:  S1[f][a2][a1][g0] = sum_a0 B0(g0, a0) C[f][a], and with B0' (2 results)
//   axis 1:  from S1: B1 * S1_B, B1' * S1_B, B1 * S1_B'               (3 results)
//   axis 2 (per point): V = B2 * S2_BB, D2 = B2' * S2_BB, D1 = B2 * S2_B'B, D0 = B2 * S2_BB'
// (2D stops after axis 0 and contracts axis 1 per point) -- about 36 FMAs per field and
// point at p = 3 instead of 30 per function and point; then geometry_point forms
// F = dx/dxi (Eq. drational), its inverse and determinant and the cached factors.
// ---------------------------------------------------------------------------
template <int DIM>
__device__ __forceinline__ void geometry_point(const double *V, const double (*D)[3], bool has_ctrl, bool has_logk, double wq,
                                               GeomLayout gl, double *rec, int NQ, int *__restrict__ err) {
  // V[0] = W, V[1..DIM] = sum w X_i, V[DIM+1] = sum w log kappa; D[f][al] their derivatives
  const double W = V[0];
  const double invW = 1.0 / W;
  double F[3][3];
  for (int i = 0; i < DIM; i++)
    for (int al = 0; al < DIM; al++)
      F[i][al] = has_ctrl ? (D[1 + i][al] - V[1 + i] * invW * D[0][al]) * invW : (i == al ? 1.0 : 0.0);
  double det, X[3][3];  // X[alpha][i] = xi_{alpha,i}
  if (DIM == 2) {
    det = F[0][0] * F[1][1] - F[0][1] * F[1][0];
    double id = 1.0 / det;
    X[0][0] = F[1][1] * id; X[0][1] = -F[0][1] * id;
    X[1][0] = -F[1][0] * id; X[1][1] = F[0][0] * id;
  } else {
    double c00 = F[1][1] * F[2][2] - F[1][2] * F[2][1];
    double c01 = F[1][2] * F[2][0] - F[1][0] * F[2][2];
    double c02 = F[1][0] * F[2][1] - F[1][1] * F[2][0];
    det = F[0][0] * c00 + F[0][1] * c01 + F[0][2] * c02;
    double id = 1.0 / det;
    X[0][0] = c00 * id; X[1][0] = c01 * id; X[2][0] = c02 * id;
    X[0][1] = (F[0][2] * F[2][1] - F[0][1] * F[2][2]) * id;
    X[1][1] = (F[0][0] * F[2][2] - F[0][2] * F[2][0]) * id;
    X[2][1] = (F[0][1] * F[2][0] - F[0][0] * F[2][1]) * id;
    X[0][2] = (F[0][1] * F[1][2] - F[0][2] * F[1][1]) * id;
    X[1][2] = (F[0][2] * F[1][0] - F[0][0] * F[1][2]) * id;
    X[2][2] = (F[0][0] * F[1][1] - F[0][1] * F[1][0]) * id;
  }
  if (!(det > 0.0)) atomicExch(err, 1);  // inverted or degenerate geometry (status only)
  double jw = det * wq;
  double kappa = has_logk ? exp(V[DIM + 1] * invW) : 1.0;
  double g[3] = {D[0][0] * invW, D[0][1] * invW, DIM == 3 ? D[0][2] * invW : 0.0};
  double S[3][3];
  double sc = kappa * jw * invW * invW;
  for (int al = 0; al < DIM; al++)
    for (int be = 0; be < DIM; be++) {
      double c = 0.0;
      for (int i = 0; i < DIM; i++) c += X[al][i] * X[be][i];
      S[al][be] = sc * c;
    }
  rec[gl.invW * NQ] = invW;
  for (int al = 0; al < DIM; al++) rec[(gl.g + al) * NQ] = g[al];
  if (DIM == 2) {
    rec[(gl.S + 0) * NQ] = S[0][0]; rec[(gl.S + 1) * NQ] = S[1][1]; rec[(gl.S + 2) * NQ] = S[0][1];
  } else {
    rec[(gl.S + 0) * NQ] = S[0][0]; rec[(gl.S + 1) * NQ] = S[1][1]; rec[(gl.S + 2) * NQ] = S[2][2];
    rec[(gl.S + 3) * NQ] = S[0][1]; rec[(gl.S + 4) * NQ] = S[0][2]; rec[(gl.S + 5) * NQ] = S[1][2];
  }
  rec[gl.jwW * NQ] = jw * invW;
  double gSg = 0.0;
  for (int al = 0; al < DIM; al++) {
    double sg = 0.0;
    for (int be = 0; be < DIM; be++) sg += S[al][be] * g[be];
    rec[(gl.Sg + al) * NQ] = -sg;  // stored negated: it enters the Jacobian as Q_0a = -(S g)_a
    gSg += g[al] * sg;
  }
  rec[gl.gSg * NQ] = gSg;
  rec[gl.jwW2 * NQ] = jw * invW * invW;
}

template <int DIM, int P> struct GeoSmem {
  static constexpr int N1 = P + 1, Q = P + 1;
  static constexpr int NEN = ipow<DIM>(N1), NQ = ipow<DIM>(Q);
  static constexpr int NF = DIM + 2;  // w, w X_i, w log kappa
  static constexpr int NE = NQ >= 128 ? 1 : 128 / NQ;
  static constexpr int TAB = DIM * Q * N1 * 2;
  static constexpr int C = NF * NEN;
  static constexpr int S1 = NF * ipow<DIM>(N1) / N1 * Q * 2;               // [f][a2][a1][g0][2] (2D: [f][a1][g0][2])
  static constexpr int S2 = DIM == 3 ? NF * N1 * Q * Q * 3 : 0;           // [f][a2][g1][g0][3]
  static constexpr int PER = TAB + C + S1 + S2;
};

template <int DIM, int P>
__global__ void __launch_bounds__(128) k_geometry(DirArgs d0, DirArgs d1, DirArgs d2, const double *__restrict__ ctrl,
                                                  const double *__restrict__ wts, const double *__restrict__ logk,
                                                  GeomLayout gl, double *__restrict__ geom, int64_t nelem,
                                                  int *__restrict__ err) {
  using SM = GeoSmem<DIM, P>;
  constexpr int N1 = SM::N1, Q = SM::Q, NQ = SM::NQ, NEN = SM::NEN, NF = SM::NF, NE = SM::NE;
  extern __shared__ double gsm[];
  const int tid = threadIdx.x, nt = blockDim.x;
  const int64_t ebase = (int64_t)blockIdx.x * NE;
  const bool has_ctrl = ctrl != nullptr, has_logk = logk != nullptr;
  // tables and the weighted coefficients of the block's elements
  for (int idx = tid; idx < NE * (SM::TAB + SM::C); idx += nt) {
    const int le = idx / (SM::TAB + SM::C), k = idx % (SM::TAB + SM::C);
    const int64_t e = ebase + le;
    double *base = gsm + (size_t)le * SM::PER;
    if (e >= nelem) { base[k] = 0.0; continue; }
    const int e0 = (int)(e % d0.nel), e1 = (int)((e / d0.nel) % d1.nel), e2 = (DIM == 3) ? (int)(e / ((int64_t)d0.nel * d1.nel)) : 0;
    if (k < SM::TAB) {
      const int ax = k / (Q * N1 * 2), r = k % (Q * N1 * 2);
      const DirArgs &d = ax == 0 ? d0 : (ax == 1 ? d1 : d2);
      const int ee = ax == 0 ? e0 : (ax == 1 ? e1 : e2);
      base[k] = d.tab[(size_t)ee * Q * N1 * 2 + r];
    } else {
      const int f = (k - SM::TAB) / NEN, a = (k - SM::TAB) % NEN;
      const int a0 = a % N1, a1 = (a / N1) % N1, a2 = (DIM == 3) ? a / (N1 * N1) : 0;
      const int64_t G = (d0.first[e0] + a0) + (int64_t)d0.n * ((d1.first[e1] + a1) + (int64_t)d1.n * ((DIM == 3 ? d2.first[e2] : 0) + a2));
      const double w = wts ? wts[G] : 1.0;
      double x = 0.0;
      if (f == 0) x = w;
      else if (f <= DIM) x = has_ctrl ? w * ctrl[G * DIM + (f - 1)] : 0.0;
      else x = has_logk ? w * logk[G] : 0.0;
      base[k] = x;
    }
  }
  __syncthreads();
#define GTB(base, ax, g, a, dv) (base)[(((ax) * Q + (g)) * N1 + (a)) * 2 + (dv)]
  // axis 0: value and derivative of B0
  constexpr int L1 = SM::S1 / (NF * Q * 2);  // lines (a2, a1) (2D: a1)
  for (int idx = tid; idx < NE * NF * L1 * Q; idx += nt) {
    const int le = idx / (NF * L1 * Q), r = idx % (NF * L1 * Q);
    const int f = r / (L1 * Q), line = (r / Q) % L1, g0 = r % Q;
    double *base = gsm + (size_t)le * SM::PER;
    const double *C = base + SM::TAB + f * NEN + line * N1;
    double v = 0.0, dv = 0.0;
#pragma unroll
    for (int a0 = 0; a0 < N1; a0++) {
      v = fma(GTB(base, 0, g0, a0, 0), C[a0], v);
      dv = fma(GTB(base, 0, g0, a0, 1), C[a0], dv);
    }
    double *o = base + SM::TAB + SM::C + ((size_t)(f * L1 + line) * Q + g0) * 2;
    o[0] = v;
    o[1] = dv;
  }
  __syncthreads();
  if (DIM == 3) {
    // axis 1: (B1, S1_B), (B1', S1_B), (B1, S1_B')
    for (int idx = tid; idx < NE * NF * N1 * Q * Q; idx += nt) {
      const int le = idx / (NF * N1 * Q * Q), r = idx % (NF * N1 * Q * Q);
      const int f = r / (N1 * Q * Q), a2 = (r / (Q * Q)) % N1, g1 = (r / Q) % Q, g0 = r % Q;
      double *base = gsm + (size_t)le * SM::PER;
      const double *S1 = base + SM::TAB + SM::C + (size_t)f * L1 * Q * 2;
      double bb = 0.0, db = 0.0, bd = 0.0;
#pragma unroll
      for (int a1 = 0; a1 < N1; a1++) {
        const double *s = S1 + ((size_t)(a2 * N1 + a1) * Q + g0) * 2;
        const double b1 = GTB(base, 1, g1, a1, 0), d1v = GTB(base, 1, g1, a1, 1);
        bb = fma(b1, s[0], bb);
        db = fma(d1v, s[0], db);
        bd = fma(b1, s[1], bd);
      }
      double *o = base + SM::TAB + SM::C + SM::S1 + ((size_t)((f * N1 + a2) * Q + g1) * Q + g0) * 3;
      o[0] = bb;
      o[1] = db;
      o[2] = bd;
    }
    __syncthreads();
  }
  // the last axis per point, then the factors
  for (int idx = tid; idx < NE * NQ; idx += nt) {
    const int le = idx / NQ, qp = idx % NQ;
    const int64_t e = ebase + le;
    if (e >= nelem) continue;
    const double *base = gsm + (size_t)le * SM::PER;
    const int g0 = qp % Q, g1 = (qp / Q) % Q, g2 = (DIM == 3) ? qp / (Q * Q) : 0;
    double V[NF], D[NF][3];
    for (int f = 0; f < NF; f++) {
      double v = 0.0, dl = 0.0, dm = 0.0, dn = 0.0;
      if (DIM == 3) {
        const double *S2 = base + SM::TAB + SM::C + SM::S1;
#pragma unroll
        for (int a2 = 0; a2 < N1; a2++) {
          const double *s = S2 + ((size_t)((f * N1 + a2) * Q + g1) * Q + g0) * 3;
          const double b2 = GTB(base, 2, g2, a2, 0), d2v = GTB(base, 2, g2, a2, 1);
          v = fma(b2, s[0], v);    // B0 B1 B2
          dn = fma(d2v, s[0], dn); // B0 B1 B2'
          dm = fma(b2, s[1], dm);  // B0 B1' B2
          dl = fma(b2, s[2], dl);  // B0' B1 B2
        }
      } else {
        const double *S1 = base + SM::TAB + SM::C + (size_t)f * L1 * Q * 2;
#pragma unroll
        for (int a1 = 0; a1 < N1; a1++) {
          const double *s = S1 + ((size_t)a1 * Q + g0) * 2;
          const double b1 = GTB(base, 1, g1, a1, 0), d1v = GTB(base, 1, g1, a1, 1);
          v = fma(b1, s[0], v);
          dm = fma(d1v, s[0], dm);
          dl = fma(b1, s[1], dl);
        }
      }
      V[f] = v;
      D[f][0] = dl;
      D[f][1] = dm;
      D[f][2] = dn;
    }
#undef GTB
    const int e0 = (int)(e % d0.nel), e1 = (int)((e / d0.nel) % d1.nel), e2 = (DIM == 3) ? (int)(e / ((int64_t)d0.nel * d1.nel)) : 0;
    const double wq = d0.wq[(size_t)e0 * Q + g0] * d1.wq[(size_t)e1 * Q + g1] * ((DIM == 3) ? d2.wq[(size_t)e2 * Q + g2] : 1.0);
    geometry_point<DIM>(V, D, has_ctrl, has_logk, wq, gl, geom + (size_t)e * gl.nf * NQ + qp, NQ, err);
  }
}

// ---------------------------------------------------------------------------
// Residual element kernel.  NE elements per CTA; all stages in shared memory.
// ---------------------------------------------------------------------------
template <int DIM, int P>
struct ResSmem {
  static constexpr int N1 = P + 1, Q = P + 1;
  static constexpr int NEN = ipow<DIM>(N1), NQ = ipow<DIM>(Q);
  static constexpr int TAB = DIM * Q * N1 * 2;
  // per-element scratch: coefficients, two stage buffers of the largest size
  static constexpr int BUF = (DIM == 3) ? 4 * NQ : 4 * NQ;
  static constexpr int PER = TAB + NEN + 2 * BUF;
};

// LIN: the Jacobian applied to a direction instead (matrix-free Newton-Krylov):
// U holds the direction x, its Dirichlet entries read as zero (the columns the
// Dirichlet fix removes), and the reaction term becomes q00[e][qp] * ũ_x, q00 the
// reaction part of Q00 at the Newton iterate (-jw/W^2 lambda e^u): the derivative
// of -jw/W lambda e^u in direction x, with u = ũ / W.
template <int DIM, int P, int NE, bool LIN = false>
__global__ void __launch_bounds__(128) k_residual(DirArgs d0, DirArgs d1, DirArgs d2, const double *__restrict__ U,
                                                  const double *__restrict__ wts, const double *__restrict__ geom,
                                                  GeomLayout gl, double lambda, double *__restrict__ Fe, int64_t nelem,
                                                  const double *__restrict__ q00 = nullptr, BndArgs bnd = BndArgs{},
                                                  const double *__restrict__ done = nullptr) {
  using SM = ResSmem<DIM, P>;
  constexpr int N1 = SM::N1, Q = SM::Q, NEN = SM::NEN, NQ = SM::NQ;
  extern __shared__ double smem[];
  if (LIN && done && done[0] != 0.0) return;
  const int tid = threadIdx.x, nt = blockDim.x;
  const int64_t ebase = (int64_t)blockIdx.x * NE;
  // ---- load tables and gather w_A U_A (Algorithm 3: U_e <- U) ----
  for (int idx = tid; idx < NE * (SM::TAB + NEN); idx += nt) {
    int le = idx / (SM::TAB + NEN), k = idx % (SM::TAB + NEN);
    int64_t e = ebase + le;
    double *base = smem + (size_t)le * SM::PER;
    if (e >= nelem) { base[k] = 0.0; continue; }
    int e0 = (int)(e % d0.nel), e1 = (int)((e / d0.nel) % d1.nel), e2 = (DIM == 3) ? (int)(e / ((int64_t)d0.nel * d1.nel)) : 0;
    if (k < SM::TAB) {
      int ax = k / (Q * N1 * 2), r = k % (Q * N1 * 2);
      const DirArgs &d = ax == 0 ? d0 : (ax == 1 ? d1 : d2);
      int ee = ax == 0 ? e0 : (ax == 1 ? e1 : e2);
      base[k] = d.tab[(size_t)ee * Q * N1 * 2 + r];
    } else {
      int a = k - SM::TAB;
      int a0 = a % N1, a1 = (a / N1) % N1, a2 = (DIM == 3) ? a / (N1 * N1) : 0;
      const int j0 = d0.first[e0] + a0, j1 = d1.first[e1] + a1, j2 = (DIM == 3 ? d2.first[e2] : 0) + a2;
      int64_t G = j0 + (int64_t)d0.n * (j1 + (int64_t)d1.n * j2);
      double x = U[G];
      if (LIN) {
        const int jj[3] = {j0, j1, j2}, nn[3] = {d0.n, d1.n, d2.n};
        for (int ax = 0; ax < DIM; ax++)
          if ((bnd.flag[ax][0] && jj[ax] == 0) || (bnd.flag[ax][1] && jj[ax] == nn[ax] - 1)) x = 0.0;
      }
      base[k] = x * (wts ? wts[G] : 1.0);
    }
  }
  __syncthreads();
  // B(ax, g, a, s) from the element's tables
#define TB(base, ax, g, a, s) (base)[(((ax) * Q + (g)) * N1 + (a)) * 2 + (s)]
  if (DIM == 3) {
    // buffers: X = base + TAB + NEN (size 4*NQ), Y = X + BUF
    // S1: T_s[a2][a1][g0] (s = 0,1) -> X[s][a2][a1][g0]
    for (int idx = tid; idx < NE * 2 * N1 * N1 * Q; idx += nt) {
      int le = idx / (2 * N1 * N1 * Q), k = idx % (2 * N1 * N1 * Q);
      int s = k / (N1 * N1 * Q), r = k % (N1 * N1 * Q);
      int a2 = r / (N1 * Q), a1 = (r / Q) % N1, g0 = r % Q;
      double *base = smem + (size_t)le * SM::PER;
      const double *C = base + SM::TAB;
      double acc = 0.0;
#pragma unroll
      for (int a0 = 0; a0 < N1; a0++) acc = fma(TB(base, 0, g0, a0, s), C[(a2 * N1 + a1) * N1 + a0], acc);
      (base + SM::TAB + NEN)[k] = acc;
    }
    __syncthreads();
    // S2: V_{st}[a2][g1][g0] for (s,t) in {(0,0),(1,0),(0,1)} -> Y[c][a2][g1][g0]
    for (int idx = tid; idx < NE * 3 * N1 * Q * Q; idx += nt) {
      int le = idx / (3 * N1 * Q * Q), k = idx % (3 * N1 * Q * Q);
      int c = k / (N1 * Q * Q), r = k % (N1 * Q * Q);
      int a2 = r / (Q * Q), g1 = (r / Q) % Q, g0 = r % Q;
      int s = (c == 1), t = (c == 2);
      double *base = smem + (size_t)le * SM::PER;
      const double *X = base + SM::TAB + NEN;
      double acc = 0.0;
#pragma unroll
      for (int a1 = 0; a1 < N1; a1++) acc = fma(TB(base, 1, g1, a1, t), X[s * N1 * N1 * Q + (a2 * N1 + a1) * Q + g0], acc);
      (base + SM::TAB + NEN + SM::BUF)[k] = acc;
    }
    __syncthreads();
    // S3: u, d0, d1, d2 at [g2][g1][g0] -> X[k][qp]
    for (int idx = tid; idx < NE * 4 * NQ; idx += nt) {
      int le = idx / (4 * NQ), k = idx % (4 * NQ);
      int c = k / NQ, qp = k % NQ;
      int g2 = qp / (Q * Q), g1 = (qp / Q) % Q, g0 = qp % Q;
      int src = (c == 1) ? 1 : (c == 2 ? 2 : 0), t = (c == 3);
      double *base = smem + (size_t)le * SM::PER;
      const double *Y = base + SM::TAB + NEN + SM::BUF;
      double acc = 0.0;
#pragma unroll
      for (int a2 = 0; a2 < N1; a2++) acc = fma(TB(base, 2, g2, a2, t), Y[src * N1 * Q * Q + (a2 * Q + g1) * Q + g0], acc);
      (base + SM::TAB + NEN)[k] = acc;
    }
    __syncthreads();
  } else {
    // S1: T_s[a1][g0] -> Y[s][a1][g0]
    for (int idx = tid; idx < NE * 2 * N1 * Q; idx += nt) {
      int le = idx / (2 * N1 * Q), k = idx % (2 * N1 * Q);
      int s = k / (N1 * Q), r = k % (N1 * Q);
      int a1 = r / Q, g0 = r % Q;
      double *base = smem + (size_t)le * SM::PER;
      const double *C = base + SM::TAB;
      double acc = 0.0;
#pragma unroll
      for (int a0 = 0; a0 < N1; a0++) acc = fma(TB(base, 0, g0, a0, s), C[a1 * N1 + a0], acc);
      (base + SM::TAB + NEN + SM::BUF)[k] = acc;
    }
    __syncthreads();
    // S2: u, d0, d1 at [g1][g0] -> X[k][qp]
    for (int idx = tid; idx < NE * 3 * NQ; idx += nt) {
      int le = idx / (3 * NQ), k = idx % (3 * NQ);
      int c = k / NQ, qp = k % NQ;
      int g1 = qp / Q, g0 = qp % Q;
      int src = (c == 1), t = (c == 2);
      double *base = smem + (size_t)le * SM::PER;
      const double *Y = base + SM::TAB + NEN + SM::BUF;
      double acc = 0.0;
#pragma unroll
      for (int a1 = 0; a1 < N1; a1++) acc = fma(TB(base, 1, g1, a1, t), Y[src * N1 * Q + a1 * Q + g0], acc);
      (base + SM::TAB + NEN)[k] = acc;
    }
    __syncthreads();
  }
  // ---- pointwise Bratu integrand at each Gauss point (Eq. residual) ----
  for (int idx = tid; idx < NE * NQ; idx += nt) {
    int le = idx / NQ, qp = idx % NQ;
    int64_t e = ebase + le;
    double *base = smem + (size_t)le * SM::PER;
    double *X = base + SM::TAB + NEN;
    if (e >= nelem) {
      for (int c = 0; c <= DIM; c++) X[c * NQ + qp] = 0.0;
      continue;
    }
    const double *rec = geom + (size_t)e * gl.nf * NQ + qp;
    double ut = X[qp];
    double r[3];
    for (int a = 0; a < DIM; a++) r[a] = X[(1 + a) * NQ + qp] - ut * rec[(gl.g + a) * NQ];
    double v[3];
    if (DIM == 2) {
      double s00 = rec[(gl.S + 0) * NQ], s11 = rec[(gl.S + 1) * NQ], s01 = rec[(gl.S + 2) * NQ];
      v[0] = s00 * r[0] + s01 * r[1];
      v[1] = s01 * r[0] + s11 * r[1];
    } else {
      double s00 = rec[(gl.S + 0) * NQ], s11 = rec[(gl.S + 1) * NQ], s22 = rec[(gl.S + 2) * NQ];
      double s01 = rec[(gl.S + 3) * NQ], s02 = rec[(gl.S + 4) * NQ], s12 = rec[(gl.S + 5) * NQ];
      v[0] = s00 * r[0] + s01 * r[1] + s02 * r[2];
      v[1] = s01 * r[0] + s11 * r[1] + s12 * r[2];
      v[2] = s02 * r[0] + s12 * r[1] + s22 * r[2];
    }
    double s;
    if (LIN) {
      s = q00[(size_t)e * NQ + qp] * ut;
    } else {
      double u = ut * rec[gl.invW * NQ];
      s = -rec[gl.jwW * NQ] * lambda * iga_exp(u);
    }
    for (int a = 0; a < DIM; a++) s -= rec[(gl.g + a) * NQ] * v[a];
    X[qp] = s;
    for (int a = 0; a < DIM; a++) X[(1 + a) * NQ + qp] = v[a];
  }
  __syncthreads();
  if (DIM == 3) {
    // B3: Y00 = sum_g2 B2 s + B2' v2; Y10 = sum B2 v0; Y01 = sum B2 v1 -> Y[c][a2][g1][g0]
    for (int idx = tid; idx < NE * 3 * N1 * Q * Q; idx += nt) {
      int le = idx / (3 * N1 * Q * Q), k = idx % (3 * N1 * Q * Q);
      int c = k / (N1 * Q * Q), r = k % (N1 * Q * Q);
      int a2 = r / (Q * Q), g1 = (r / Q) % Q, g0 = r % Q;
      double *base = smem + (size_t)le * SM::PER;
      const double *X = base + SM::TAB + NEN;
      double acc = 0.0;
      int src = (c == 0) ? 0 : (c == 1 ? 1 : 2);
#pragma unroll
      for (int g2 = 0; g2 < Q; g2++) {
        int qp = (g2 * Q + g1) * Q + g0;
        acc = fma(TB(base, 2, g2, a2, 0), X[src * NQ + qp], acc);
        if (c == 0) acc = fma(TB(base, 2, g2, a2, 1), X[3 * NQ + qp], acc);
      }
      (base + SM::TAB + NEN + SM::BUF)[k] = acc;
    }
    __syncthreads();
    // B2: Z0 = sum_g1 B1 Y00 + B1' Y01; Z1 = sum B1 Y10 -> X[c][a2][a1][g0]
    for (int idx = tid; idx < NE * 2 * N1 * N1 * Q; idx += nt) {
      int le = idx / (2 * N1 * N1 * Q), k = idx % (2 * N1 * N1 * Q);
      int c = k / (N1 * N1 * Q), r = k % (N1 * N1 * Q);
      int a2 = r / (N1 * Q), a1 = (r / Q) % N1, g0 = r % Q;
      double *base = smem + (size_t)le * SM::PER;
      const double *Y = base + SM::TAB + NEN + SM::BUF;
      double acc = 0.0;
#pragma unroll
      for (int g1 = 0; g1 < Q; g1++) {
        int o = (a2 * Q + g1) * Q + g0;
        if (c == 0) {
          acc = fma(TB(base, 1, g1, a1, 0), Y[0 * N1 * Q * Q + o], acc);
          acc = fma(TB(base, 1, g1, a1, 1), Y[2 * N1 * Q * Q + o], acc);
        } else {
          acc = fma(TB(base, 1, g1, a1, 0), Y[1 * N1 * Q * Q + o], acc);
        }
      }
      (base + SM::TAB + NEN)[k] = acc;
    }
    __syncthreads();
    // B1: F[a2][a1][a0] = sum_g0 B0 Z0 + B0' Z1, times w_A
    for (int idx = tid; idx < NE * NEN; idx += nt) {
      int le = idx / NEN, a = idx % NEN;
      int64_t e = ebase + le;
      if (e >= nelem) continue;
      int a0 = a % N1, a1 = (a / N1) % N1, a2 = a / (N1 * N1);
      double *base = smem + (size_t)le * SM::PER;
      const double *Z = base + SM::TAB + NEN;
      double acc = 0.0;
#pragma unroll
      for (int g0 = 0; g0 < Q; g0++) {
        int o = (a2 * N1 + a1) * Q + g0;
        acc = fma(TB(base, 0, g0, a0, 0), Z[o], acc);
        acc = fma(TB(base, 0, g0, a0, 1), Z[N1 * N1 * Q + o], acc);
      }
      if (wts) {
        int e0 = (int)(e % d0.nel), e1 = (int)((e / d0.nel) % d1.nel), e2 = (int)(e / ((int64_t)d0.nel * d1.nel));
        int64_t G = (d0.first[e0] + a0) + (int64_t)d0.n * ((d1.first[e1] + a1) + (int64_t)d1.n * (d2.first[e2] + a2));
        acc *= wts[G];
      }
      Fe[(size_t)e * NEN + a] = acc;
    }
  } else {
    // B2: Z0[a1][g0] = sum_g1 B1 s + B1' v1; Z1 = sum B1 v0 -> Y[c][a1][g0]
    for (int idx = tid; idx < NE * 2 * N1 * Q; idx += nt) {
      int le = idx / (2 * N1 * Q), k = idx % (2 * N1 * Q);
      int c = k / (N1 * Q), r = k % (N1 * Q);
      int a1 = r / Q, g0 = r % Q;
      double *base = smem + (size_t)le * SM::PER;
      const double *X = base + SM::TAB + NEN;
      double acc = 0.0;
#pragma unroll
      for (int g1 = 0; g1 < Q; g1++) {
        int qp = g1 * Q + g0;
        if (c == 0) {
          acc = fma(TB(base, 1, g1, a1, 0), X[qp], acc);
          acc = fma(TB(base, 1, g1, a1, 1), X[2 * NQ + qp], acc);
        } else {
          acc = fma(TB(base, 1, g1, a1, 0), X[NQ + qp], acc);
        }
      }
      (base + SM::TAB + NEN + SM::BUF)[k] = acc;
    }
    __syncthreads();
    for (int idx = tid; idx < NE * NEN; idx += nt) {
      int le = idx / NEN, a = idx % NEN;
      int64_t e = ebase + le;
      if (e >= nelem) continue;
      int a0 = a % N1, a1 = a / N1;
      double *base = smem + (size_t)le * SM::PER;
      const double *Z = base + SM::TAB + NEN + SM::BUF;
      double acc = 0.0;
#pragma unroll
      for (int g0 = 0; g0 < Q; g0++) {
        acc = fma(TB(base, 0, g0, a0, 0), Z[a1 * Q + g0], acc);
        acc = fma(TB(base, 0, g0, a0, 1), Z[N1 * Q + a1 * Q + g0], acc);
      }
      if (wts) {
        int e0 = (int)(e % d0.nel), e1 = (int)(e / d0.nel);
        int64_t G = (d0.first[e0] + a0) + (int64_t)d0.n * (d1.first[e1] + a1);
        acc *= wts[G];
      }
      Fe[(size_t)e * NEN + a] = acc;
    }
  }
#undef TB
}

// Gather F_A = sum of the element vectors of the elements containing A
// (Algorithm 3: F_e -> F), fixed order e2, e1, e0 ascending, added to add[A]
// when given; Dirichlet rows.
template <int DIM>
__global__ void k_gather_residual(DirArgs d0, DirArgs d1, DirArgs d2, const double *__restrict__ Fe,
                                  const double *__restrict__ U, BndArgs bnd, double *__restrict__ F, int64_t N, int N1,
                                  const double *__restrict__ add, int lin = 0, const double *__restrict__ done = nullptr) {
  if (done && done[0] != 0.0) return;
  int64_t A = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (A >= N) return;
  int i0 = (int)(A % d0.n), i1 = (int)((A / d0.n) % d1.n), i2 = (DIM == 3) ? (int)(A / ((int64_t)d0.n * d1.n)) : 0;
  int NEN = (DIM == 3) ? N1 * N1 * N1 : N1 * N1;
  double acc = add ? add[A] : 0.0;
  int lo2 = (DIM == 3) ? d2.node_e0[i2] : 0, hi2 = (DIM == 3) ? lo2 + d2.node_ne[i2] : 1;
  for (int e2 = lo2; e2 < hi2; e2++) {
    int a2 = (DIM == 3) ? i2 - d2.first[e2] : 0;
    for (int e1 = d1.node_e0[i1]; e1 < d1.node_e0[i1] + d1.node_ne[i1]; e1++) {
      int a1 = i1 - d1.first[e1];
      for (int e0 = d0.node_e0[i0]; e0 < d0.node_e0[i0] + d0.node_ne[i0]; e0++) {
        int a0 = i0 - d0.first[e0];
        int64_t e = e0 + (int64_t)d0.nel * (e1 + (int64_t)d1.nel * e2);
        acc += Fe[(size_t)e * NEN + (a2 * N1 + a1) * N1 + a0];
      }
    }
  }
  // Dirichlet rows: F_A = U_A - g (face order decides the value at edges)
  int idx[3] = {i0, i1, i2};
  int nn[3] = {d0.n, d1.n, d2.n};
  bool on = false;
  double g = 0.0;
  for (int ax = 0; ax < DIM; ax++) {
    if (bnd.flag[ax][0] && idx[ax] == 0) { on = true; g = bnd.val[ax][0]; }
    if (bnd.flag[ax][1] && idx[ax] == nn[ax] - 1) { on = true; g = bnd.val[ax][1]; }
  }
  // lin 1: Jacobian times a direction (identity rows); 2: Jacobian diagonal (1)
  F[A] = on ? (lin == 2 ? 1.0 : (lin ? U[A] : U[A] - g)) : acc;
}

// ---------------------------------------------------------------------------
// Q_00 at the Gauss points: sum-factorised value-only interpolation of u~,
// then Q00 = cs * g^T S g - cr * jw/W^2 * lambda * exp(u~/W).
// ---------------------------------------------------------------------------
//
// With MODE 1 the same interpolation yields the reaction part of the residual
// instead (and the reaction part of Q00 at the same U, for the Jacobian that
// follows an accepted line-search point): s = -jw/W * lambda * exp(u) at the Gauss points, projected back on
// the element's functions (value tables only) into Fe[e][A] (times w_A).  The
// Newton solver adds it to K U, K the assembled U-independent stiffness: since
// Eq. (residual) is K U plus this term under the same quadrature, F(U) then
// needs one operator product and a quarter of the sum-factorised contractions.
//
// With MODE 2 it adds the rate term of the time-dependent residual (Sec. 4.2),
// (N_A, v^h) with v^h = sum (shift U_B + C_B) N_B, to Fe: the interpolated value is
// ṽ = sum w_B (shift U_B + C_B) M_B, s = jw/W^2 ṽ.  In MODES 0 and 1 shift is the
// coefficient of dR/dU-dot in the Jacobian: Q00 gains cr * shift * jw/W^2.
template <int DIM, int P, int NE, int MODE>
__global__ void __launch_bounds__(128) k_q00(DirArgs d0, DirArgs d1, DirArgs d2, const double *__restrict__ U,
                                             const double *__restrict__ wts, const double *__restrict__ geom, GeomLayout gl,
                                             double lambda, double cs, double cr, double *__restrict__ Q00, int64_t nelem,
                                             double *__restrict__ q00_out, double shift = 0.0,
                                             const double *__restrict__ C = nullptr) {
  constexpr bool RES = MODE != 0;
  using SM = ResSmem<DIM, P>;
  constexpr int N1 = SM::N1, Q = SM::Q, NEN = SM::NEN, NQ = SM::NQ;
  extern __shared__ double smem[];
  const int tid = threadIdx.x, nt = blockDim.x;
  const int64_t ebase = (int64_t)blockIdx.x * NE;
  for (int idx = tid; idx < NE * (SM::TAB + NEN); idx += nt) {
    int le = idx / (SM::TAB + NEN), k = idx % (SM::TAB + NEN);
    int64_t e = ebase + le;
    double *base = smem + (size_t)le * SM::PER;
    if (e >= nelem) { base[k] = 0.0; continue; }
    int e0 = (int)(e % d0.nel), e1 = (int)((e / d0.nel) % d1.nel), e2 = (DIM == 3) ? (int)(e / ((int64_t)d0.nel * d1.nel)) : 0;
    if (k < SM::TAB) {
      int ax = k / (Q * N1 * 2), r = k % (Q * N1 * 2);
      const DirArgs &d = ax == 0 ? d0 : (ax == 1 ? d1 : d2);
      int ee = ax == 0 ? e0 : (ax == 1 ? e1 : e2);
      base[k] = d.tab[(size_t)ee * Q * N1 * 2 + r];
    } else {
      int a = k - SM::TAB;
      int a0 = a % N1, a1 = (a / N1) % N1, a2 = (DIM == 3) ? a / (N1 * N1) : 0;
      int64_t G = (d0.first[e0] + a0) + (int64_t)d0.n * ((d1.first[e1] + a1) + (int64_t)d1.n * ((DIM == 3 ? d2.first[e2] : 0) + a2));
      double x = U ? U[G] : 0.0;
      if (MODE == 2) x = shift * x + (C ? C[G] : 0.0);
      base[k] = x * (wts ? wts[G] : 1.0);
    }
  }
  __syncthreads();
#define TB(base, ax, g, a) (base)[(((ax) * Q + (g)) * N1 + (a)) * 2]
  // contract axis 0, then 1, then 2 (values only)
  if (DIM == 3) {
    for (int idx = tid; idx < NE * N1 * N1 * Q; idx += nt) {
      int le = idx / (N1 * N1 * Q), r = idx % (N1 * N1 * Q);
      int a2 = r / (N1 * Q), a1 = (r / Q) % N1, g0 = r % Q;
      double *base = smem + (size_t)le * SM::PER;
      const double *C = base + SM::TAB;
      double acc = 0.0;
#pragma unroll
      for (int a0 = 0; a0 < N1; a0++) acc = fma(TB(base, 0, g0, a0), C[(a2 * N1 + a1) * N1 + a0], acc);
      (base + SM::TAB + NEN)[r] = acc;
    }
    __syncthreads();
    for (int idx = tid; idx < NE * N1 * Q * Q; idx += nt) {
      int le = idx / (N1 * Q * Q), r = idx % (N1 * Q * Q);
      int a2 = r / (Q * Q), g1 = (r / Q) % Q, g0 = r % Q;
      double *base = smem + (size_t)le * SM::PER;
      const double *X = base + SM::TAB + NEN;
      double acc = 0.0;
#pragma unroll
      for (int a1 = 0; a1 < N1; a1++) acc = fma(TB(base, 1, g1, a1), X[(a2 * N1 + a1) * Q + g0], acc);
      (base + SM::TAB + NEN + SM::BUF)[r] = acc;
    }
    __syncthreads();
  } else {
    for (int idx = tid; idx < NE * N1 * Q; idx += nt) {
      int le = idx / (N1 * Q), r = idx % (N1 * Q);
      int a1 = r / Q, g0 = r % Q;
      double *base = smem + (size_t)le * SM::PER;
      const double *C = base + SM::TAB;
      double acc = 0.0;
#pragma unroll
      for (int a0 = 0; a0 < N1; a0++) acc = fma(TB(base, 0, g0, a0), C[a1 * N1 + a0], acc);
      (base + SM::TAB + NEN + SM::BUF)[r] = acc;
    }
    __syncthreads();
  }
  for (int idx = tid; idx < NE * NQ; idx += nt) {
    int le = idx / NQ, qp = idx % NQ;
    int64_t e = ebase + le;
    if (e >= nelem) continue;
    double *base = smem + (size_t)le * SM::PER;
    const double *Y = base + SM::TAB + NEN + SM::BUF;
    double ut = 0.0;
    if (DIM == 3) {
      int g2 = qp / (Q * Q), g1 = (qp / Q) % Q, g0 = qp % Q;
#pragma unroll
      for (int a2 = 0; a2 < N1; a2++) ut = fma(TB(base, 2, g2, a2), Y[(a2 * Q + g1) * Q + g0], ut);
    } else {
      int g1 = qp / Q, g0 = qp % Q;
#pragma unroll
      for (int a1 = 0; a1 < N1; a1++) ut = fma(TB(base, 1, g1, a1), Y[a1 * Q + g0], ut);
    }
    const double *rec = geom + (size_t)e * gl.nf * NQ + qp;
    if (MODE == 2) {
      (base + SM::TAB + NEN)[qp] = rec[gl.jwW2 * NQ] * ut;
      continue;
    }
    if (RES) {
      const double lex = lambda * iga_exp(ut * rec[gl.invW * NQ]);
      (base + SM::TAB + NEN)[qp] = -rec[gl.jwW * NQ] * lex;
      // the reaction part of Q00 at the same point, for the next Jacobian
      if (q00_out) {
        double v = -rec[gl.jwW2 * NQ] * lex;
        if (shift != 0.0) v += shift * rec[gl.jwW2 * NQ];
        q00_out[(size_t)e * NQ + qp] = v;
      }
      continue;
    }
    double v = 0.0;
    if (cs != 0.0) v = cs * rec[gl.gSg * NQ];
    if (cr != 0.0) {
      v -= cr * rec[gl.jwW2 * NQ] * lambda * iga_exp(ut * rec[gl.invW * NQ]);
      if (shift != 0.0) v += cr * shift * rec[gl.jwW2 * NQ];
    }
    Q00[(size_t)e * NQ + qp] = v;
  }
  if (!RES) return;
  __syncthreads();
  // project s on the element's functions: contract axis 2 (3D), then 1, then 0
  if (DIM == 3) {
    for (int idx = tid; idx < NE * N1 * Q * Q; idx += nt) {
      int le = idx / (N1 * Q * Q), r = idx % (N1 * Q * Q);
      int a2 = r / (Q * Q), g1 = (r / Q) % Q, g0 = r % Q;
      double *base = smem + (size_t)le * SM::PER;
      const double *X = base + SM::TAB + NEN;
      double acc = 0.0;
#pragma unroll
      for (int g2 = 0; g2 < Q; g2++) acc = fma(TB(base, 2, g2, a2), X[(g2 * Q + g1) * Q + g0], acc);
      (base + SM::TAB + NEN + SM::BUF)[r] = acc;
    }
    __syncthreads();
    for (int idx = tid; idx < NE * N1 * N1 * Q; idx += nt) {
      int le = idx / (N1 * N1 * Q), r = idx % (N1 * N1 * Q);
      int a2 = r / (N1 * Q), a1 = (r / Q) % N1, g0 = r % Q;
      double *base = smem + (size_t)le * SM::PER;
      const double *Y = base + SM::TAB + NEN + SM::BUF;
      double acc = 0.0;
#pragma unroll
      for (int g1 = 0; g1 < Q; g1++) acc = fma(TB(base, 1, g1, a1), Y[(a2 * Q + g1) * Q + g0], acc);
      (base + SM::TAB + NEN)[r] = acc;
    }
    __syncthreads();
    for (int idx = tid; idx < NE * NEN; idx += nt) {
      int le = idx / NEN, a = idx % NEN;
      int64_t e = ebase + le;
      if (e >= nelem) continue;
      int a0 = a % N1, a1 = (a / N1) % N1, a2 = a / (N1 * N1);
      double *base = smem + (size_t)le * SM::PER;
      const double *Z = base + SM::TAB + NEN;
      double acc = 0.0;
#pragma unroll
      for (int g0 = 0; g0 < Q; g0++) acc = fma(TB(base, 0, g0, a0), Z[(a2 * N1 + a1) * Q + g0], acc);
      if (wts) {
        int e0 = (int)(e % d0.nel), e1 = (int)((e / d0.nel) % d1.nel), e2 = (int)(e / ((int64_t)d0.nel * d1.nel));
        acc *= wts[(d0.first[e0] + a0) + (int64_t)d0.n * ((d1.first[e1] + a1) + (int64_t)d1.n * (d2.first[e2] + a2))];
      }
      if (MODE == 2) Q00[(size_t)e * NEN + a] += acc;
      else Q00[(size_t)e * NEN + a] = acc;
    }
  } else {
    for (int idx = tid; idx < NE * N1 * Q; idx += nt) {
      int le = idx / (N1 * Q), r = idx % (N1 * Q);
      int a1 = r / Q, g0 = r % Q;
      double *base = smem + (size_t)le * SM::PER;
      const double *X = base + SM::TAB + NEN;
      double acc = 0.0;
#pragma unroll
      for (int g1 = 0; g1 < Q; g1++) acc = fma(TB(base, 1, g1, a1), X[g1 * Q + g0], acc);
      (base + SM::TAB + NEN + SM::BUF)[r] = acc;
    }
    __syncthreads();
    for (int idx = tid; idx < NE * NEN; idx += nt) {
      int le = idx / NEN, a = idx % NEN;
      int64_t e = ebase + le;
      if (e >= nelem) continue;
      int a0 = a % N1, a1 = a / N1;
      double *base = smem + (size_t)le * SM::PER;
      const double *Y = base + SM::TAB + NEN + SM::BUF;
      double acc = 0.0;
#pragma unroll
      for (int g0 = 0; g0 < Q; g0++) acc = fma(TB(base, 0, g0, a0), Y[a1 * Q + g0], acc);
      if (wts) {
        int e0 = (int)(e % d0.nel), e1 = (int)(e / d0.nel);
        acc *= wts[(d0.first[e0] + a0) + (int64_t)d0.n * (d1.first[e1] + a1)];
      }
      if (MODE == 2) Q00[(size_t)e * NEN + a] += acc;
      else Q00[(size_t)e * NEN + a] = acc;
    }
  }
#undef TB
}

// Column indices of the CSR pattern (Sec. 2.5): row A lists the lexicographic
// product of the BasisStencil ranges, axis 0 fastest, so columns ascend.
__global__ void k_colidx(DirArgs d0, DirArgs d1, DirArgs d2, int dim, const int64_t *__restrict__ rowptr,
                         int32_t *__restrict__ colidx, int64_t N) {
  int64_t A = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (A >= N) return;
  int i0 = (int)(A % d0.n), i1 = (int)((A / d0.n) % d1.n), i2 = (dim == 3) ? (int)(A / ((int64_t)d0.n * d1.n)) : 0;
  int64_t k = rowptr[A];
  int l2 = dim == 3 ? d2.l[i2] : 0, r2 = dim == 3 ? d2.r[i2] : 0;
  for (int j2 = l2; j2 <= r2; j2++)
    for (int j1 = d1.l[i1]; j1 <= d1.r[i1]; j1++)
      for (int j0 = d0.l[i0]; j0 <= d0.r[i0]; j0++)
        colidx[k++] = (int32_t)(j0 + (int64_t)d0.n * (j1 + (int64_t)d1.n * j2));
}

// ---------------------------------------------------------------------------
// Launchers
// ---------------------------------------------------------------------------
#define DISPATCH_DP(DIM_, P_, CALL)                         \
  do {                                                      \
    if ((DIM_) == 2) {                                      \
      switch (P_) {                                         \
        case 1: { constexpr int D = 2, PP = 1; CALL; } break; \
        case 2: { constexpr int D = 2, PP = 2; CALL; } break; \
        case 3: { constexpr int D = 2, PP = 3; CALL; } break; \
        case 4: { constexpr int D = 2, PP = 4; CALL; } break; \
      }                                                     \
    } else {                                                \
      switch (P_) {                                         \
        case 1: { constexpr int D = 3, PP = 1; CALL; } break; \
        case 2: { constexpr int D = 3, PP = 2; CALL; } break; \
        case 3: { constexpr int D = 3, PP = 3; CALL; } break; \
        case 4: { constexpr int D = 3, PP = 4; CALL; } break; \
      }                                                     \
    }                                                       \
  } while (0)

cudaError_t launch_geometry(iga_s *h, const double *ctrl_dev, const double *logk_dev) {
  int *err = nullptr;
  cudaError_t ce = cudaMallocAsync((void **)&err, sizeof(int), h->stream);
  if (ce) return ce;
  cudaMemsetAsync(err, 0, sizeof(int), h->stream);
  DirArgs a0 = dir_args(h->ddev[0]), a1 = dir_args(h->ddev[1]), a2 = dir_args(h->ddev[2]);
  IGA_LAUNCH(h, KC_GEOM, DISPATCH_DP(h->dim, h->p, ({
    using GS = GeoSmem<D, PP>;
    const size_t sm = (size_t)GS::NE * GS::PER * sizeof(double);
    if (sm > 48 * 1024) cudaFuncSetAttribute(k_geometry<D, PP>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    const unsigned grid = (unsigned)((h->nelem + GS::NE - 1) / GS::NE);
    k_geometry<D, PP><<<grid, 128, sm, h->stream>>>(a0, a1, a2, ctrl_dev, h->weights, logk_dev, h->gl, h->geom, h->nelem, err);
  })));
  int herr = 0;
  cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, h->stream);
  ce = cudaStreamSynchronize(h->stream);
  cudaFreeAsync(err, h->stream);
  if (ce) return ce;
  if (herr) return cudaErrorInvalidValue;  // det <= 0 somewhere: reported as EINVAL by the caller
  return cudaGetLastError();
}

template <int DIM, int P>
static size_t res_smem(int NE) { return (size_t)NE * ResSmem<DIM, P>::PER * sizeof(double); }

// Adds the rate term (N_A, v^h) of the time-dependent residual (Sec. 4.2) to the
// element vectors Fe, v = ts_a U + ts_C per control variable; nothing unless h->ts_on.
static cudaError_t launch_rate_term(iga_s *h, const double *U, double *Fe) {
  if (!h->ts_on) return cudaSuccess;
  DirArgs a0 = dir_args(h->ddev[0]), a1 = dir_args(h->ddev[1]), a2 = dir_args(h->ddev[2]);
  constexpr int NE = 4;
  unsigned grid = (unsigned)((h->nelem + NE - 1) / NE);
  IGA_LAUNCH(h, KC_RES_ELEM, DISPATCH_DP(h->dim, h->p, ({
    size_t sm = res_smem<D, PP>(NE);
    if (sm > 48 * 1024) cudaFuncSetAttribute(k_q00<D, PP, NE, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    k_q00<D, PP, NE, 2><<<grid, 128, sm, h->stream>>>(a0, a1, a2, U, h->weights, h->geom, h->gl, 0.0, 0.0, 0.0, Fe,
                                                      h->nelem, nullptr, h->ts_a, h->ts_C);
  })));
  return cudaGetLastError();
}

cudaError_t launch_residual(iga_s *h, const double *U, double *F) {
  if (h->inner) return periodic_residual(h, U, F);
  return launch_residual_into(h, U, F, h->Fe);
}

// The residual kernels (element pass, rate term, row gather) with the element-vector
// buffer supplied by the caller: the handle's own (launch_residual) or the fixed
// array of iga_form_residual_noalloc, so both entry points run the same code.
cudaError_t launch_residual_into(iga_s *h, const double *U, double *F, double *Fe) {
  DirArgs a0 = dir_args(h->ddev[0]), a1 = dir_args(h->ddev[1]), a2 = dir_args(h->ddev[2]);
  constexpr int NE = 4;
  unsigned grid = (unsigned)((h->nelem + NE - 1) / NE);
  IGA_LAUNCH(h, KC_RES_ELEM, DISPATCH_DP(h->dim, h->p, ({
    size_t sm = res_smem<D, PP>(NE);
    if (sm > 48 * 1024) cudaFuncSetAttribute(k_residual<D, PP, NE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    k_residual<D, PP, NE><<<grid, 128, sm, h->stream>>>(a0, a1, a2, U, h->weights, h->geom, h->gl, h->lambda, Fe, h->nelem);
  })));
  cudaError_t ce = launch_rate_term(h, U, Fe);
  if (ce) return ce;
  unsigned g2 = (unsigned)((h->N + 255) / 256);
  if (h->dim == 3)
    IGA_LAUNCH(h, KC_RES_GATHER, (k_gather_residual<3><<<g2, 256, 0, h->stream>>>(a0, a1, a2, Fe, U, h->bnd, F, h->N, h->p + 1, nullptr)));
  else
    IGA_LAUNCH(h, KC_RES_GATHER, (k_gather_residual<2><<<g2, 256, 0, h->stream>>>(a0, a1, a2, Fe, U, h->bnd, F, h->N, h->p + 1, nullptr)));
  return cudaGetLastError();
}

// Q00 = cs gSg (no reaction term: the stiffness alone), straight from the geometry cache
__global__ static void k_q00_geom(const double *__restrict__ geom, GeomLayout gl, int nq, int64_t nelem, double cs,
                                  double *__restrict__ Q00) {
  const int64_t tot = nelem * nq;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < tot; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t e = t / nq;
    const int qp = (int)(t - e * nq);
    Q00[t] = cs * geom[((size_t)e * gl.nf + gl.gSg) * nq + qp];
  }
}

cudaError_t launch_q00(iga_s *h, const double *U, double cs, double cr) {
  DirArgs a0 = dir_args(h->ddev[0]), a1 = dir_args(h->ddev[1]), a2 = dir_args(h->ddev[2]);
  if (cr == 0.0) {  // the U-independent stiffness: no interpolation, no exponential
    const int nq = h->dim == 3 ? h->q * h->q * h->q : h->q * h->q;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int64_t want = (h->nelem * nq + 255) / 256;
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(want, (int64_t)(sms > 0 ? sms : 1) * 8));
    IGA_LAUNCH(h, KC_Q00, (k_q00_geom<<<grid, 256, 0, h->stream>>>(h->geom, h->gl, nq, h->nelem, cs, h->Q00)));
    return cudaGetLastError();
  }
  constexpr int NE = 8;  // value-only interpolation: more elements per CTA
  unsigned grid = (unsigned)((h->nelem + NE - 1) / NE);
  IGA_LAUNCH(h, KC_Q00, DISPATCH_DP(h->dim, h->p, ({
    size_t sm = res_smem<D, PP>(NE);
    if (sm > 48 * 1024) cudaFuncSetAttribute(k_q00<D, PP, NE, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    k_q00<D, PP, NE, 0><<<grid, 128, sm, h->stream>>>(a0, a1, a2, U, h->weights, h->geom, h->gl, h->lambda, cs, cr, h->Q00, h->nelem,
                                                      nullptr, h->ts_on ? h->ts_a : 0.0);
  })));
  return cudaGetLastError();
}

// Q00 in FP32 arithmetic for the reduced-precision Jacobians (same definition as
// k_q00 MODE 0), stored as double.
template <int DIM, int P>
__global__ void __launch_bounds__(128) k_q00_f32(DirArgs d0, DirArgs d1, DirArgs d2, const double *__restrict__ U,
                                                 const double *__restrict__ wts, const double *__restrict__ geom, GeomLayout gl,
                                                 float lambda, float cs, float cr, float shift, double *__restrict__ Q00,
                                                 int64_t nelem) {
  using S = InterpF32<DIM, P>;
  __shared__ float ue[S::EB * S::NEN], tb[S::EB * DIM * S::Q * S::N1];
  const int64_t e_first = (int64_t)blockIdx.x * S::EB;
  const float ut = interp_u_block<DIM, P>(d0, d1, d2, cr != 0.f ? U : nullptr, wts, e_first, nelem, ue, tb);
  const int le = threadIdx.x / S::NQ, qp = threadIdx.x - le * S::NQ;
  const int64_t e = e_first + le;
  if (le >= S::EB || e >= nelem) return;
  const double *rec = geom + (size_t)e * gl.nf * S::NQ + qp;
  float v = cs != 0.f ? cs * (float)rec[gl.gSg * S::NQ] : 0.f;
  if (cr != 0.f) {
    const float jw2 = (float)rec[gl.jwW2 * S::NQ];
    v -= cr * jw2 * lambda * __expf(ut * (float)rec[gl.invW * S::NQ]);
    if (shift != 0.f) v += cr * shift * jw2;
  }
  Q00[(size_t)e * S::NQ + qp] = (double)v;
}

// The same Q00 for elements of at most 27 Gauss points (2D, or 3D with p <= 2), in two
// phases per block of 128 elements: one thread per element computes u~ at its Gauss
// points (weighted coefficients and FP32 1D tables in registers, the nested sums of
// interp_u_block -- axis 0 innermost, then axis 1, then axis 2, each in function order --
// with the partial sums shared between points) into shared memory; then one thread per
// (element, Gauss point) of the block's contiguous range reads the geometry factors and
// writes Q00, both coalesced.  The same operations per point as k_q00_f32.
template <int DIM, int P>
__global__ void __launch_bounds__(128) k_q00_f32e(DirArgs d0, DirArgs d1, DirArgs d2, const double *__restrict__ U,
                                                  const double *__restrict__ wts, const double *__restrict__ geom, GeomLayout gl,
                                                  float lambda, float cs, float cr, float shift, double *__restrict__ Q00,
                                                  int64_t nelem) {
  constexpr int Q = P + 1, EB = 128, NQ = DIM == 3 ? Q * Q * Q : Q * Q;
  __shared__ float ut_s[EB * NQ];
  const int64_t e_first = (int64_t)blockIdx.x * EB, e = e_first + threadIdx.x;
  if (e < nelem) interp_u_elem<DIM, P>(d0, d1, d2, cr != 0.f ? U : nullptr, wts, e, ut_s + threadIdx.x * NQ);
  __syncthreads();
  const int nb = (int)min((int64_t)EB, nelem - e_first);
  for (int k = threadIdx.x; k < nb * NQ; k += EB) {
    const int le = k / NQ, qp = k - le * NQ;
    const double *rec = geom + (size_t)(e_first + le) * gl.nf * NQ + qp;
    float v = cs != 0.f ? cs * (float)rec[gl.gSg * NQ] : 0.f;
    if (cr != 0.f) {
      const float jw2 = (float)rec[gl.jwW2 * NQ];
      v -= cr * jw2 * lambda * __expf(ut_s[k] * (float)rec[gl.invW * NQ]);
      if (shift != 0.f) v += cr * shift * jw2;
    }
    Q00[(size_t)e_first * NQ + k] = (double)v;
  }
}

cudaError_t launch_q00_f32(iga_s *h, const double *U, double cs, double cr) {
  DirArgs a0 = dir_args(h->ddev[0]), a1 = dir_args(h->ddev[1]), a2 = dir_args(h->ddev[2]);
  const float ts = h->ts_on ? (float)h->ts_a : 0.f;
  if (h->dim == 2 || h->p <= 2) {
    const unsigned grid = (unsigned)((h->nelem + 127) / 128);
    IGA_LAUNCH(h, KC_Q00, DISPATCH_DP(h->dim, h->p, ({
      constexpr int PE = (D == 2 || PP <= 2) ? PP : 2;  // 3D p > 2 does not reach this branch
      k_q00_f32e<D, PE><<<grid, 128, 0, h->stream>>>(a0, a1, a2, U, h->weights, h->geom, h->gl, (float)h->lambda, (float)cs,
                                                      (float)cr, ts, h->Q00, h->nelem);
    })));
    return cudaGetLastError();
  }
  IGA_LAUNCH(h, KC_Q00, DISPATCH_DP(h->dim, h->p, ({
    using S = InterpF32<D, PP>;
    const unsigned grid = (unsigned)((h->nelem + S::EB - 1) / S::EB);
    k_q00_f32<D, PP><<<grid, S::THREADS, 0, h->stream>>>(a0, a1, a2, U, h->weights, h->geom, h->gl, (float)h->lambda, (float)cs,
                                                         (float)cr, ts, h->Q00, h->nelem);
  })));
  return cudaGetLastError();
}

cudaError_t launch_residual_split(iga_s *h, const double *U, double *F, const double *K, double *KU) {
  DirArgs a0 = dir_args(h->ddev[0]), a1 = dir_args(h->ddev[1]), a2 = dir_args(h->ddev[2]);
  cudaError_t ce = launch_spmv64_residual(h, K, U, KU);
  if (ce) return ce;
  constexpr int NE = 4;
  unsigned grid = (unsigned)((h->nelem + NE - 1) / NE);
  IGA_LAUNCH(h, KC_RES_ELEM, DISPATCH_DP(h->dim, h->p, ({
    size_t sm = res_smem<D, PP>(NE);
    if (sm > 48 * 1024) cudaFuncSetAttribute(k_q00<D, PP, NE, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    k_q00<D, PP, NE, 1><<<grid, 128, sm, h->stream>>>(a0, a1, a2, U, h->weights, h->geom, h->gl, h->lambda, 0.0, 1.0, h->Fe, h->nelem,
                                                      h->Q00, h->ts_on ? h->ts_a : 0.0);
  })));
  ce = launch_rate_term(h, U, h->Fe);
  if (ce) return ce;
  unsigned g2 = (unsigned)((h->N + 255) / 256);
  if (h->dim == 3)
    IGA_LAUNCH(h, KC_RES_GATHER, (k_gather_residual<3><<<g2, 256, 0, h->stream>>>(a0, a1, a2, h->Fe, U, h->bnd, F, h->N, h->p + 1, KU)));
  else
    IGA_LAUNCH(h, KC_RES_GATHER, (k_gather_residual<2><<<g2, 256, 0, h->stream>>>(a0, a1, a2, h->Fe, U, h->bnd, F, h->N, h->p + 1, KU)));
  return cudaGetLastError();
}


// ---------------------------------------------------------------------------
// Diagonal of the Jacobian (the Jacobi preconditioner of the matrix-free solve):
//   J_AA = w_A^2 sum_q [Q00 M^2 + 2 sum_a Q0a M dM_a + sum_ab S_ab dM_a dM_b](x_q),
// Q00 = g^T S g + q00 (q00: the reaction part at the Newton iterate), Q0a = (-S g)_a.
// One CTA per element; its geometry record and 1D tables in shared memory, one
// thread per local function A.  Element contributions go to Fe and are gathered
// per row in a fixed order (Dirichlet rows: 1).
// ---------------------------------------------------------------------------
template <int DIM, int P>
__global__ void __launch_bounds__(128) k_diag_elem(DirArgs d0, DirArgs d1, DirArgs d2, const double *__restrict__ wts,
                                                   const double *__restrict__ geom, GeomLayout gl,
                                                   const double *__restrict__ q00, double *__restrict__ Fe, int64_t nelem) {
  constexpr int N1 = P + 1, Q = P + 1;
  constexpr int NEN = DIM == 3 ? N1 * N1 * N1 : N1 * N1, NQ = DIM == 3 ? Q * Q * Q : Q * Q;
  constexpr int NS = DIM * (DIM + 1) / 2;
  __shared__ double tab[3][Q][N1][2];
  __shared__ double qf[1 + DIM + NS][NQ];  // Q00, Q0a, S_ab (00,11,22,01,02,12 / 00,11,01)
  const int64_t e = blockIdx.x;
  if (e >= nelem) return;
  const int e0 = (int)(e % d0.nel), e1 = (int)((e / d0.nel) % d1.nel), e2 = DIM == 3 ? (int)(e / ((int64_t)d0.nel * d1.nel)) : 0;
  for (int k = threadIdx.x; k < DIM * Q * N1 * 2; k += blockDim.x) {
    const int ax = k / (Q * N1 * 2), r = k % (Q * N1 * 2);
    const DirArgs &d = ax == 0 ? d0 : (ax == 1 ? d1 : d2);
    const int ee = ax == 0 ? e0 : (ax == 1 ? e1 : e2);
    (&tab[ax][0][0][0])[r] = d.tab[(size_t)ee * Q * N1 * 2 + r];
  }
  const double *rec = geom + (size_t)e * gl.nf * NQ;
  for (int k = threadIdx.x; k < NQ; k += blockDim.x) {
    qf[0][k] = rec[gl.gSg * NQ + k] + q00[(size_t)e * NQ + k];
    for (int a = 0; a < DIM; a++) qf[1 + a][k] = rec[(gl.Sg + a) * NQ + k];
    for (int b = 0; b < NS; b++) qf[1 + DIM + b][k] = rec[(gl.S + b) * NQ + k];
  }
  __syncthreads();
  for (int A = threadIdx.x; A < NEN; A += blockDim.x) {
    const int a0 = A % N1, a1 = (A / N1) % N1, a2 = DIM == 3 ? A / (N1 * N1) : 0;
    double acc = 0.0;
    for (int qp = 0; qp < NQ; qp++) {
      const int g0 = qp % Q, g1 = (qp / Q) % Q, g2 = DIM == 3 ? qp / (Q * Q) : 0;
      const double b0 = tab[0][g0][a0][0], db0 = tab[0][g0][a0][1];
      const double b1 = tab[1][g1][a1][0], db1 = tab[1][g1][a1][1];
      double m, d[3];
      if (DIM == 3) {
        const double b2 = tab[2][g2][a2][0], db2 = tab[2][g2][a2][1];
        m = b0 * b1 * b2;
        d[0] = db0 * b1 * b2;
        d[1] = b0 * db1 * b2;
        d[2] = b0 * b1 * db2;
        const double t = qf[0][qp] * m * m + 2.0 * m * (qf[1][qp] * d[0] + qf[2][qp] * d[1] + qf[3][qp] * d[2]) +
                         qf[4][qp] * d[0] * d[0] + qf[5][qp] * d[1] * d[1] + qf[6][qp] * d[2] * d[2] +
                         2.0 * (qf[7][qp] * d[0] * d[1] + qf[8][qp] * d[0] * d[2] + qf[9][qp] * d[1] * d[2]);
        acc += t;
      } else {
        m = b0 * b1;
        d[0] = db0 * b1;
        d[1] = b0 * db1;
        const double t = qf[0][qp] * m * m + 2.0 * m * (qf[1][qp] * d[0] + qf[2][qp] * d[1]) + qf[3][qp] * d[0] * d[0] +
                         qf[4][qp] * d[1] * d[1] + 2.0 * qf[5][qp] * d[0] * d[1];
        acc += t;
      }
    }
    if (wts) {
      const int64_t G = (d0.first[e0] + a0) + (int64_t)d0.n * ((d1.first[e1] + a1) + (int64_t)d1.n * ((DIM == 3 ? d2.first[e2] : 0) + a2));
      acc *= wts[G] * wts[G];
    }
    Fe[(size_t)e * NEN + A] = acc;
  }
}

// y = J(U) x without an assembled matrix; h->Q00 must hold the reaction part of Q00 at U
// (launch_q00(h, U, 0, 1)).  done: device flag that skips the work once set (may be null).
cudaError_t launch_jv(iga_s *h, const double *x, double *y, const double *done) {
  DirArgs a0 = dir_args(h->ddev[0]), a1 = dir_args(h->ddev[1]), a2 = dir_args(h->ddev[2]);
  constexpr int NE = 4;
  unsigned grid = (unsigned)((h->nelem + NE - 1) / NE);
  IGA_LAUNCH(h, KC_RES_ELEM, DISPATCH_DP(h->dim, h->p, ({
    size_t sm = res_smem<D, PP>(NE);
    if (sm > 48 * 1024) cudaFuncSetAttribute(k_residual<D, PP, NE, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    k_residual<D, PP, NE, true><<<grid, 128, sm, h->stream>>>(a0, a1, a2, x, h->weights, h->geom, h->gl, h->lambda, h->Fe,
                                                             h->nelem, h->Q00, h->bnd, done);
  })));
  unsigned g2 = (unsigned)((h->N + 255) / 256);
  if (h->dim == 3)
    IGA_LAUNCH(h, KC_RES_GATHER, (k_gather_residual<3><<<g2, 256, 0, h->stream>>>(a0, a1, a2, h->Fe, x, h->bnd, y, h->N, h->p + 1, nullptr, 1, done)));
  else
    IGA_LAUNCH(h, KC_RES_GATHER, (k_gather_residual<2><<<g2, 256, 0, h->stream>>>(a0, a1, a2, h->Fe, x, h->bnd, y, h->N, h->p + 1, nullptr, 1, done)));
  return cudaGetLastError();
}

// diag(J(U)) (Dirichlet rows 1); h->Q00 as for launch_jv
cudaError_t launch_jacobian_diagonal(iga_s *h, double *diag) {
  DirArgs a0 = dir_args(h->ddev[0]), a1 = dir_args(h->ddev[1]), a2 = dir_args(h->ddev[2]);
  IGA_LAUNCH(h, KC_RES_ELEM, DISPATCH_DP(h->dim, h->p, ({
    k_diag_elem<D, PP><<<(unsigned)h->nelem, 128, 0, h->stream>>>(a0, a1, a2, h->weights, h->geom, h->gl, h->Q00, h->Fe, h->nelem);
  })));
  unsigned g2 = (unsigned)((h->N + 255) / 256);
  if (h->dim == 3)
    IGA_LAUNCH(h, KC_RES_GATHER, (k_gather_residual<3><<<g2, 256, 0, h->stream>>>(a0, a1, a2, h->Fe, nullptr, h->bnd, diag, h->N, h->p + 1, nullptr, 2, nullptr)));
  else
    IGA_LAUNCH(h, KC_RES_GATHER, (k_gather_residual<2><<<g2, 256, 0, h->stream>>>(a0, a1, a2, h->Fe, nullptr, h->bnd, diag, h->N, h->p + 1, nullptr, 2, nullptr)));
  return cudaGetLastError();
}

cudaError_t launch_colidx(iga_s *h) {
  DirArgs a0 = dir_args(h->ddev[0]), a1 = dir_args(h->ddev[1]), a2 = dir_args(h->ddev[2]);
  unsigned g = (unsigned)((h->N + 255) / 256);
  IGA_LAUNCH(h, KC_PATTERN, (k_colidx<<<g, 256, 0, h->stream>>>(a0, a1, a2, h->dim, h->rowptr, h->colidx, h->N)));
  return cudaGetLastError();
}

namespace {
__global__ void k_exp_eval(const double *__restrict__ x, double *__restrict__ y, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    y[i] = iga_exp(x[i]);
}
}  // namespace

extern "C" iga_status iga_exp_eval(void *stream, const double *x, double *y, int64_t n) {
  if (n < 0 || (n > 0 && (!x || !y))) return IGA_EINVAL;
  if (n == 0) return IGA_OK;
  const int64_t blocks = std::min<int64_t>((n + 255) / 256, 152 * 8);
  k_exp_eval<<<(unsigned)blocks, 256, 0, (cudaStream_t)stream>>>(x, y, n);
  return cudaGetLastError() == cudaSuccess ? IGA_OK : IGA_ECUDA;
}
