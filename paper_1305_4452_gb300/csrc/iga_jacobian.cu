// Jacobian assembly of libiga by global sum factorisation (Eq. jacobian).
//
// With the cached geometry factors the Jacobian entry is
//     J_AB = w_A w_B sum_q sum_{mu,nu} Q_{mu nu}(q) D_mu M_A(q) D_nu M_B(q),
// mu, nu in {value, d/dxi_0, d/dxi_1, d/dxi_2}, Q symmetric.  M_A is a tensor
// product of 1D B-splines, so the sum over the Gauss points of the whole mesh is
// done one direction at a time: stage 1 contracts axis 0 into 1D function pairs
// (i0, j0) -- the BasisStencil pairs of Sec. 2.5 -- stage 2 contracts axis 1, and
// the final stage contracts the last axis and writes each CSR entry exactly once
// (deterministic, no atomics).  After a stage, terms that share their derivative
// pattern in the remaining directions are added, and Q's symmetry makes some
// partial sums the pair-transposes of others, so the stiffness needs 10, 7 and 4
// one-dimensional contractions per output in 3D (6 and 4 in 2D) instead of
// 16, 9 and 4; stage 1 also forms the transpose-invariant groups once per pair of
// transposed 1D pairs.  On an identity map with unit weights (g = 0, S diagonal) the
// counts drop to 4, 3 and 2 (2D: 3 and 2).  The reaction term alone (Q00 only) is one
// chain of single contractions and can be added onto a previously assembled stiffness.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <stdint.h>

#include "iga_internal.h"

namespace {

template <int DIM> __host__ __device__ constexpr int ipow(int b) { return DIM == 2 ? b * b : b * b * b; }

enum { PLAN_STIFF = 0, PLAN_MASS = 1, PLAN_DIAG = 2, PLAN_DIAGS = 3 };

struct CsrArgs {
  const int64_t *rowptr;
  const int64_t *rp_line;  // first CSR position of each line (i1, i2) of rows
  const int *rp_p0;        // prefix sums of the axis-0 stencil widths
  const double *wts;       // rational weights (J_AB carries w_A w_B) or null
  BndArgs bnd;
};

template <typename T> __device__ __forceinline__ const T *ptab(const DirArgs &d);
template <> __device__ __forceinline__ const double *ptab<double>(const DirArgs &d) { return d.pair_val; }
template <> __device__ __forceinline__ const float *ptab<float>(const DirArgs &d) { return d.pair_val_f; }

template <int PLAN, int DIM> struct Shape {
  // Q slots read by stage 1
  static constexpr int NS = (PLAN == PLAN_MASS) ? 1 : (PLAN == PLAN_DIAG ? DIM + 1 : (DIM == 3 ? 10 : 6));
};

// Stage 1: one CTA per Gauss line (x1, x2); contract axis 0.
// Q slots, 3D: 0 Q00, 1 S00, 2 S11, 3 S22, 4 S01, 5 S02, 6 S12, 7..9 nSg0..2
//          2D: 0 Q00, 1 S00, 2 S11, 3 S01, 4 nSg0, 5 nSg1
// Stored groups, keyed by the (axis-1, axis-2) derivative patterns:
//   3D: G0 (00,00)  G1 (10,00)  G2 (11,00)  G3 (00,10)  G4 (10,01)  G5 (00,11)
//       [(01,00), (00,01), (01,10) are the pair-transposes of G1, G3, G4]
//   2D: G0 (00)  G1 (10)  G2 (11)   [(01) is the transpose of G1]
// G0, G2, G4 and G5 (2D: G0, G2) do not change when the axis-0 pair is transposed
// (their 1D factors are B_i B_j, B'_i B'_j and B'_i B_j + B_i B'_j), so each thread
// takes a canonical pair (i <= j in pair order), forms those once and writes them at
// the pair and at its transpose; G1 and G3 are formed for both, with B_i B'_j for the
// pair and B'_i B_j (the transpose's B_j B'_i) for the transpose.  The values are those
// of the per-pair contraction: the same factors in the same order.
// PLAN_DIAG (identity map, unit weights: g = 0 and S diagonal, so Q_0a and S_ab,
// a != b, vanish): G0, G2, G5 only (2D: G0, G2), from Q00 and the three diagonal S.
// PLAN_DIAGS (S diagonal at every Gauss point -- an orthogonal parametrisation such as the
// annulus, whose radial and angular directions are perpendicular and whose height is
// separate -- with rational weights): S_ab, a != b, vanish, so G4 vanishes and G1, G3 reduce
// to the weight-gradient terms B_i B_j (S g)_a, which do not change when the pair is
// transposed; gmask bit a says whether (S g)_a is nonzero (the others are skipped).
// The reaction-only plan has one contraction per output, so a CTA takes
// STAGE1_MASS_LINES consecutive axis-1 lines to give its threads enough work.
constexpr int STAGE1_MASS_LINES = 8;

template <typename T, int DIM, int P, int PLAN>
__global__ void __launch_bounds__(256) k_stage1(DirArgs d0, DirArgs d1, DirArgs d2, const double *__restrict__ geom,
                                                const double *__restrict__ Q00, GeomLayout gl, T *__restrict__ out,
                                                int gmask) {
  const T *tab = ptab<T>(d0);
  // FP64: DFMA-bound, so warps get pairs of equal overlap length; FP32: bound by memory
  // traffic, so pairs stay in pair order (neighbouring stores)
  const int *clist = sizeof(T) == 8 ? d0.pair_cs : d0.pair_c;
  if (PLAN == PLAN_MASS) {
    // lines x1 = blockIdx.x * LINES + l; each line's Q00 in shared memory
    constexpr int Q = P + 1, NQ = ipow<DIM>(Q), LINES = STAGE1_MASS_LINES;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *lines = reinterpret_cast<T *>(smem_raw);  // [LINES][X0]
    const int X0 = d0.X, x2 = blockIdx.y;
    const int e2 = x2 / Q, g2 = x2 % Q;
    const int x1a = blockIdx.x * LINES, nl = min(LINES, d1.X - x1a);
    for (int idx = threadIdx.x; idx < nl * X0; idx += blockDim.x) {
      const int l = idx / X0, x0 = idx % X0, x1 = x1a + l;
      const int e0 = x0 / Q, g0 = x0 % Q, e1 = x1 / Q, g1 = x1 % Q;
      const int64_t e = e0 + (int64_t)d0.nel * (e1 + (int64_t)d1.nel * e2);
      lines[idx] = (T)Q00[(size_t)e * NQ + g0 + Q * (g1 + Q * g2)];
    }
    __syncthreads();
    // one canonical pair per thread, all lines at once: each table value serves LINES FMAs
    for (int c = threadIdx.x; c < d0.nc; c += blockDim.x) {
      const int pi = clist[c], piT = d0.pair_T[pi];
      const int xs = d0.pair_x0[pi], np = d0.pair_np[pi];
      const T *pv = tab + (size_t)d0.pair_po[pi] * IGA_PVS;
      T acc[LINES];
#pragma unroll
      for (int l = 0; l < LINES; l++) acc[l] = 0;
      for (int k = 0; k < np; k++) {
        const T p00 = pv[IGA_PVS * k];
#pragma unroll
        for (int l = 0; l < LINES; l++) acc[l] = fma(p00, lines[l * X0 + xs + k], acc[l]);
      }
#pragma unroll
      for (int l = 0; l < LINES; l++)
        if (l < nl) {
          T *o = out + ((size_t)x2 * d1.X + x1a + l) * d0.np;
          o[pi] = acc[l];
          o[piT] = acc[l];
        }
    }
    return;
  }
  constexpr int Q = P + 1, NQ = ipow<DIM>(Q);
  using SH = Shape<PLAN, DIM>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T *line = reinterpret_cast<T *>(smem_raw);  // [NS][X0]
  const int X0 = d0.X;
  const int x1 = blockIdx.x, x2 = blockIdx.y;
  const int e1 = x1 / Q, g1 = x1 % Q, e2 = x2 / Q, g2 = x2 % Q;
  for (int idx = threadIdx.x; idx < SH::NS * X0; idx += blockDim.x) {
    int s = idx / X0, x0 = idx % X0;
    int e0 = x0 / Q, g0 = x0 % Q;
    int64_t e = e0 + (int64_t)d0.nel * (e1 + (int64_t)d1.nel * e2);
    int qp = g0 + Q * (g1 + Q * g2);
    int f;
    if (s == 0) f = -1;
    else if (PLAN == PLAN_DIAG) f = gl.S + (s - 1);
    else if (DIM == 3) f = (s <= 6) ? gl.S + (s - 1) : gl.Sg + (s - 7);
    else f = (s <= 3) ? gl.S + (s - 1) : gl.Sg + (s - 4);
    line[idx] = (T)((f < 0) ? Q00[(size_t)e * NQ + qp] : geom[((size_t)e * gl.nf + f) * NQ + qp]);
  }
  __syncthreads();
  const size_t plane = (size_t)d0.np * d1.X * (DIM == 3 ? d2.X : 1);
  T *const ol = out + ((size_t)x2 * d1.X + x1) * d0.np;
  for (int c = threadIdx.x; c < d0.nc; c += blockDim.x) {
    const int pi = clist[c], piT = d0.pair_T[pi];
    const int xs = d0.pair_x0[pi], np = d0.pair_np[pi];
    const T *pv = tab + (size_t)d0.pair_po[pi] * IGA_PVS;
    const T *L = line + xs;
    // a*: the pair's groups (G0..G5); b1, b3: G1, G3 of the transposed pair
    T a0 = 0, a1 = 0, a2 = 0, a3 = 0, a4 = 0, a5 = 0, b1 = 0, b3 = 0;
    for (int k = 0; k < np; k++) {
      const T p00 = pv[IGA_PVS * k + 0], p11 = pv[IGA_PVS * k + 3];
      if (PLAN == PLAN_DIAG) {
        a0 = fma(p00, L[k], a0);
        a0 = fma(p11, L[1 * X0 + k], a0);
        a2 = fma(p00, L[2 * X0 + k], a2);
        if (DIM == 3) a5 = fma(p00, L[3 * X0 + k], a5);
      } else if (PLAN == PLAN_DIAGS) {
        // the STIFF terms less those of the off-diagonal S (and of zero (S g)_a), in the
        // same order
        a0 = fma(p00, L[k], a0);
        if (gmask & 1) a0 = fma(pv[IGA_PVS * k + 4], L[(DIM == 3 ? 7 : 4) * X0 + k], a0);
        a0 = fma(p11, L[1 * X0 + k], a0);
        if (gmask & 2) a1 = fma(p00, L[(DIM == 3 ? 8 : 5) * X0 + k], a1);
        a2 = fma(p00, L[2 * X0 + k], a2);
        if (DIM == 3) {
          if (gmask & 4) a3 = fma(p00, L[9 * X0 + k], a3);
          a5 = fma(p00, L[3 * X0 + k], a5);
        }
      } else {
        const T p10 = pv[IGA_PVS * k + 1], p01 = pv[IGA_PVS * k + 2], psym = pv[IGA_PVS * k + 4];
        if (DIM == 3) {
          a0 = fma(p00, L[k], a0);
          a0 = fma(psym, L[7 * X0 + k], a0);
          a0 = fma(p11, L[1 * X0 + k], a0);
          a1 = fma(p00, L[8 * X0 + k], a1);
          a1 = fma(p01, L[4 * X0 + k], a1);
          b1 = fma(p00, L[8 * X0 + k], b1);
          b1 = fma(p10, L[4 * X0 + k], b1);
          a2 = fma(p00, L[2 * X0 + k], a2);
          a3 = fma(p00, L[9 * X0 + k], a3);
          a3 = fma(p01, L[5 * X0 + k], a3);
          b3 = fma(p00, L[9 * X0 + k], b3);
          b3 = fma(p10, L[5 * X0 + k], b3);
          a4 = fma(p00, L[6 * X0 + k], a4);
          a5 = fma(p00, L[3 * X0 + k], a5);
        } else {
          a0 = fma(p00, L[k], a0);
          a0 = fma(psym, L[4 * X0 + k], a0);
          a0 = fma(p11, L[1 * X0 + k], a0);
          a1 = fma(p00, L[5 * X0 + k], a1);
          a1 = fma(p01, L[3 * X0 + k], a1);
          b1 = fma(p00, L[5 * X0 + k], b1);
          b1 = fma(p10, L[3 * X0 + k], b1);
          a2 = fma(p00, L[2 * X0 + k], a2);
        }
      }
    }
    // the transposed pair's slots; for a pair that is its own transpose b1, b3 equal a1, a3
    const int pj[2] = {pi, piT};
#pragma unroll
    for (int t = 0; t < 2; t++) {
      if (t == 1 && piT == pi) break;
      T *o = ol + pj[t];
      o[0] = a0;
      o[2 * plane] = a2;
      if (PLAN == PLAN_STIFF) o[plane] = t ? b1 : a1;
      if (PLAN == PLAN_DIAGS && (gmask & 2)) o[plane] = a1;
      if (DIM == 3) {
        o[5 * plane] = a5;
        if (PLAN == PLAN_STIFF) {
          o[3 * plane] = t ? b3 : a3;
          o[4 * plane] = a4;
        }
        if (PLAN == PLAN_DIAGS && (gmask & 4)) o[3 * plane] = a3;
      }
    }
  }
}

// Stage 2 (3D): contract axis 1.  in[g1][x2][x1][pi0] -> out[g2][x2][pi1][pi0] with
//   H0 (axis-2 pattern 00) = P^00 G0 + P^10 G1 + P^01 G1^T + P^11 G2
//   H1 (axis-2 pattern 10) = P^00 G3 + P^01 G4^T
//   H2 (axis-2 pattern 11) = P^00 G5          [pattern 01 is the transpose of H1]
// H0 and H2 are unchanged when both pairs are transposed, so they are formed only
// for pi1 <= pi1T; the final stage reads them at (pi1T, pi0T) otherwise.
// PLAN_DIAG: H0 = P^00 G0 + P^11 G2, H2 = P^00 G5 (G1, G3, G4 and so H1 vanish).
// PLAN_DIAGS: G1 and G3 are transpose-invariant and G4 = 0, so
//   H0 = P^00 G0 + (P^10 + P^01) G1 + P^11 G2, H1 = P^00 G3, H2 = P^00 G5,
// with the G1 term only when (S g)_1 is nonzero and H1 only when (S g)_2 is (gmask).
template <typename T, int PLAN>
__global__ void __launch_bounds__(128, 6) k_stage2(DirArgs d0, DirArgs d1, DirArgs d2, const T *__restrict__ in,
                                                T *__restrict__ out, int chunk, int gmask) {
  const int pi0 = blockIdx.x * blockDim.x + threadIdx.x;
  const int x2 = blockIdx.z;
  const int pa = blockIdx.y * chunk, pb = min(pa + chunk, d1.np);
  if (pi0 >= d0.np) return;
  const int pi0T = d0.pair_T[pi0];
  const size_t inplane = (size_t)d0.np * d1.X * d2.X;
  const size_t outplane = (size_t)d0.np * d1.np * d2.X;
  const T *tab = ptab<T>(d1);
  for (int pi1 = pa; pi1 < pb; pi1++) {
    const bool sym = pi1 <= d1.pair_T[pi1];  // uniform across the block
    // a non-canonical pair has only H1 to form
    const bool h1_on = PLAN == PLAN_STIFF || (PLAN == PLAN_DIAGS && (gmask & 4));
    if (!sym && !h1_on) continue;
    const int xs = d1.pair_x0[pi1], np = d1.pair_np[pi1];
    const T *pv = tab + (size_t)d1.pair_po[pi1] * IGA_PVS;
    T h0 = 0, h1 = 0, h2 = 0;
    // g: this thread's entry at Gauss point xs + k of axis 1 (gT: the transposed axis-0 pair)
    const T *g = in + ((size_t)x2 * d1.X + xs) * d0.np + pi0;
    const T *gT = g - pi0 + pi0T;
#pragma unroll(sizeof(T) == 4 ? 4 : 1)
    for (int k = 0; k < np; k++, g += d0.np, gT += d0.np) {
      const T p00 = pv[IGA_PVS * k + 0];
      if (PLAN == PLAN_MASS) {
        h0 = fma(p00, g[0], h0);
      } else if (PLAN == PLAN_DIAG) {
        h0 = fma(p00, g[0], h0);
        h0 = fma(pv[IGA_PVS * k + 3], g[2 * inplane], h0);
        h2 = fma(p00, g[5 * inplane], h2);
      } else if (PLAN == PLAN_DIAGS) {
        if (sym) {
          h0 = fma(p00, g[0], h0);
          if (gmask & 2) h0 = fma(pv[IGA_PVS * k + 4], g[inplane], h0);
          h0 = fma(pv[IGA_PVS * k + 3], g[2 * inplane], h0);
          h2 = fma(p00, g[5 * inplane], h2);
        }
        if (gmask & 4) h1 = fma(p00, g[3 * inplane], h1);
      } else {
        const T p01 = pv[IGA_PVS * k + 2];
        if (sym) {
          const T p10 = pv[IGA_PVS * k + 1], p11 = pv[IGA_PVS * k + 3];
          h0 = fma(p00, g[0], h0);
          h0 = fma(p10, g[inplane], h0);
          h0 = fma(p01, gT[inplane], h0);
          h0 = fma(p11, g[2 * inplane], h0);
          h2 = fma(p00, g[5 * inplane], h2);
        }
        h1 = fma(p00, g[3 * inplane], h1);
        h1 = fma(p01, gT[4 * inplane], h1);
      }
    }
    T *o = out + ((size_t)x2 * d1.np + pi1) * d0.np + pi0;
    if (sym) o[0] = h0;
    if (h1_on) o[outplane] = h1;
    if (PLAN != PLAN_MASS && sym) o[2 * outplane] = h2;
  }
}

// Final stage: contract the last axis and write the CSR entries.
//   3D: in = T2[g2][x2][pi1][pi0];  J = P^00 H0 + P^10 H1 + P^01 H1^T + P^11 H2
//   2D: in = T1[g1][x1][pi0];       J = P^00 G0 + P^10 G1 + P^01 G1^T + P^11 G2
//   PLAN_DIAG: the H1 (2D: G1) terms vanish.
// vals = base + contribution (base optional).  fix = 1: entries in Dirichlet rows
// or columns become those of an identity row and a zeroed column instead.
// J is symmetric (Q is), so only the entries whose pair triple (pl, pmid, pi0)
// is not above its transpose (plT, pmidT, pi0T) in lexicographic order are
// contracted; each value is written at (A, B) and at (B, A).  A block walks a range
// of at most FINAL_CHUNK canonical last-axis pairs (pl <= plT) for its pmid and 128
// axis-0 pairs; everything that depends only on the last-axis pair (its overlap, its
// table rows, its functions, their Dirichlet flags, the CSR line starts of the row and
// of the transposed row) is formed once per block in shared memory.  CSR row starts come
// from the start of the row's line (i1, i2) plus the line's stencil width times the
// prefix sum of the axis-0 widths before i0.
constexpr int FINAL_CHUNK = 16;

struct FinalPair {
  int pl, skip_diag, xs, np, po, il, jl, ol, olT, wl, wlT, dirI, dirJ;
  int64_t lineA, lineB;
};

template <typename T, typename V, int DIM, int PLAN>
__global__ void __launch_bounds__(128) k_final(DirArgs d0, DirArgs d1, DirArgs d2, const T *__restrict__ in, CsrArgs csr,
                                               V *__restrict__ vals, const V *__restrict__ base, int chunk, int fix) {
  __shared__ FinalPair fp[FINAL_CHUNK];
  const int pi0 = blockIdx.x * blockDim.x + threadIdx.x;
  const bool active = pi0 < d0.np;
  const DirArgs &dl = (DIM == 3) ? d2 : d1;
  const int pmid = (DIM == 3) ? blockIdx.z : 0;
  // the block's range of canonical last-axis pairs (pair index <= its transpose's)
  const int pa = blockIdx.y * chunk, pb = min(pa + chunk, dl.nc);
  const size_t plane = (DIM == 3) ? (size_t)d0.np * d1.np * d2.X : (size_t)d0.np * d1.X;
  int i1 = 0, j1 = 0, o1 = 0, w1 = 1, pmidT = 0, o1T = 0, w1T = 1;
  if (DIM == 3) {
    i1 = d1.pair_i[pmid]; j1 = d1.pair_j[pmid];
    o1 = pmid - d1.pair_off[i1]; w1 = d1.r[i1] - d1.l[i1] + 1;
    pmidT = d1.pair_T[pmid];
    o1T = pmidT - d1.pair_off[j1]; w1T = d1.r[j1] - d1.l[j1] + 1;
  }
  const int LAX = DIM - 1;  // the last axis
  if ((int)threadIdx.x < pb - pa) {
    FinalPair &f = fp[threadIdx.x];
    const int pl = dl.pair_c[pa + threadIdx.x], plT = dl.pair_T[pl];
    f.pl = pl;
    f.skip_diag = pl == plT;  // a self-transposed pair: the triple order decides
    f.xs = dl.pair_x0[pl];
    f.np = dl.pair_np[pl];
    f.po = dl.pair_po[pl];
    const int il = dl.pair_i[pl], jl = dl.pair_j[pl];
    f.il = il;
    f.jl = jl;
    f.ol = pl - dl.pair_off[il];
    f.olT = plT - dl.pair_off[jl];
    f.wl = dl.r[il] - dl.l[il] + 1;
    f.wlT = dl.r[jl] - dl.l[jl] + 1;
    f.dirI = (csr.bnd.flag[LAX][0] && il == 0) || (csr.bnd.flag[LAX][1] && il == dl.n - 1);
    f.dirJ = (csr.bnd.flag[LAX][0] && jl == 0) || (csr.bnd.flag[LAX][1] && jl == dl.n - 1);
    f.lineA = DIM == 3 ? csr.rp_line[i1 + (int64_t)d1.n * il] : csr.rp_line[il];
    f.lineB = DIM == 3 ? csr.rp_line[j1 + (int64_t)d1.n * jl] : csr.rp_line[jl];
  }
  __syncthreads();
  if (!active) return;
  const int pi0T = d0.pair_T[pi0];
  const int i0 = d0.pair_i[pi0], j0 = d0.pair_j[pi0];
  const int o0 = pi0 - d0.pair_off[i0], w0 = d0.r[i0] - d0.l[i0] + 1;
  const int o0T = pi0T - d0.pair_off[j0], w0T = d0.r[j0] - d0.l[j0] + 1;
  const T *tab = ptab<T>(dl);
  const bool mid_sym = pmid <= pmidT;  // 3D: where stage 2 stored H0 and H2
  // Dirichlet flags of the row and column functions along the axes before the last
  bool dirI = (csr.bnd.flag[0][0] && i0 == 0) || (csr.bnd.flag[0][1] && i0 == d0.n - 1);
  bool dirJ = (csr.bnd.flag[0][0] && j0 == 0) || (csr.bnd.flag[0][1] && j0 == d0.n - 1);
  if (DIM == 3) {
    dirI = dirI || (csr.bnd.flag[1][0] && i1 == 0) || (csr.bnd.flag[1][1] && i1 == d1.n - 1);
    dirJ = dirJ || (csr.bnd.flag[1][0] && j1 == 0) || (csr.bnd.flag[1][1] && j1 == d1.n - 1);
  }
  // CSR row starts: line start (the same for the whole block at a given pl) plus the
  // row's offset within its line
  const int64_t rA0 = (int64_t)w1 * csr.rp_p0[i0], rB0 = (int64_t)w1T * csr.rp_p0[j0];
  const int64_t inA = ((int64_t)o1 * w0 + o0), inB = ((int64_t)o1T * w0T + o0T);  // 3D in-line offsets before ol
  const bool skip_self = pmid > pmidT || (pmid == pmidT && pi0 > pi0T);
  for (int c = 0; c < pb - pa; c++) {
    const FinalPair &f = fp[c];
    if (f.skip_diag && skip_self) continue;
    const int xs = f.xs, np = f.np;
    const T *pv = tab + (size_t)f.po * IGA_PVS;
    T acc = 0;
    // the stage-2 entries of this pair at its first common Gauss point; the next points
    // are one line (step) further (the same indices as r, rT = ((xs + k) n1 + pmid) n0 + pi0)
    const size_t step = (DIM == 3) ? (size_t)d1.np * d0.np : (size_t)d0.np;
    const T *ir = in + (DIM == 3 ? ((size_t)xs * d1.np + pmid) * d0.np + pi0 : (size_t)xs * d0.np + pi0);
    const T *irT = in + (DIM == 3 ? ((size_t)xs * d1.np + pmidT) * d0.np + pi0T : (size_t)xs * d0.np + pi0T);
    const T *irs = (DIM == 2 || mid_sym) ? ir : irT;
    for (int k = 0; k < np; k++, pv += IGA_PVS, ir += step, irT += step, irs += step) {
      const T p00 = pv[0];
      if (PLAN == PLAN_MASS) {
        acc = fma(p00, irs[0], acc);
      } else if (PLAN == PLAN_DIAG) {
        acc = fma(p00, irs[0], acc);
        acc = fma(pv[3], irs[2 * plane], acc);
      } else {
        const T p10 = pv[1], p01 = pv[2], p11 = pv[3];
        acc = fma(p00, irs[0], acc);
        acc = fma(p10, ir[plane], acc);
        acc = fma(p01, irT[plane], acc);
        acc = fma(p11, irs[2 * plane], acc);
      }
    }
    int64_t A, B, pos, posT;
    if (DIM == 3) {
      A = i0 + (int64_t)d0.n * (i1 + (int64_t)d1.n * f.il);
      B = j0 + (int64_t)d0.n * (j1 + (int64_t)d1.n * f.jl);
      pos = f.lineA + f.wl * rA0 + (int64_t)f.ol * w1 * w0 + inA;
      posT = f.lineB + f.wlT * rB0 + (int64_t)f.olT * w1T * w0T + inB;
    } else {
      A = i0 + (int64_t)d0.n * f.il;
      B = j0 + (int64_t)d0.n * f.jl;
      pos = f.lineA + f.wl * rA0 + (int64_t)f.ol * w0 + o0;
      posT = f.lineB + f.wlT * rB0 + (int64_t)f.olT * w0T + o0T;
    }
    if (fix && (dirI || f.dirI || dirJ || f.dirJ)) {
      const V e = (V)(A == B ? 1.0 : 0.0);  // identity row, zeroed column
      vals[pos] = e;
      vals[posT] = e;
    } else if constexpr (sizeof(V) == 4) {
      // FP32 values: the sum with the base in FP32 (one correctly rounded addition), no
      // FP64 operations on GB300's narrow FP64 pipe except the rational weights' product
      float v = (float)acc;
      if (csr.wts) v *= (float)(csr.wts[A] * csr.wts[B]);
      vals[pos] = base ? (V)(base[pos] + v) : (V)v;
      if (posT != pos) vals[posT] = base ? (V)(base[posT] + v) : (V)v;
    } else {
      double v = (double)acc;
      if (csr.wts) v *= csr.wts[A] * csr.wts[B];
      vals[pos] = base ? (V)((double)base[pos] + v) : (V)v;
      if (posT != pos) vals[posT] = base ? (V)((double)base[posT] + v) : (V)v;
    }
  }
}

#define DISPATCH_P(P_, CALL)                        \
  do {                                              \
    switch (P_) {                                   \
      case 1: { constexpr int PP = 1; CALL; } break; \
      case 2: { constexpr int PP = 2; CALL; } break; \
      case 3: { constexpr int PP = 3; CALL; } break; \
      case 4: { constexpr int PP = 4; CALL; } break; \
    }                                               \
  } while (0)

template <typename T, int DIM, int PLAN>
cudaError_t run_stage1(iga_s *h, T *T1) {
  DirArgs a0 = dir_args(h->ddev[0]), a1 = dir_args(h->ddev[1]), a2 = dir_args(h->ddev[2]);
  const int lines = (PLAN == PLAN_MASS) ? STAGE1_MASS_LINES : 1;
  dim3 grid((a1.X + lines - 1) / lines, DIM == 3 ? a2.X : 1);
  size_t sm = (size_t)(PLAN == PLAN_MASS ? lines : Shape<PLAN, DIM>::NS) * a0.X * sizeof(T);
  IGA_LAUNCH(h, KC_STAGE1, DISPATCH_P(h->p, ({
    auto kern = k_stage1<T, DIM, PP, PLAN>;
    if (sm > 48 * 1024) cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    kern<<<grid, 256, sm, h->stream>>>(a0, a1, a2, h->geom, h->Q00, h->gl, T1, h->plan_gmask);
  })));
  return cudaGetLastError();
}

template <typename T, typename V, int DIM, int PLAN>
cudaError_t run_stages(iga_s *h, V *vals, const V *base, int fix) {
  DirArgs a0 = dir_args(h->ddev[0]), a1 = dir_args(h->ddev[1]), a2 = dir_args(h->ddev[2]);
  T *T1 = (T *)h->T1, *T2 = (T *)h->T2;
  cudaError_t ce = run_stage1<T, DIM, PLAN>(h, T1);
  if (ce) return ce;
  // weights folded into the pair tables: nothing left to multiply in the final stage
  CsrArgs csr{h->rowptr, h->rp_line, h->rp_p0, h->w_folded ? nullptr : h->weights, h->bnd};
  const int chunk = 8, fchunk = FINAL_CHUNK;  // stage-2 pairs per block; final-stage canonical pairs per block
  // the final stage of PLAN_DIAGS is that of PLAN_DIAG when the last axis's weight-gradient
  // term vanishes (no H1; 2D: no G1) and that of PLAN_STIFF otherwise (its H1 and H1^T
  // reads find the transpose-invariant values at both pairs)
  const bool diag_final = PLAN == PLAN_DIAGS && !((h->plan_gmask >> (DIM - 1)) & 1);
  constexpr int FPLAN = PLAN == PLAN_DIAGS ? PLAN_STIFF : PLAN;
  if (DIM == 3) {
    dim3 g2((a0.np + 127) / 128, (a1.np + chunk - 1) / chunk, a2.X);
    IGA_LAUNCH(h, KC_STAGE2, (k_stage2<T, PLAN><<<g2, 128, 0, h->stream>>>(a0, a1, a2, T1, T2, chunk, h->plan_gmask)));
    dim3 g3((a0.np + 127) / 128, (a2.nc + fchunk - 1) / fchunk, a1.np);
    if (diag_final)
      IGA_LAUNCH(h, KC_FINAL, (k_final<T, V, 3, PLAN_DIAG><<<g3, 128, 0, h->stream>>>(a0, a1, a2, T2, csr, vals, base, fchunk, fix)));
    else
      IGA_LAUNCH(h, KC_FINAL, (k_final<T, V, 3, FPLAN><<<g3, 128, 0, h->stream>>>(a0, a1, a2, T2, csr, vals, base, fchunk, fix)));
  } else {
    dim3 g3((a0.np + 127) / 128, (a1.nc + fchunk - 1) / fchunk, 1);
    if (diag_final)
      IGA_LAUNCH(h, KC_FINAL, (k_final<T, V, 2, PLAN_DIAG><<<g3, 128, 0, h->stream>>>(a0, a1, a2, T1, csr, vals, base, fchunk, fix)));
    else
      IGA_LAUNCH(h, KC_FINAL, (k_final<T, V, 2, FPLAN><<<g3, 128, 0, h->stream>>>(a0, a1, a2, T1, csr, vals, base, fchunk, fix)));
  }
  return cudaGetLastError();
}

template <typename T, typename V>
cudaError_t jacobian(iga_s *h, const double *U, V *vals, int mode, const V *base) {
  // mode 0: full, Dirichlet-fixed; 1: stiffness only (U-independent), unfixed;
  // 2: base (a mode-1 stiffness) + reaction, Dirichlet-fixed
  // 3: full, without the Dirichlet fix (the unwrapped space of a periodic handle)
  double cs = (mode == 2) ? 0.0 : 1.0, cr = (mode == 1) ? 0.0 : 1.0;
  // mode 2 after an accepted split-residual evaluation at this U: Q00 is already there
  if (!(mode == 2 && h->q00_valid)) {
    // the FP32 Jacobian takes its reaction coefficient from FP32 arithmetic too
    cudaError_t ce = sizeof(T) == 4 ? launch_q00_f32(h, U, cs, cr) : launch_q00(h, U, cs, cr);
    if (ce) return ce;
  }
  h->q00_valid = false;
  if (mode == 2) {
    if (!base) return cudaErrorInvalidValue;
    return h->dim == 3 ? run_stages<T, V, 3, PLAN_MASS>(h, vals, base, 1) : run_stages<T, V, 2, PLAN_MASS>(h, vals, base, 1);
  }
  const int fix = (mode == 1 || mode == 3) ? 0 : 1;
  // identity map with unit weights: the geometry factors are g = 0 and a diagonal S
  if (!h->has_geom && !h->has_w)
    return h->dim == 3 ? run_stages<T, V, 3, PLAN_DIAG>(h, vals, nullptr, fix) : run_stages<T, V, 2, PLAN_DIAG>(h, vals, nullptr, fix);
  // a diagonal S at every Gauss point (classify_stiffness_plan)
  if (h->plan_diag_s && !h->plan_general)
    return h->dim == 3 ? run_stages<T, V, 3, PLAN_DIAGS>(h, vals, nullptr, fix) : run_stages<T, V, 2, PLAN_DIAGS>(h, vals, nullptr, fix);
  return h->dim == 3 ? run_stages<T, V, 3, PLAN_STIFF>(h, vals, nullptr, fix) : run_stages<T, V, 2, PLAN_STIFF>(h, vals, nullptr, fix);
}

}  // namespace

namespace {
// max |f| over every element and Gauss point for the fields S_ab and (S g)_a of the
// geometry cache: out[i] for field i of fld (as the bits of a non-negative double, whose
// integer order is the numeric one)
constexpr int CLS_MAXF = 9;
__global__ void __launch_bounds__(256) k_geom_absmax(const double *__restrict__ geom, int nf, int nq, int64_t nelem,
                                                     const int *__restrict__ fld, int nfld,
                                                     unsigned long long *__restrict__ out) {
  __shared__ unsigned long long m_s[CLS_MAXF];
  if (threadIdx.x < CLS_MAXF) m_s[threadIdx.x] = 0ull;
  __syncthreads();
  double m[CLS_MAXF];
  for (int i = 0; i < CLS_MAXF; i++) m[i] = 0.0;
  const int64_t tot = nelem * nq;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < tot; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t e = t / nq;
    const int qp = (int)(t - e * nq);
    const double *rec = geom + (size_t)e * nf * nq + qp;
    for (int i = 0; i < nfld; i++) m[i] = fmax(m[i], fabs(rec[(size_t)fld[i] * nq]));
  }
  for (int i = 0; i < nfld; i++) atomicMax(&m_s[i], (unsigned long long)__double_as_longlong(m[i]));
  __syncthreads();
  if (threadIdx.x < nfld) atomicMax(&out[threadIdx.x], m_s[threadIdx.x]);
}
}  // namespace

// The stiffness plan of a mapped or rational geometry, from the geometry cache: S is
// taken as diagonal when every off-diagonal S_ab is below 5e-13 times the largest |S_aa|,
// and (S g)_a as zero when it is below 5e-13 times the largest |S_bb| and |(S g)_b|.  An
// orthogonal parametrisation (the annulus: radial and angular directions perpendicular,
// the height separate, the weights a function of the angle alone) has these terms zero
// in exact arithmetic and at rounding level in the cache: the map's derivatives are sums
// of B-spline derivatives of size p/h that cancel, so the level grows with refinement
// (64^3 cubic annulus: off-diagonal S at 1.6e-13 of the diagonal, (S g)_0 and (S g)_2 at
// 1e-14 and 6e-14; 8^3: 1.5e-14).  Dropping terms of that relative size changes the
// Jacobian by a comparable fraction of its largest entry, below its 1e-12 FP64 parity
// tolerance; the terms the exact map has are kept.  Synchronises the stream.
cudaError_t classify_stiffness_plan(iga_s *h) {
  const int dim = h->dim, ns = dim * (dim + 1) / 2;
  const int nq = dim == 3 ? h->q * h->q * h->q : h->q * h->q;
  int fld[CLS_MAXF], nfld = 0;
  for (int i = 0; i < ns; i++) fld[nfld++] = h->gl.S + i;  // diagonal first, then S01 (, S02, S12)
  for (int a = 0; a < dim; a++) fld[nfld++] = h->gl.Sg + a;
  int *fld_d = nullptr;
  unsigned long long *out_d = nullptr;
  cudaError_t ce = cudaMalloc((void **)&fld_d, sizeof(fld));
  if (!ce) ce = cudaMalloc((void **)&out_d, CLS_MAXF * sizeof(unsigned long long));
  if (!ce) ce = cudaMemcpyAsync(fld_d, fld, sizeof(fld), cudaMemcpyHostToDevice, h->stream);
  if (!ce) ce = cudaMemsetAsync(out_d, 0, CLS_MAXF * sizeof(unsigned long long), h->stream);
  unsigned long long m[CLS_MAXF] = {0};
  if (!ce) {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int64_t want = (h->nelem * nq + 255) / 256;
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(want, (int64_t)(sms > 0 ? sms : 1) * 4));
    k_geom_absmax<<<grid, 256, 0, h->stream>>>(h->geom, h->gl.nf, nq, h->nelem, fld_d, nfld, out_d);
    ce = cudaGetLastError();
  }
  if (!ce) ce = cudaMemcpyAsync(m, out_d, sizeof(m), cudaMemcpyDeviceToHost, h->stream);
  if (!ce) ce = cudaStreamSynchronize(h->stream);
  if (fld_d) cudaFree(fld_d);
  if (out_d) cudaFree(out_d);
  if (ce) return ce;
  double v[CLS_MAXF];
  for (int i = 0; i < nfld; i++) memcpy(&v[i], &m[i], sizeof(double));
  double sdiag = 0.0, sg = 0.0, soff = 0.0;
  for (int i = 0; i < dim; i++) sdiag = std::max(sdiag, v[i]);
  for (int i = dim; i < ns; i++) soff = std::max(soff, v[i]);
  for (int a = 0; a < dim; a++) sg = std::max(sg, v[ns + a]);
  const double tau = 5e-13;
  h->plan_diag_s = std::isfinite(sdiag) && sdiag > 0.0 && soff <= tau * sdiag;
  const double gscale = std::max(sdiag, sg);
  h->plan_gmask = 0;
  for (int a = 0; a < dim; a++)
    if (!(v[ns + a] <= tau * gscale)) h->plan_gmask |= 1 << a;
  return cudaSuccess;
}

size_t jacobian_t1_groups(int dim) { return dim == 3 ? 6 : 3; }
size_t jacobian_t2_groups(int dim) { return dim == 3 ? 3 : 0; }

cudaError_t launch_jacobian64(iga_s *h, const double *U, double *vals, int mode, const double *base) {
  if (h->inner) return mode == 0 ? periodic_jacobian64(h, U, vals) : cudaErrorInvalidValue;
  return jacobian<double, double>(h, U, vals, mode, base);
}

namespace {
// y = fl32(x), two values per thread and step (nnz-sized arrays: bound by HBM)
__global__ void __launch_bounds__(256) k_round_f32(const double *__restrict__ x, float *__restrict__ y, int64_t n) {
  const int64_t n2 = n / 2, stride = (int64_t)gridDim.x * blockDim.x;
  const double2 *x2 = reinterpret_cast<const double2 *>(x);
  float2 *y2 = reinterpret_cast<float2 *>(y);
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n2; i += stride) {
    const double2 v = x2[i];
    y2[i] = make_float2((float)v.x, (float)v.y);
  }
  if (blockIdx.x == 0 && threadIdx.x == 0 && (n & 1)) y[n - 1] = (float)x[n - 1];
}
}  // namespace

cudaError_t launch_round_f32(iga_s *h, const double *x, float *y, int64_t n) {
  if (n <= 0) return cudaSuccess;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int64_t want = (n / 2 + 255) / 256;
  const int grid = (int)std::min<int64_t>(want > 0 ? want : 1, (int64_t)(sms > 0 ? sms : 1) * 8);
  IGA_LAUNCH(h, KC_VEC, (k_round_f32<<<grid, 256, 0, h->stream>>>(x, y, n)));
  return cudaGetLastError();
}

cudaError_t launch_jacobian32(iga_s *h, const double *U, float *vals, int mode, const float *base) {
  if (h->inner) return mode == 0 ? periodic_jacobian32(h, U, vals) : cudaErrorInvalidValue;
  return jacobian<float, float>(h, U, vals, mode, base);
}
