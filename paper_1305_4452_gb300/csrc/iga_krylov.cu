// Krylov kernels of libiga: CSR SpMV, Jacobi scaling, deterministic dot
// products and norms, and restarted GMRES(m) with right Jacobi preconditioning
// and classical Gram-Schmidt applied once or twice, all in FP64.  The scalar GMRES
// bookkeeping (Givens rotations, residual estimate, triangular solve) runs in
// one-thread kernels on the device; every kernel of an iteration returns at
// once when the device "done" flag is set, so the host enqueues several
// iterations between synchronisations.  Every reduction has a fixed shape and
// order, so results do not depend on scheduling.
#include <cuda_runtime.h>
#include <math.h>

#include <algorithm>
#include <stdint.h>

#include "iga_internal.h"

namespace {

constexpr int RED_THREADS = 256;
constexpr int RED_BLOCKS = 304;  // 2 x 152 SMs
constexpr int GS_THREADS = 1024;  // Gram-Schmidt passes: one block of 32 warps per SM

// GMRES scalar block layout (doubles) for restart m
struct GmLayout {
  int m;
  int H, cs, sn, g, y, flags;
  int size;
};
__host__ __device__ inline GmLayout gm_layout(int m) {
  GmLayout L;
  L.m = m;
  L.H = 0;                     // (m+1) x m, column j at H + j*(m+1)
  L.cs = L.H + (m + 1) * m;
  L.sn = L.cs + m;
  L.g = L.sn + m;              // m+1
  L.y = L.g + m + 1;           // m
  L.flags = L.y + m;           // 0: done, 1: iterations in cycle, 2: residual estimate, 3: breakdown
  L.size = L.flags + 8;
  return L;
}

__device__ __forceinline__ double warp_sum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

// block-wide sum with a fixed tree; result valid in thread 0
__device__ double block_sum(double v, double *sh) {
  int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  v = warp_sum(v);
  if (lane == 0) sh[wid] = v;
  __syncthreads();
  double r = 0.0;
  if (wid == 0) {
    r = (lane < (int)(blockDim.x >> 5)) ? sh[lane] : 0.0;
    r = warp_sum(r);
  }
  __syncthreads();
  return r;
}

// The CSR pattern is the stencil product of Sec. 4: the columns of row
// A = (i0, i1, i2) are the lexicographic product of the 1D BasisStencil ranges
// [l_d(i_d), r_d(i_d)], ascending.  The column of every stored value therefore
// follows from its position in the row, and the operator product streams the
// values and gathers x without reading column indices (8 instead of 12 bytes
// per FP64 nonzero, 4 instead of 8 per FP32 one).
struct StencilRows {
  int n0, n01;                 // functions along axis 0, along axes 0 and 1
  const int *l0, *r0, *l1, *r1, *l2, *r2;
};

struct RowShape {
  int lo0, w0, lo1, w1, lo2, w2;
};

template <int DIM>
__device__ __forceinline__ RowShape row_shape(const StencilRows &S, int row) {
  int i0, i1, i2 = 0;
  if (DIM == 3) {
    i2 = row / S.n01;
    int t = row - i2 * S.n01;
    i1 = t / S.n0;
    i0 = t - i1 * S.n0;
  } else {
    i1 = row / S.n0;
    i0 = row - i1 * S.n0;
  }
  RowShape R;
  R.lo0 = S.l0[i0];
  R.w0 = S.r0[i0] - R.lo0 + 1;
  R.lo1 = S.l1[i1];
  R.w1 = S.r1[i1] - R.lo1 + 1;
  R.lo2 = 0;
  R.w2 = 1;
  if (DIM == 3) {
    R.lo2 = S.l2[i2];
    R.w2 = S.r2[i2] - R.lo2 + 1;
  }
  return R;
}

// y = A x over the stencil CSR, LPR lanes per row.  Lane t of a row takes the
// row's entries t, t+LPR, ...; the column is advanced incrementally (a run of w0
// consecutive columns per (i1, i2) offset).  Every lane reaches the shuffles.
template <int DIM, int LPR, typename V, typename X, typename ACC>
__global__ void __launch_bounds__(256) k_spmv_stencil(StencilRows S, const int64_t *__restrict__ rowptr,
                                                      const V *__restrict__ val, const X *__restrict__ x,
                                                      double *__restrict__ y, int N, const double *__restrict__ done) {
  if (done && done[0] != 0.0) return;
  const int gid = blockIdx.x * blockDim.x + threadIdx.x;
  const int row = gid / LPR, lane = gid % LPR;
  ACC acc = 0;
  if (row < N) {
    const RowShape R = row_shape<DIM>(S, row);
    const int cnt = R.w0 * R.w1 * R.w2;
    const V *v = val + rowptr[row];
    int ii = lane, jj = 0, kk = 0;
    while (ii >= R.w0) { ii -= R.w0; jj++; }
    while (jj >= R.w1) { jj -= R.w1; kk++; }
    int col = (R.lo0 + ii) + (R.lo1 + jj) * S.n0 + (R.lo2 + kk) * S.n01;
    const int djj = S.n0 - R.w0, dkk = S.n01 - R.w1 * S.n0;
#pragma unroll 4
    for (int e = lane; e < cnt; e += LPR) {
      acc = fma((ACC)v[e], (ACC)x[col], acc);
      ii += LPR;
      col += LPR;
      while (ii >= R.w0) {
        ii -= R.w0;
        col += djj;
        if (++jj == R.w1) { jj = 0; col += dkk; }
      }
    }
  }
#pragma unroll
  for (int o = LPR / 2; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o, LPR);
  if (row < N && lane == 0) y[row] = (double)acc;
}

// y = J x for an assembled Newton Jacobian after the Dirichlet fix: a Dirichlet row is
// e_A and a Dirichlet column is zero off the diagonal.  A row of a Dirichlet function
// gives y_A = x_A; every other row runs k_spmv_stencil's loop over a contiguous part of
// its stored values: the planes of its stencil along the last axis that hold Dirichlet
// columns (a Dirichlet face of that axis: bit 2 (DIM-1) + side of dmask) are skipped by
// starting or ending the loop there.  The Dirichlet columns of the other axes are
// interleaved with the rest and are multiplied as the exact zeros they are (skipping them
// would make the value index depend on the column walk and serialise the value loads).
// The sum runs over the same values less exact zeros; rows away from the Dirichlet faces
// of the last axis take them in k_spmv_stencil's lanes and order.
template <int DIM, int LPR>
__global__ void __launch_bounds__(256) k_spmv_fixed(StencilRows S, const int64_t *__restrict__ rowptr,
                                                    const double *__restrict__ val, const double *__restrict__ x,
                                                    double *__restrict__ y, int N, const double *__restrict__ done, int dmask) {
  // launched as a programmatic dependent of the orthogonalisation (see spmv_fixed_launch):
  // its blocks may be resident before that grid ends; nothing is read before it has
  asm volatile("griddepcontrol.wait;" ::: "memory");
  if (done && done[0] != 0.0) return;
  const int gid = blockIdx.x * blockDim.x + threadIdx.x;
  const int row = gid / LPR, lane = gid % LPR;
  double acc = 0.0;
  bool dir_row = false;
  if (row < N) {
    int i0, i1, i2 = 0, n1, n2 = 1;
    if (DIM == 3) {
      i2 = row / S.n01;
      const int t = row - i2 * S.n01;
      i1 = t / S.n0;
      i0 = t - i1 * S.n0;
      n1 = S.n01 / S.n0;
      n2 = N / S.n01;
    } else {
      i1 = row / S.n0;
      i0 = row - i1 * S.n0;
      n1 = N / S.n0;
    }
    dir_row = ((dmask & 1) && i0 == 0) || ((dmask & 2) && i0 == S.n0 - 1) || ((dmask & 4) && i1 == 0) ||
              ((dmask & 8) && i1 == n1 - 1) || (DIM == 3 && (((dmask & 16) && i2 == 0) || ((dmask & 32) && i2 == n2 - 1)));
    if (!dir_row) {
      const RowShape R = row_shape<DIM>(S, row);
      // stencil planes along the last axis: [lo, lo + w) clipped to the non-Dirichlet ones
      const int lo = DIM == 3 ? R.lo2 : R.lo1, w = DIM == 3 ? R.w2 : R.w1, nl = DIM == 3 ? n2 : n1;
      const int fl = DIM == 3 ? 16 : 4, fh = DIM == 3 ? 32 : 8;
      const int p0 = ((dmask & fl) && lo == 0) ? 1 : 0;
      const int p1 = ((dmask & fh) && lo + w - 1 == nl - 1) ? w - 1 : w;
      const int plane = DIM == 3 ? R.w0 * R.w1 : R.w0;
      const int e0 = p0 * plane, e1 = p1 * plane;
      const double *v = val + rowptr[row];
      int ii = lane, jj = 0, kk = 0;
      while (ii >= R.w0) { ii -= R.w0; jj++; }
      if (DIM == 3) {
        while (jj >= R.w1) { jj -= R.w1; kk++; }
        kk += p0;
      } else {
        jj += p0;
      }
      int col = (R.lo0 + ii) + (R.lo1 + jj) * S.n0 + (R.lo2 + kk) * S.n01;
      const int djj = S.n0 - R.w0, dkk = S.n01 - R.w1 * S.n0;
      // the values stream through once per product: loaded evict-first (__ldcs), so that
      // they do not push x and the Krylov basis, which the orthogonalisation re-reads every
      // iteration, out of L2
#pragma unroll 4
      for (int e = e0 + lane; e < e1; e += LPR) {
        acc = fma(__ldcs(v + e), x[col], acc);
        ii += LPR;
        col += LPR;
        while (ii >= R.w0) {
          ii -= R.w0;
          col += djj;
          if (++jj == R.w1) {
            jj = 0;
            col += dkk;
          }
        }
      }
    }
  }
#pragma unroll
  for (int o = LPR / 2; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o, LPR);
  if (row < N && lane == 0) y[row] = dir_row ? x[row] : acc;
}

// Sliced copy of FP32 CSR values for the reduced-precision Krylov solves: rows in slices
// of 32, slot-major within a slice.  Slot s = a + WF (b + WF c) of row A = (i0, i1, i2)
// (WF = 2p+1, a < WF along axis 0, ...) holds the row's value for column
// (l0 + a, l1 + b, l2 + c) when that is inside the row's stencil, else 0; it sits at
// [(A / 32) 32 WF^DIM + 32 s + A % 32], so that one slot of a warp's 32 rows is one
// 128-byte access.  One thread per (row, slot), the writes coalesced.
__host__ __device__ __forceinline__ int64_t sl_index(int A, int s, int nslot) {
  return (int64_t)(A >> 5) * 32 * nslot + 32 * s + (A & 31);
}

template <int DIM, int P>
__global__ void __launch_bounds__(256) k_csr_to_sliced(StencilRows S, const int64_t *__restrict__ rowptr,
                                                       const float *__restrict__ csr, float *__restrict__ sl, int N) {
  // one thread per row: it reads its own CSR row front to back (each 32-byte sector serves
  // eight consecutive values through L1) and writes its slot values, which the warp's 32
  // rows of one slice store as one 128-byte line per slot
  constexpr int WF = 2 * P + 1, NC = DIM == 3 ? WF : 1, NSLOT = WF * WF * NC;
  const int A = blockIdx.x * blockDim.x + threadIdx.x;
  if (A >= (N + 31) / 32 * 32) return;
  float *o = sl + sl_index(A, 0, NSLOT);
  if (A >= N) {  // the last slice's padding rows
    for (int s = 0; s < NSLOT; s++) o[32 * s] = 0.f;
    return;
  }
  const RowShape R = row_shape<DIM>(S, A);
  const float *v = csr + rowptr[A];
  int k = 0;  // the next stored value of the row: slots run in the row's column order
  for (int c = 0; c < NC; c++)
    for (int b = 0; b < WF; b++) {
      const bool line = b < R.w1 && c < R.w2;
#pragma unroll
      for (int a = 0; a < WF; a++) {
        float x = 0.f;
        if (line && a < R.w0) x = v[k++];
        o[32 * (a + WF * (b + WF * c))] = x;
      }
    }
}

// y = A x on the sliced values, one thread per row, FP32 products and sums: each slot is
// one coalesced load of the warp's 32 values and, for rows with complete stencils, of 32
// consecutive x (the column of a slot is the row's own index plus a fixed offset).  A slot
// outside a row's stencil holds 0 and reads a clamped column of the row, so it adds
// nothing; the sum over the row's own columns runs in their CSR order.
template <int DIM, int P>
__global__ void __launch_bounds__(256) k_spmv_sliced(StencilRows S, const float *__restrict__ sl, const float *__restrict__ x,
                                                     double *__restrict__ y, int N, const double *__restrict__ done) {
  constexpr int WF = 2 * P + 1, NC = DIM == 3 ? WF : 1, NSLOT = WF * WF * NC;
  if (done && done[0] != 0.0) return;
  const int A = blockIdx.x * blockDim.x + threadIdx.x;
  if (A >= N) return;
  const RowShape R = row_shape<DIM>(S, A);
  const float *v = sl + sl_index(A, 0, NSLOT);
  float acc = 0.f;
  for (int c = 0; c < NC; c++) {
    const int cc = min(c, R.w2 - 1);
#pragma unroll
    for (int b = 0; b < WF; b++) {
      const float *xr = x + R.lo0 + (int64_t)S.n0 * (R.lo1 + min(b, R.w1 - 1)) + (int64_t)S.n01 * (R.lo2 + cc);
#pragma unroll
      for (int a = 0; a < WF; a++) acc = fmaf(__ldcs(v + 32 * (a + WF * (b + WF * c))), xr[min(a, R.w0 - 1)], acc);
    }
  }
  y[A] = (double)acc;
}

__global__ void k_cvt_f32(const double *__restrict__ x, float *__restrict__ y, int64_t N, const double *__restrict__ done) {
  if (done && done[0] != 0.0) return;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) y[i] = (float)x[i];
}

template <int DIM, typename V>
__global__ void k_diag_stencil(StencilRows S, const int64_t *__restrict__ rowptr, const V *__restrict__ val,
                               double *__restrict__ dinv, int N) {
  int row = blockIdx.x * blockDim.x + threadIdx.x;
  if (row >= N) return;
  const RowShape R = row_shape<DIM>(S, row);
  int i2 = (DIM == 3) ? row / S.n01 : 0;
  int t = row - i2 * S.n01;
  int i1 = t / S.n0, i0 = t - i1 * S.n0;
  int pos = (i0 - R.lo0) + R.w0 * ((i1 - R.lo1) + R.w1 * (DIM == 3 ? i2 - R.lo2 : 0));
  double d = (double)val[rowptr[row] + pos];
  dinv[row] = (d != 0.0) ? 1.0 / d : 1.0;
}

// partial[blk] = sum over the block's fixed row range of x*y
__global__ void __launch_bounds__(RED_THREADS) k_dot_partial(const double *__restrict__ x, const double *__restrict__ y,
                                                             double *__restrict__ partial, int64_t N, const double *__restrict__ done) {
  __shared__ double sh[32];
  if (done && done[0] != 0.0) return;
  int64_t per = (N + gridDim.x - 1) / gridDim.x;
  int64_t a = blockIdx.x * per, b = min(N, a + per);
  double acc = 0.0;
  for (int64_t r = a + threadIdx.x; r < b; r += blockDim.x) acc = fma(x[r], y[r], acc);
  acc = block_sum(acc, sh);
  if (threadIdx.x == 0) partial[blockIdx.x] = acc;
}

// out[i] (+)= sum_blk partial[i][blk] in index order (one block per i)
__global__ void __launch_bounds__(RED_THREADS) k_reduce_rows(const double *__restrict__ partial, int nb, double *__restrict__ out,
                                                             int accumulate, const double *__restrict__ done) {
  __shared__ double sh[32];
  if (done && done[0] != 0.0) return;
  int i = blockIdx.x;
  double acc = 0.0;
  for (int k = threadIdx.x; k < nb; k += blockDim.x) acc += partial[(size_t)i * nb + k];
  acc = block_sum(acc, sh);
  if (threadIdx.x == 0) out[i] = accumulate ? out[i] + acc : acc;
}

// Classical Gram-Schmidt applied twice, as three passes over a block-contiguous
// row partition (block b owns rows [b*per, min(N, (b+1)*per))), each reading the
// active basis once:
//   pass 1:  partial1[i][b] = sum over the block's rows of V[i][r] w[r]
//   pass 2:  h1 = sum_b partial1 (every block forms the same sums, in the same
//            order); H[:, j] = h1 (block 0); w -= V h1; partial2[i][b] = V[i] . w
//   pass 3:  h2 = sum_b partial2; H[:, j] += h2 (block 0); w -= V h2;
//            partial3[b] = sum of w[r]^2
//   pass 4:  (one pass, no refinement, in place of passes 2 and 3) h1 = sum_b partial1;
//            H[:, j] = h1 (block 0); w -= V h1; partial3[b] = sum of w[r]^2
// followed by k_gs_finish (norm, Givens step, next basis vector).  Dots use one
// warp per basis vector over the block's rows with w in shared memory; the
// block-local sums of the partials make the separate reduction launches
// unnecessary.  Every sum has a fixed shape and order.

// out_sh[i] = sum_{b < nb} partial[i * nb + b], i < n: eight lanes per i, lane t summing
// b = t + 8 (4 q + k) into four accumulators k (short chains of dependent FP64 adds: their
// latency, not their count, bounds this step), added as (a0 + a1) + (a2 + a3), then a fixed
// 3-level shuffle tree (the same result in every block); warps whose four columns are all
// past n skip the step, since an idle lane's FP64 add costs the narrow pipe as much as a
// busy one's
__device__ void block_sum_cols(const double *__restrict__ partial, int nb, int n, double *out_sh) {
  const int g = threadIdx.x >> 3, t = threadIdx.x & 7, ng = blockDim.x >> 3;
  for (int i0 = 0; i0 < n; i0 += ng) {
    const int i = i0 + g;
    if (i0 + ((threadIdx.x >> 5) << 2) >= n) continue;  // the whole warp's columns are past n
    double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
    if (i < n) {
      const double *pi = partial + (size_t)i * nb;
      int b = t;
      for (; b + 24 < nb; b += 32) {
        a0 += pi[b];
        a1 += pi[b + 8];
        a2 += pi[b + 16];
        a3 += pi[b + 24];
      }
      if (b < nb) a0 += pi[b];
      if (b + 8 < nb) a1 += pi[b + 8];
      if (b + 16 < nb) a2 += pi[b + 16];
    }
    double acc = (a0 + a1) + (a2 + a3);
    acc += __shfl_down_sync(0xffffffffu, acc, 4, 8);
    acc += __shfl_down_sync(0xffffffffu, acc, 2, 8);
    acc += __shfl_down_sync(0xffffffffu, acc, 1, 8);
    if (t == 0 && i < n) out_sh[i] = acc;
  }
  __syncthreads();
}

// partial[i * gridDim.x + blockIdx.x] = sum over the block's rows r < cnt of V[i][a + r] ws[r],
// i < jp1: items (column i, row chunk c), R chunks per column so that the warps are busy
// even for few columns; chunk sums in shared memory (dp, one per warp), then per column in
// order.  ws holds the block's rows of w; all threads of the block take part.
__device__ void block_dots(const double *__restrict__ Vb, int64_t ld, int jp1, int64_t a, int cnt, const double *ws,
                           double *dp, double *__restrict__ partial) {
  const int T = blockDim.x;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = T >> 5;
  const int R = jp1 >= nw ? 1 : nw / jp1;
  const int items = jp1 * R, clen = (cnt + R - 1) / R;
  for (int base = 0; base < items; base += nw) {
    const int it = base + warp;
    if (it < items) {
      const int i = it / R, c = it - i * R;
      const int r0 = c * clen, r1 = min(cnt, r0 + clen);
      const double *v = Vb + (size_t)i * ld + a;
      // four independent chains (rows r0 + lane + 32 q + 128 k, q < 4), added at the end as
      // (acc0 + acc1) + (acc2 + acc3): four loads of V in flight per lane and step, since
      // the basis comes from HBM and few warps share an SM's FP64 pipe here
      double acc0 = 0.0, acc1 = 0.0, acc2 = 0.0, acc3 = 0.0;
      int r = r0 + lane;
      for (; r + 96 < r1; r += 128) {
        const double x0 = v[r], x1 = v[r + 32], x2 = v[r + 64], x3 = v[r + 96];
        acc0 = fma(x0, ws[r], acc0);
        acc1 = fma(x1, ws[r + 32], acc1);
        acc2 = fma(x2, ws[r + 64], acc2);
        acc3 = fma(x3, ws[r + 96], acc3);
      }
      if (r < r1) acc0 = fma(v[r], ws[r], acc0);
      if (r + 32 < r1) acc1 = fma(v[r + 32], ws[r + 32], acc1);
      if (r + 64 < r1) acc2 = fma(v[r + 64], ws[r + 64], acc2);
      double acc = warp_sum((acc0 + acc1) + (acc2 + acc3));
      if (lane == 0) dp[warp] = acc;
    }
    __syncthreads();
    // columns completed in this round: items [base, base + nw)
    if (threadIdx.x < nw) {
      const int it0 = base + threadIdx.x;
      if (it0 < items && (it0 % R) == 0) {
        const int i = it0 / R;
        double acc = 0.0;
        for (int c = 0; c < R; c++) acc += dp[threadIdx.x + c];
        partial[(size_t)i * gridDim.x + blockIdx.x] = acc;
      }
    }
    __syncthreads();
  }
}

template <int PASS>
__global__ void __launch_bounds__(GS_THREADS) k_gs_pass(const double *__restrict__ Vb, int64_t ld, int jp1,
                                                        const double *__restrict__ prev, double *__restrict__ Hj,
                                                        double *__restrict__ w, double *__restrict__ partial, int64_t N,
                                                        int per, const double *__restrict__ done) {
  extern __shared__ double gs_sm[];
  double *ws = gs_sm;                   // [per]
  double *hs = gs_sm + per;             // [jp1]
  double *dp = gs_sm + per + jp1;       // [GS_THREADS / 32] dot partials of the (column, chunk) items
  __shared__ double sh[32];
  if (done[0] != 0.0) return;
  const int64_t a = (int64_t)blockIdx.x * per;
  const int cnt = (int)max((int64_t)0, min((int64_t)per, N - a));
  if (PASS >= 2) {
    block_sum_cols(prev, gridDim.x, jp1, hs);
    if (blockIdx.x == 0)
      for (int i = threadIdx.x; i < jp1; i += blockDim.x) Hj[i] = (PASS == 3) ? Hj[i] + hs[i] : hs[i];
  }
  double sq = 0.0;
  // two rows per thread and step: two independent FMA chains, their loads interleaved
  const int T = blockDim.x;
  for (int r = threadIdx.x; r < cnt; r += 2 * T) {
    const int r2 = r + T;
    const bool two = r2 < cnt;
    double v = w[a + r], v2 = two ? w[a + r2] : 0.0;
    if (PASS >= 2) {
      const double *c1 = Vb + a + r, *c2 = Vb + a + (two ? r2 : r);
#pragma unroll 4
      for (int i = 0; i < jp1; i++) {
        const double hi = hs[i];
        v = fma(-hi, c1[(size_t)i * ld], v);
        v2 = fma(-hi, c2[(size_t)i * ld], v2);
      }
      w[a + r] = v;
      if (two) w[a + r2] = v2;
    }
    if (PASS >= 3) {
      sq = fma(v, v, sq);
      if (two) sq = fma(v2, v2, sq);
    } else {
      ws[r] = v;
      if (two) ws[r2] = v2;
    }
  }
  if (PASS >= 3) {
    sq = block_sum(sq, sh);
    if (threadIdx.x == 0) partial[blockIdx.x] = sq;
    return;
  }
  __syncthreads();
  block_dots(Vb, ld, jp1, a, cnt, ws, dp, partial);
}

// v_next = w / hnorm ; z = dinv .* v_next   (skipped on breakdown)
__global__ void k_normalize(const double *w, const double *__restrict__ hn, double *vnext,
                            const double *__restrict__ dinv, double *__restrict__ z, int64_t N, const double *__restrict__ done) {
  if (done[0] != 0.0) return;
  __shared__ double inv_s;  // 1 / ||w|| once per block, not per thread
  if (threadIdx.x == 0) inv_s = (hn[0] > 0.0) ? 1.0 / hn[0] : 0.0;
  __syncthreads();
  const double inv = inv_s;
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < N; r += (int64_t)gridDim.x * blockDim.x) {
    double v = w[r] * inv;
    vnext[r] = v;
    z[r] = dinv[r] * v;
  }
}

// Givens step for column j of H, on a copy of the column and of the previous
// rotations in shared memory (Hs[0..j+1], cs_s[0..j), sn_s[0..j)), one thread, in two
// parts: givens_apply_prev rotates Hs[0..j] by the previous rotations (it needs only the
// Gram-Schmidt coefficients, so it can run before ||w|| is known) and returns the rotated
// last component t; givens_new forms the new rotation from t and H[j+1][j] = sqrt(hn2),
// writes the rotated column, the rotation, g (gj = g[j] on entry) and the flags to gm.
__device__ double givens_apply_prev(double *Hs, const double *cs_s, const double *sn_s, int j) {
  // the running component t carried in a register: one dependent FMA per rotation
  // (single-thread FP64 latency on GB300's narrow pipe is the cost here)
  double t = Hs[0];
  for (int i = 0; i < j; i++) {
    const double c = cs_s[i], s = sn_s[i], b = Hs[i + 1];
    const double cb = c * b, sb = s * b;
    Hs[i] = fma(c, t, sb);
    t = fma(-s, t, cb);
  }
  return t;
}

__device__ void givens_new(double *Hs, double t, double hn2, double gj, double *__restrict__ gm, int m, int j,
                           double tol) {
  GmLayout L = gm_layout(m);
  double *fl = gm + L.flags;
  double *Hj = gm + L.H + (size_t)j * (m + 1);
  const double hn = sqrt(hn2);
  const double a = t, b = hn;
  const double r = hypot(a, b);
  const double c = (r > 0.0) ? a / r : 1.0, s = (r > 0.0) ? b / r : 0.0;
  gm[L.cs + j] = c;
  gm[L.sn + j] = s;
  Hs[j] = r;
  Hs[j + 1] = 0.0;
  for (int i = 0; i <= j + 1; i++) Hj[i] = Hs[i];
  gm[L.g + j] = c * gj;
  gm[L.g + j + 1] = -s * gj;
  const double res = fabs(s * gj);
  fl[1] = j + 1;
  fl[2] = res;
  const bool breakdown = !(hn > 1e-300) || !isfinite(res);
  if (breakdown) fl[3] = 1.0;
  if (res <= tol || breakdown || j + 1 == m) fl[0] = 1.0;
  fl[4] = hn;
}

// H[j+1][j] arrives in Hs[j+1] as a sum of squares.
__device__ void givens_step_sm(double *Hs, const double *cs_s, const double *sn_s, double *__restrict__ gm, int m, int j,
                               double tol) {
  GmLayout L = gm_layout(m);
  const double gj = gm[L.g + j];
  const double t = givens_apply_prev(Hs, cs_s, sn_s, j);
  givens_new(Hs, t, Hs[j + 1], gj, gm, m, j, tol);
}

// End of a GMRES iteration: ||w||^2 = sum of the pass-3 partials (every block,
// same order); v_{j+1} = w / ||w||, z = dinv .* v_{j+1}; block 0 also stores
// H[j+1][j] and runs the Givens step, which sets the done flag for the kernels
// that follow (blocks of this kernel may still form v_{j+1}; it is then unused).
__global__ void __launch_bounds__(GS_THREADS) k_gs_finish(const double *__restrict__ partial, int nb, const double *w,
                                                          double *vnext, const double *__restrict__ dinv,
                                                          double *__restrict__ z, int64_t N, int per,
                                                          double *__restrict__ gm, int m, int j, double tol) {
  __shared__ double hn2;
  GmLayout L = gm_layout(m);
  if (gm[L.flags] != 0.0) return;
  if (threadIdx.x < 32) {
    double acc = 0.0;
    for (int b = threadIdx.x; b < nb; b += 32) acc += partial[b];
    acc = warp_sum(acc);
    if (threadIdx.x == 0) hn2 = acc;
  }
  __syncthreads();
  const double s2 = hn2;
  const double hn = sqrt(s2);
  const double inv = (hn > 0.0) ? 1.0 / hn : 0.0;
  const int64_t a = (int64_t)blockIdx.x * per;
  const int cnt = (int)max((int64_t)0, min((int64_t)per, N - a));
  for (int r = threadIdx.x; r < cnt; r += blockDim.x) {
    const double v = w[a + r] * inv;
    vnext[a + r] = v;
    z[a + r] = dinv[a + r] * v;
  }
  if (blockIdx.x == 0) {
    // the column and the previous rotations, loaded in parallel, then one thread rotates
    extern __shared__ double fin_sm[];
    double *Hs = fin_sm, *cs_s = Hs + (m + 2), *sn_s = cs_s + m;
    const double *Hj = gm + L.H + (size_t)j * (m + 1);
    for (int i = threadIdx.x; i <= j; i += blockDim.x) Hs[i] = Hj[i];
    for (int i = threadIdx.x; i < j; i += blockDim.x) {
      cs_s[i] = gm[L.cs + i];
      sn_s[i] = gm[L.sn + i];
    }
    if (threadIdx.x == 0) Hs[j + 1] = s2;
    __syncthreads();
    if (threadIdx.x == 0) givens_step_sm(Hs, cs_s, sn_s, gm, m, j, tol);
  }
}

// ---- one Arnoldi orthogonalisation in a single cooperative launch ----
// Flag slots of the GMRES scalar block used by the fused kernel: 6 = a grid barrier gave
// up (the solve reports IGA_ETIMEOUT).
constexpr int GS_FLAG_TIMEOUT = 6;
constexpr unsigned long long GS_BARRIER_NS = 1000000000ull;  // 1 s: far above any phase

__device__ __forceinline__ unsigned long long gs_gtimer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
  return t;
}

// Barrier over the blocks of a cooperative launch (all resident): bar[0] counts the
// arrivals, bar[1] is the generation; the last block to arrive resets the count and
// advances the generation, the others wait for that (at most GS_BARRIER_NS, then false).
// Every block's writes before the barrier are visible to every block after it.
__device__ bool gs_grid_sync(unsigned *bar) {
  __shared__ int ok_s;
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile unsigned *vgen = bar + 1;
    const unsigned gen = *vgen;
    __threadfence();
    int ok = 1;
    if (atomicAdd(bar, 1u) == gridDim.x - 1) {
      atomicExch(bar, 0u);
      __threadfence();
      atomicAdd(bar + 1, 1u);
    } else {
      const unsigned long long t0 = gs_gtimer();
      for (unsigned i = 1; *vgen == gen; i++)
        if ((i & 255) == 0 && gs_gtimer() - t0 > GS_BARRIER_NS) {
          ok = 0;
          break;
        }
    }
    __threadfence();
    ok_s = ok;
  }
  __syncthreads();
  return ok_s != 0;
}

// ws[r] -= sum_{i < jp1} h[i] V[i][a + r] for the block's rows r < cnt, taken by T threads
// numbered t0 (the rows t0 + k T), two rows per thread and step (two independent FMA
// chains sharing each h[i]); returns the thread's sum of the updated ws[r]^2 (rows in the
// order visited).
__device__ __forceinline__ double gs_update_rows(const double *__restrict__ Vb, int64_t ld, int jp1, int64_t a, int cnt,
                                                 const double *h, double *ws, int t0, int T) {
  double sq = 0.0;
  for (int r = t0; r < cnt; r += 2 * T) {
    const int r2 = r + T;
    const bool two = r2 < cnt;
    double v = ws[r], v2 = two ? ws[r2] : 0.0;
    const double *c1 = Vb + a + r, *c2 = Vb + a + (two ? r2 : r);
#pragma unroll 4
    for (int i = 0; i < jp1; i++) {
      const double hi = h[i];
      v = fma(-hi, c1[(size_t)i * ld], v);
      v2 = fma(-hi, c2[(size_t)i * ld], v2);
    }
    ws[r] = v;
    sq = fma(v, v, sq);
    if (two) {
      ws[r2] = v2;
      sq = fma(v2, v2, sq);
    }
  }
  return sq;
}

// The Gram-Schmidt passes and the end of the iteration (k_gs_pass<1..4> and k_gs_finish)
// as one kernel: classical Gram-Schmidt applied once or twice (refine, the modes of
// gmres_cgs_refine) to w = A z_j against V_0..V_j, the new column of H, v_{j+1} = w / ||w||,
// z = dinv .* v_{j+1} and the Givens step.  Blocks own the row ranges of gs_partition and
// keep their rows of w in shared memory from the first phase to the last; the phases are
// separated by grid barriers.
//   phase 1: partial1[i][b] = V_i . w over the block's rows (and, unless refine is
//            ALWAYS, partial1[j+1][b] = w . w)
//   phase 2 (second pass: always, or if needed when the first pass would remove more than
//            half of ||w||^2): h1 = sum_b partial1 (same sums in every block); w -= V h1;
//            partial2[i][b] = V_i . w, partial2[j+1][b] = w . w
//   phase 3: h2 = sum_b partial2 (with one pass: h2 = h1, and the h1 of phase 2 taken as 0);
//            H[:, j] = h1 + h2; w -= V h2 and, with s1 = ||w||^2 before this update,
//            ||w||^2 = s1 - ||h2||^2 (Pythagoras: w - V h2 is orthogonal to V h2 up to
//            rounding and the basis's loss of orthogonality) -- unless that removes more than
//            half of s1, when the norm is summed directly after one more barrier; then
//            v_{j+1}, z, Givens.
// The passes read V as the separate kernels do (2 or 4 (j+1) N values); w does not go back
// to global memory.  All blocks take the same branches (their sums are identical).
__global__ void __launch_bounds__(GS_THREADS) k_gs_fused(const double *__restrict__ Vb, int64_t ld, int j,
                                                         const double *__restrict__ w, const double *__restrict__ dinv,
                                                         double *__restrict__ z, double *__restrict__ P1,
                                                         double *__restrict__ P2, int64_t N, int per, double *__restrict__ gm,
                                                         int m, double tol, unsigned *bar, int refine) {
  extern __shared__ double fs_sm[];
  // the operator product that follows may start launching its blocks now; they wait for
  // this grid's end before reading (griddepcontrol.wait in k_spmv_fixed)
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  const int jp1 = j + 1;
  double *ws = fs_sm;                  // [per]
  double *hs = ws + per;               // [m + 2]: h1 (0 with one pass)
  double *h2 = hs + (m + 2);           // [m + 2]: h2 and s1
  double *dp = h2 + (m + 2);           // [GS_THREADS / 32]
  double *cs_s = dp + GS_THREADS / 32; // [m]
  double *sn_s = cs_s + m;             // [m]
  double *Hs = sn_s + m;               // [m + 2]
  __shared__ double sh[32];
  __shared__ double sc[4];
  GmLayout L = gm_layout(m);
  double *fl = gm + L.flags;
  if (fl[0] != 0.0) return;
  const int T = blockDim.x;
  const int64_t a = (int64_t)blockIdx.x * per;
  const int cnt = (int)max((int64_t)0, min((int64_t)per, N - a));
  bool twice = refine == IGA_CGS_REFINE_ALWAYS;
  // the partials of the direct norm: a buffer that no block still reads
  double *Pd = P2;
  // phase 1
  if (twice) {
    for (int r = threadIdx.x; r < cnt; r += T) ws[r] = w[a + r];
  } else {
    double sq = 0.0;
    for (int r = threadIdx.x; r < cnt; r += T) {
      const double v = w[a + r];
      ws[r] = v;
      sq = fma(v, v, sq);
    }
    sq = block_sum(sq, sh);
    if (threadIdx.x == 0) P1[(size_t)jp1 * gridDim.x + blockIdx.x] = sq;
  }
  __syncthreads();
  block_dots(Vb, ld, jp1, a, cnt, ws, dp, P1);
  if (!gs_grid_sync(bar)) goto timeout;
  // phase 2
  if (!twice) {
    block_sum_cols(P1, gridDim.x, jp1 + 1, h2);  // h1 and s1 = ||w||^2
    if (refine == IGA_CGS_REFINE_IFNEEDED) {
      if (threadIdx.x < 32) {
        double t = 0.0;
        for (int i = threadIdx.x; i < jp1; i += 32) t = fma(h2[i], h2[i], t);
        t = warp_sum(t);
        if (threadIdx.x == 0) sc[3] = (h2[jp1] - t > 0.5 * h2[jp1]) ? 0.0 : 1.0;
      }
      __syncthreads();
      twice = sc[3] != 0.0;
    }
    for (int i = threadIdx.x; i < jp1; i += T) hs[i] = twice ? h2[i] : 0.0;
    __syncthreads();
  } else {
    block_sum_cols(P1, gridDim.x, jp1, hs);
  }
  if (twice) {
    Pd = P1;
    {
      double sq = gs_update_rows(Vb, ld, jp1, a, cnt, hs, ws, threadIdx.x, T);
      sq = block_sum(sq, sh);
      if (threadIdx.x == 0) P2[(size_t)jp1 * gridDim.x + blockIdx.x] = sq;
    }
    __syncthreads();
    block_dots(Vb, ld, jp1, a, cnt, ws, dp, P2);
    if (!gs_grid_sync(bar)) goto timeout;
    block_sum_cols(P2, gridDim.x, jp1 + 1, h2);
  }
  // phase 3
  {
    // the block's scalars once, by warp 0 (fixed order), not by every thread: on GB300 a
    // FP64 instruction costs the narrow pipe the same for one active lane as for 32
    //   sc[0] = s2 = ||w1||^2 - ||h2||^2, sc[1] = direct, sc[2] = 1 / sqrt(s2)
    if (threadIdx.x < 32) {
      double t = 0.0;
      for (int i = threadIdx.x; i < jp1; i += 32) t = fma(h2[i], h2[i], t);
      t = warp_sum(t);
      if (threadIdx.x == 0) {
        const double s2 = h2[jp1] - t;
        const bool direct = !(s2 > 0.5 * h2[jp1]);
        const double hn = sqrt(fmax(s2, 0.0));
        sc[0] = s2;
        sc[1] = direct ? 1.0 : 0.0;
        sc[2] = (hn > 0.0) ? 1.0 / hn : 0.0;
      }
    }
    __syncthreads();
    double s2 = sc[0];
    const bool direct = sc[1] != 0.0;
    double *vnext = const_cast<double *>(Vb) + (size_t)jp1 * ld;
    // rows of this block's update and normalisation: every thread, except in block 0, whose
    // warp 0 assembles the new column of H and applies the previous rotations to it (thread
    // 0, a serial chain of dependent FP64 operations) while warps 1.. update the rows; the
    // new rotation follows at once when ||w|| is known, else after the direct norm
    int r0 = threadIdx.x, rs = T;
    double gt = 0.0, gj = 0.0;  // thread 0 of block 0: the rotated last component and g[j]
    if (blockIdx.x == 0) {
      if (threadIdx.x < 32) {
        if (threadIdx.x == 0) gj = gm[L.g + j];
        for (int i = threadIdx.x; i < jp1; i += 32) Hs[i] = hs[i] + h2[i];
        for (int i = threadIdx.x; i < j; i += 32) {
          cs_s[i] = gm[L.cs + i];
          sn_s[i] = gm[L.sn + i];
        }
        __syncwarp();
        if (threadIdx.x == 0) {
          gt = givens_apply_prev(Hs, cs_s, sn_s, j);
          if (!direct) givens_new(Hs, gt, fmax(s2, 0.0), gj, gm, m, j, tol);
        }
      }
      r0 = threadIdx.x - 32;
      rs = T - 32;
    }
    double sq = 0.0;
    if (r0 >= 0) sq = gs_update_rows(Vb, ld, jp1, a, cnt, h2, ws, r0, rs);
    if (direct) {  // severe cancellation: sum ||w||^2 itself
      sq = block_sum(sq, sh);
      if (threadIdx.x == 0) Pd[blockIdx.x] = sq;
      if (!gs_grid_sync(bar)) goto timeout;
      if (threadIdx.x < 32) {
        double acc = 0.0;
        for (int b = threadIdx.x; b < (int)gridDim.x; b += 32) acc += Pd[b];
        acc = warp_sum(acc);
        if (threadIdx.x == 0) {
          const double hn = sqrt(fmax(acc, 0.0));
          sc[0] = acc;
          sc[2] = (hn > 0.0) ? 1.0 / hn : 0.0;
        }
      }
      __syncthreads();
      s2 = sc[0];
      if (blockIdx.x == 0 && threadIdx.x == 0) givens_new(Hs, gt, fmax(s2, 0.0), gj, gm, m, j, tol);
    }
    const double inv = sc[2];
    // a thread normalises the rows it updated (the same r0, rs), so no barrier between
    if (r0 >= 0)
      for (int r = r0; r < cnt; r += rs) {
        const double v = ws[r] * inv;
        vnext[a + r] = v;
        z[a + r] = dinv[a + r] * v;
      }
  }
  return;
timeout:
  if (threadIdx.x == 0) {
    fl[GS_FLAG_TIMEOUT] = 1.0;
    fl[3] = 1.0;
    fl[0] = 1.0;
  }
}

// solve the k x k upper triangular system H y = g (k = fl[1]) by columns, one warp: from
// i = k - 1 down, y_i = g_i / H_ii (0 for a zero pivot), then g_c -= H_ci y_i for the rows
// c < i, the lanes taking the rows (on a shared copy of g).  A single thread summing each
// row took the FP64 latency of every product in turn; here a row costs one division and one
// FMA per lane.
__global__ void k_trisolve(double *__restrict__ gm, int m) {
  GmLayout L = gm_layout(m);
  __shared__ double sg[1024];
  const int k = (int)gm[L.flags + 1];
  const int lane = threadIdx.x;
  for (int i = lane; i < k; i += 32) sg[i] = gm[L.g + i];
  __syncwarp();
  for (int i = k - 1; i >= 0; i--) {
    const double *Hi = gm + L.H + (size_t)i * (m + 1);  // column i of H: H_ci, c <= i
    double yi = 0.0;
    if (lane == 0) {
      const double d = Hi[i];
      yi = (d != 0.0) ? sg[i] / d : 0.0;
      gm[L.y + i] = yi;
    }
    yi = __shfl_sync(0xffffffffu, yi, 0);
    for (int c = lane; c < i; c += 32) sg[c] -= Hi[c] * yi;
    __syncwarp();
  }
}

// x += dinv .* (sum_i y_i V[i])
__global__ void k_update_x(const double *__restrict__ Vb, int64_t ld, const double *__restrict__ gm, int m,
                           const double *__restrict__ dinv, double *__restrict__ x, int64_t N) {
  GmLayout L = gm_layout(m);
  __shared__ double ys[1024];
  int k = (int)gm[L.flags + 1];
  for (int i = threadIdx.x; i < k; i += blockDim.x) ys[i] = gm[L.y + i];
  __syncthreads();
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < N; r += (int64_t)gridDim.x * blockDim.x) {
    double acc = 0.0;
    for (int i = 0; i < k; i++) acc = fma(ys[i], Vb[(size_t)i * ld + r], acc);
    x[r] += dinv[r] * acc;
  }
}

// r = b - Ax ; then the caller normalises
__global__ void k_residual_vec(const double *__restrict__ b, const double *__restrict__ Ax, double *__restrict__ r, int64_t N) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) r[i] = b[i] - Ax[i];
}

// start a cycle: beta = sqrt(sumsq); V0 = r / beta; z = dinv V0; g = (beta, 0..); flags reset
__global__ void k_cycle_init_scalars(double *__restrict__ gm, int m, const double *__restrict__ sumsq, double tol) {
  GmLayout L = gm_layout(m);
  for (int i = threadIdx.x; i < L.size; i += blockDim.x) gm[i] = 0.0;  // the whole block clears
  __syncthreads();
  if (threadIdx.x != 0) return;
  double beta = sqrt(sumsq[0]);
  gm[L.g] = beta;
  gm[L.flags + 2] = beta;
  gm[L.flags + 4] = beta;
  if (!(beta > tol) || !isfinite(beta)) {
    gm[L.flags + 0] = 1.0;  // already converged (or NaN): nothing to do
    if (!isfinite(beta)) gm[L.flags + 3] = 1.0;
  }
}

__global__ void k_fill(double *__restrict__ x, double v, int64_t N) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) x[i] = v;
}

__global__ void k_nan_partial(const double *__restrict__ x, double *__restrict__ partial, int64_t N) {
  __shared__ double sh[32];
  int64_t per = (N + gridDim.x - 1) / gridDim.x;
  int64_t a = blockIdx.x * per, b = min(N, a + per);
  double bad = 0.0;
  for (int64_t r = a + threadIdx.x; r < b; r += blockDim.x)
    if (!isfinite(x[r])) bad = 1.0;
  bad = block_sum(bad, sh);
  if (threadIdx.x == 0) partial[blockIdx.x] = bad;
}

}  // namespace

static int grid_for(int64_t N, int threads, int cap) {
  int64_t g = (N + threads - 1) / threads;
  if (g > cap) g = cap;
  if (g < 1) g = 1;
  return (int)g;
}

static StencilRows stencil_rows(const iga_s *h) {
  StencilRows S;
  S.n0 = h->dir[0].n;
  S.n01 = h->dir[0].n * h->dir[1].n;
  S.l0 = h->ddev[0].l; S.r0 = h->ddev[0].r;
  S.l1 = h->ddev[1].l; S.r1 = h->ddev[1].r;
  S.l2 = h->dim == 3 ? h->ddev[2].l : nullptr;
  S.r2 = h->dim == 3 ? h->ddev[2].r : nullptr;
  return S;
}

// The sliced product runs one thread per row: it needs many rows to fill the GPU, and
// its sequential FP32 row sums lose accuracy with long rows ((2p+1)^3 = 729 slots at
// p = 4).  It serves p <= 2 and meshes of at least half a million rows; the CSR product
// (8 lanes per row, a tree over the lanes) serves the rest.
static bool slice_pays(const iga_s *h) { return h->p <= 2 || h->N >= 500000; }

// FP32-value operator product used by the mixed-precision Newton: x -> FP32 copy, then
// the product on the sliced copy of the values when one is current (h->J32s, made by
// launch_slice32 for h->J32), else on the CSR values (8 lanes x 4 B = one 32 B sector
// per row and step).  The operator only steers Newton (its values are rounded already);
// its FP32 sums limit the linear residual to the FP32 level, which the forcing floor of
// the reduced-precision Jacobians stays above.
static cudaError_t spmv_f32_launch(iga_s *h, const float *vals, const double *x, double *y, const double *done) {
  if (h->inner) return periodic_spmv(h, vals, 1, x, y, done);
  int eg = (int)((h->N + 255) / 256);
  if (eg > 608) eg = 608;
  IGA_LAUNCH(h, KC_VEC, (k_cvt_f32<<<eg, 256, 0, h->stream>>>(x, h->z32, h->N, done)));
  const StencilRows S = stencil_rows(h);
  const int N = (int)h->N;
  if (h->J32s && vals == h->J32 && h->J32s_valid && slice_pays(h)) {
    const unsigned gs = (unsigned)((N + 255) / 256);
    if (h->dim == 3) {
      switch (h->p) {
        case 1: IGA_LAUNCH(h, KC_SPMV, (k_spmv_sliced<3, 1><<<gs, 256, 0, h->stream>>>(S, h->J32s, h->z32, y, N, done))); break;
        case 2: IGA_LAUNCH(h, KC_SPMV, (k_spmv_sliced<3, 2><<<gs, 256, 0, h->stream>>>(S, h->J32s, h->z32, y, N, done))); break;
        case 3: IGA_LAUNCH(h, KC_SPMV, (k_spmv_sliced<3, 3><<<gs, 256, 0, h->stream>>>(S, h->J32s, h->z32, y, N, done))); break;
        default: IGA_LAUNCH(h, KC_SPMV, (k_spmv_sliced<3, 4><<<gs, 256, 0, h->stream>>>(S, h->J32s, h->z32, y, N, done))); break;
      }
    } else {
      switch (h->p) {
        case 1: IGA_LAUNCH(h, KC_SPMV, (k_spmv_sliced<2, 1><<<gs, 256, 0, h->stream>>>(S, h->J32s, h->z32, y, N, done))); break;
        case 2: IGA_LAUNCH(h, KC_SPMV, (k_spmv_sliced<2, 2><<<gs, 256, 0, h->stream>>>(S, h->J32s, h->z32, y, N, done))); break;
        case 3: IGA_LAUNCH(h, KC_SPMV, (k_spmv_sliced<2, 3><<<gs, 256, 0, h->stream>>>(S, h->J32s, h->z32, y, N, done))); break;
        default: IGA_LAUNCH(h, KC_SPMV, (k_spmv_sliced<2, 4><<<gs, 256, 0, h->stream>>>(S, h->J32s, h->z32, y, N, done))); break;
      }
    }
    return cudaGetLastError();
  }
  unsigned grid = (unsigned)(((int64_t)N * 8 + 255) / 256);
  if (h->dim == 3)
    IGA_LAUNCH(h, KC_SPMV, (k_spmv_stencil<3, 8, float, float, float><<<grid, 256, 0, h->stream>>>(S, h->rowptr, vals, h->z32, y, N, done)));
  else
    IGA_LAUNCH(h, KC_SPMV, (k_spmv_stencil<2, 8, float, float, float><<<grid, 256, 0, h->stream>>>(S, h->rowptr, vals, h->z32, y, N, done)));
  return cudaGetLastError();
}

// h->J32s = the sliced copy of the FP32 CSR values in h->J32 (allocated on first use)
cudaError_t launch_slice32(iga_s *h) {
  h->J32s_valid = false;
  if (h->inner || !slice_pays(h)) return cudaSuccess;
  const int wf = 2 * h->p + 1, nslot = h->dim == 3 ? wf * wf * wf : wf * wf;
  const int64_t total = (h->N + 31) / 32 * 32 * (int64_t)nslot;  // floats of the sliced copy
  if (!h->J32s) {
    cudaError_t ce = cudaMalloc((void **)&h->J32s, total * sizeof(float));
    if (ce) return ce;
  }
  const StencilRows S = stencil_rows(h);
  const unsigned g = (unsigned)(((h->N + 31) / 32 * 32 + 255) / 256);
  const int N = (int)h->N;
  IGA_LAUNCH(h, KC_VEC, ({
    if (h->dim == 3) {
      switch (h->p) {
        case 1: k_csr_to_sliced<3, 1><<<g, 256, 0, h->stream>>>(S, h->rowptr, h->J32, h->J32s, N); break;
        case 2: k_csr_to_sliced<3, 2><<<g, 256, 0, h->stream>>>(S, h->rowptr, h->J32, h->J32s, N); break;
        case 3: k_csr_to_sliced<3, 3><<<g, 256, 0, h->stream>>>(S, h->rowptr, h->J32, h->J32s, N); break;
        default: k_csr_to_sliced<3, 4><<<g, 256, 0, h->stream>>>(S, h->rowptr, h->J32, h->J32s, N); break;
      }
    } else {
      switch (h->p) {
        case 1: k_csr_to_sliced<2, 1><<<g, 256, 0, h->stream>>>(S, h->rowptr, h->J32, h->J32s, N); break;
        case 2: k_csr_to_sliced<2, 2><<<g, 256, 0, h->stream>>>(S, h->rowptr, h->J32, h->J32s, N); break;
        case 3: k_csr_to_sliced<2, 3><<<g, 256, 0, h->stream>>>(S, h->rowptr, h->J32, h->J32s, N); break;
        default: k_csr_to_sliced<2, 4><<<g, 256, 0, h->stream>>>(S, h->rowptr, h->J32, h->J32s, N); break;
      }
    }
  }));
  cudaError_t ce = cudaGetLastError();
  if (!ce) h->J32s_valid = true;
  return ce;
}

template <typename V>
static cudaError_t spmv_launch(iga_s *h, const V *vals, const double *x, double *y, const double *done, int cls = KC_SPMV) {
  // Few lanes per row: the cross-lane reduction costs log2(LPR) FP64 adds on every
  // lane of the group, which on GB300's narrow FP64 pipe is not free; 4 lanes keep
  // the loads sector-efficient (4 x 8 B contiguous per row and step).
  if (h->inner) return periodic_spmv(h, vals, sizeof(V) == 4, x, y, done);
  const StencilRows S = stencil_rows(h);
  const int N = (int)h->N;
  unsigned grid = (unsigned)(((int64_t)N * 4 + 255) / 256);
  if (h->dim == 3)
    IGA_LAUNCH(h, cls, (k_spmv_stencil<3, 4, V, double, double><<<grid, 256, 0, h->stream>>>(S, h->rowptr, vals, x, y, N, done)));
  else
    IGA_LAUNCH(h, cls, (k_spmv_stencil<2, 4, V, double, double><<<grid, 256, 0, h->stream>>>(S, h->rowptr, vals, x, y, N, done)));
  return cudaGetLastError();
}

// the product with an assembled, Dirichlet-fixed FP64 Newton Jacobian (k_spmv_fixed)
static cudaError_t spmv_fixed_launch(iga_s *h, const double *vals, const double *x, double *y, const double *done) {
  if (h->inner) return periodic_spmv(h, vals, false, x, y, done);
  int dmask = 0;
  for (int d = 0; d < h->dim; d++)
    for (int s = 0; s < 2; s++)
      if (h->bnd.flag[d][s]) dmask |= 1 << (2 * d + s);
  const StencilRows S = stencil_rows(h);
  const int N = (int)h->N;
  // a programmatic dependent launch: when the preceding kernel (the orthogonalisation)
  // signals early, the product's blocks become resident beside it and start the moment it
  // ends, instead of after a full launch latency
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(((int64_t)N * 4 + 255) / 256));
  cfg.blockDim = dim3(256);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = h->stream;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  cudaError_t le = cudaSuccess;
  if (h->dim == 3)
    IGA_LAUNCH(h, KC_SPMV, (le = cudaLaunchKernelEx(&cfg, k_spmv_fixed<3, 4>, S, h->rowptr, vals, x, y, N, done, dmask)));
  else
    IGA_LAUNCH(h, KC_SPMV, (le = cudaLaunchKernelEx(&cfg, k_spmv_fixed<2, 4>, S, h->rowptr, vals, x, y, N, done, dmask)));
  return le != cudaSuccess ? le : cudaGetLastError();
}

cudaError_t launch_spmv64_fixed(iga_s *h, const double *vals, const double *x, double *y) {
  return spmv_fixed_launch(h, vals, x, y, nullptr);
}

cudaError_t launch_spmv64(iga_s *h, const double *vals, const double *x, double *y) { return spmv_launch<double>(h, vals, x, y, nullptr); }
cudaError_t launch_spmv64_residual(iga_s *h, const double *vals, const double *x, double *y) {
  return spmv_launch<double>(h, vals, x, y, nullptr, KC_RES_SPMV);
}
cudaError_t launch_spmv32(iga_s *h, const float *vals, const double *x, double *y) { return spmv_launch<float>(h, vals, x, y, nullptr); }

cudaError_t launch_diag_inv(iga_s *h, const void *vals, int is_f32, double *dinv) {
  if (h->inner) return periodic_diag_inv(h, vals, is_f32, dinv);
  const StencilRows S = stencil_rows(h);
  const int N = (int)h->N;
  unsigned g = (unsigned)((N + 255) / 256);
  if (h->dim == 3) {
    if (is_f32) IGA_LAUNCH(h, KC_VEC, (k_diag_stencil<3, float><<<g, 256, 0, h->stream>>>(S, h->rowptr, (const float *)vals, dinv, N)));
    else IGA_LAUNCH(h, KC_VEC, (k_diag_stencil<3, double><<<g, 256, 0, h->stream>>>(S, h->rowptr, (const double *)vals, dinv, N)));
  } else {
    if (is_f32) IGA_LAUNCH(h, KC_VEC, (k_diag_stencil<2, float><<<g, 256, 0, h->stream>>>(S, h->rowptr, (const float *)vals, dinv, N)));
    else IGA_LAUNCH(h, KC_VEC, (k_diag_stencil<2, double><<<g, 256, 0, h->stream>>>(S, h->rowptr, (const double *)vals, dinv, N)));
  }
  return cudaGetLastError();
}

GsPartition gs_partition(int64_t N) {
  // one block per SM (the passes re-sum the previous pass's per-block partials in
  // every block, so few blocks keep that cheap); more when a block would exceed
  // 16384 rows (128 KB of shared memory for w); fewer for small systems, so that a
  // block keeps at least about one row per thread (a 16^2 mesh: one block)
  GsPartition g;
  int64_t nb = (N + 16383) / 16384;
  if (nb < 152) nb = std::min<int64_t>(152, std::max<int64_t>(nb, (N + 1023) / 1024));
  g.per = (int)((N + nb - 1) / nb);
  if (g.per < 1) g.per = 1;
  g.nb = (int)((N + g.per - 1) / g.per);
  if (g.nb < 1) g.nb = 1;
  return g;
}

// out_dev[0] = sum x^2 (deterministic)
static void sumsq(iga_s *h, const double *x, double *out_dev) {
  IGA_LAUNCH(h, KC_VEC, (k_dot_partial<<<RED_BLOCKS, RED_THREADS, 0, h->stream>>>(x, x, h->red, h->N, nullptr)));
  IGA_LAUNCH(h, KC_GMRES_SCALAR, (k_reduce_rows<<<1, RED_THREADS, 0, h->stream>>>(h->red, RED_BLOCKS, out_dev, 0, nullptr)));
}

cudaError_t launch_norm2(iga_s *h, const double *x, double *out_dev) {
  sumsq(h, x, out_dev);
  return cudaGetLastError();
}

cudaError_t launch_nan_check(iga_s *h, const double *x, double *out_dev) {
  IGA_LAUNCH(h, KC_VEC, (k_nan_partial<<<RED_BLOCKS, RED_THREADS, 0, h->stream>>>(x, h->red, h->N)));
  IGA_LAUNCH(h, KC_GMRES_SCALAR, (k_reduce_rows<<<1, RED_THREADS, 0, h->stream>>>(h->red, RED_BLOCKS, out_dev, 0, nullptr)));
  return cudaGetLastError();
}

// Restarted GMRES(m), right Jacobi preconditioning: solves A x = b from x = 0
// until ||b - A x|| <= tol_abs or maxit iterations.  Returns 0 on convergence,
// 1 when the cap was hit, 2 on breakdown/NaN, 3 when a grid barrier of the fused
// orthogonalisation gave up, -1 on a CUDA error.
// Operator of the Krylov solvers: FP64 values (kind 0), FP32 values (1), the
// matrix-free product J(U) x (2; vals unused, h->Q00 holds the reaction part at U) or
// FP64 values of a Jacobian with the Dirichlet fix (3: rows e_A, zero columns skipped)
static void apply_op(iga_s *h, const void *vals, int kind, const double *x, double *y, const double *done) {
  if (kind == 2) launch_jv(h, x, y, done);
  else if (kind == 1) spmv_f32_launch(h, (const float *)vals, x, y, done);
  else if (kind == 3) spmv_fixed_launch(h, (const double *)vals, x, y, done);
  else spmv_launch<double>(h, (const double *)vals, x, y, done);
}

__global__ void k_invert_diag(double *__restrict__ d, int64_t N) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x)
    d[i] = (d[i] != 0.0) ? 1.0 / d[i] : 1.0;
}

static void jacobi_scaling(iga_s *h, const void *vals, int kind, double *dinv) {
  if (kind == 2) {
    launch_jacobian_diagonal(h, dinv);
    IGA_LAUNCH(h, KC_VEC, (k_invert_diag<<<grid_for(h->N, 256, 4 * 152), 256, 0, h->stream>>>(dinv, h->N)));
  } else {
    launch_diag_inv(h, vals, kind == 1, dinv);
  }
}

int gmres_solve(iga_s *h, const void *vals, int is_f32, const double *b, double *x, double tol_abs, int m, int maxit,
                int refine, int *its, cudaError_t *cerr) {
  const int64_t N = h->N, ld = N;
  GmLayout L = gm_layout(m);
  double *gm = h->ctl;
  double *fl_host = h->ctl_host;
  double *dinv = h->wk + 4 * N, *z = h->wk + 5 * N, *w = h->wk + 6 * N, *tmp = h->wk + 7 * N;
  double *scal = h->wk + 8 * N;        // device scalars
  double *Vb = h->V;
  int total = 0, rc = 1;
  *cerr = cudaSuccess;
  int eg = grid_for(N, 256, 4 * 152);
  const GsPartition gs = gs_partition(N);
  {
    const int smax = (int)((gs.per + m + 1 + GS_THREADS / 32) * sizeof(double));
    if (smax > 48 * 1024) {
      cudaFuncSetAttribute(k_gs_pass<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, smax);
      cudaFuncSetAttribute(k_gs_pass<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, smax);
      cudaFuncSetAttribute(k_gs_pass<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, smax);
    }
  }
  // one cooperative launch per orthogonalisation when every block of the row partition
  // can be resident at once (one 1024-thread block per SM), else the four kernels
  const size_t fsmem = (size_t)(gs.per + 3 * (m + 2) + GS_THREADS / 32 + 2 * m) * sizeof(double);
  bool fused = false;
  if (h->gsbar && !h->gs_unfused && fsmem <= 227 * 1024) {
    int dev = 0, coop = 0, nsm = 0, per_sm = 0;
    if (fsmem > 48 * 1024) cudaFuncSetAttribute(k_gs_fused, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)fsmem);
    if (cudaGetDevice(&dev) == cudaSuccess && cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev) == cudaSuccess &&
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess &&
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_gs_fused, GS_THREADS, fsmem) == cudaSuccess)
      fused = coop && (int64_t)per_sm * nsm >= gs.nb;
    cudaGetLastError();
  }
  jacobi_scaling(h, vals, is_f32, dinv);
  IGA_LAUNCH(h, KC_VEC, (k_fill<<<eg, 256, 0, h->stream>>>(x, 0.0, N)));
  const int batch = 8;
  while (total < maxit) {
    // r = b - A x
    if (total == 0) {
      cudaMemcpyAsync(Vb, b, N * sizeof(double), cudaMemcpyDeviceToDevice, h->stream);
    } else {
      apply_op(h, vals, is_f32, x, tmp, nullptr);
      IGA_LAUNCH(h, KC_VEC, (k_residual_vec<<<eg, 256, 0, h->stream>>>(b, tmp, Vb, N)));
    }
    sumsq(h, Vb, scal);
    IGA_LAUNCH(h, KC_GMRES_SCALAR, (k_cycle_init_scalars<<<1, 256, 0, h->stream>>>(gm, m, scal, tol_abs)));
    IGA_LAUNCH(h, KC_VEC, (k_normalize<<<eg, 256, 0, h->stream>>>(Vb, gm + L.flags + 4, Vb, dinv, z, N, gm + L.flags + 5)));  // flags[5] stays 0
    int j = 0;
    bool cycle_done = false;
    while (!cycle_done) {
      int jend = j + batch < m ? j + batch : m;
      for (; j < jend; j++) {
        const double *done = gm + L.flags;
        double *Hj = gm + L.H + (size_t)j * (m + 1);
        apply_op(h, vals, is_f32, z, w, done);
        // classical Gram-Schmidt, once or twice, then norm + Givens + next vector
        const int jp1 = j + 1;
        const size_t smem = (size_t)(gs.per + jp1 + GS_THREADS / 32) * sizeof(double);
        double *P1 = h->red, *P2 = h->red + (size_t)(m + 1) * gs.nb, *P3 = h->red;
        if (fused) {
          const double *Vc = Vb;
          const double *wc = w, *dc = dinv;
          int jj = j, mm = m, per = gs.per;
          int64_t NN = N, ldd = ld;
          double tt = tol_abs;
          unsigned *bar = h->gsbar;
          int rf = refine;
          void *args[] = {(void *)&Vc, (void *)&ldd, (void *)&jj, (void *)&wc, (void *)&dc, (void *)&z, (void *)&P1,
                          (void *)&P2, (void *)&NN, (void *)&per, (void *)&gm, (void *)&mm, (void *)&tt, (void *)&bar,
                          (void *)&rf};
          cudaError_t le = cudaSuccess;
          IGA_LAUNCH(h, KC_ORTH, (le = cudaLaunchCooperativeKernel((const void *)k_gs_fused, dim3(gs.nb), dim3(GS_THREADS), args,
                                                                   fsmem, h->stream)));
          if (le != cudaSuccess) { *cerr = le; return -1; }
          continue;
        }
        // unfused: IFNEEDED refines always (the test would need the sums on the host)
        IGA_LAUNCH(h, KC_ORTH, (k_gs_pass<1><<<gs.nb, GS_THREADS, smem, h->stream>>>(Vb, ld, jp1, nullptr, Hj, w, P1, N, gs.per, done)));
        if (refine == IGA_CGS_REFINE_NEVER) {  // the norm's partials in P2: P1 is still being read
          P3 = P2;
          IGA_LAUNCH(h, KC_ORTH, (k_gs_pass<4><<<gs.nb, GS_THREADS, smem, h->stream>>>(Vb, ld, jp1, P1, Hj, w, P3, N, gs.per, done)));
        } else {
          IGA_LAUNCH(h, KC_ORTH, (k_gs_pass<2><<<gs.nb, GS_THREADS, smem, h->stream>>>(Vb, ld, jp1, P1, Hj, w, P2, N, gs.per, done)));
          IGA_LAUNCH(h, KC_ORTH, (k_gs_pass<3><<<gs.nb, GS_THREADS, smem, h->stream>>>(Vb, ld, jp1, P2, Hj, w, P3, N, gs.per, done)));
        }
        IGA_LAUNCH(h, KC_VEC, (k_gs_finish<<<gs.nb, GS_THREADS, (size_t)(3 * m + 2) * sizeof(double), h->stream>>>(
                                  P3, gs.nb, w, Vb + (size_t)(j + 1) * ld, dinv, z, N, gs.per, gm, m, j, tol_abs)));
      }
      cudaMemcpyAsync(fl_host, gm + L.flags, 8 * sizeof(double), cudaMemcpyDeviceToHost, h->stream);
      cudaError_t ce = cudaStreamSynchronize(h->stream);
      if (ce) { *cerr = ce; return -1; }
      if (fl_host[GS_FLAG_TIMEOUT] != 0.0) {  // a grid barrier gave up: reset it and report
        cudaMemsetAsync(h->gsbar, 0, 2 * sizeof(unsigned), h->stream);
        cudaStreamSynchronize(h->stream);
        *its = total + j;
        return 3;
      }
      if (fl_host[0] != 0.0 || j >= m) cycle_done = true;
    }
    int k = (int)fl_host[1];
    total += k;
    if (k > 0) {
      IGA_LAUNCH(h, KC_GMRES_SCALAR, (k_trisolve<<<1, 32, 0, h->stream>>>(gm, m)));
      IGA_LAUNCH(h, KC_VEC, (k_update_x<<<eg, 256, 0, h->stream>>>(Vb, ld, gm, m, dinv, x, N)));
    }
    if (fl_host[3] != 0.0) { rc = (fl_host[2] <= tol_abs) ? 0 : 2; break; }
    if (fl_host[2] <= tol_abs) { rc = 0; break; }
    if (k == 0) { rc = 0; break; }
  }
  cudaError_t ce = cudaGetLastError();
  if (ce) { *cerr = ce; return -1; }
  *its = total;
  return rc;
}

// ---------------------------------------------------------------------------
// Jacobi-preconditioned conjugate gradients (the -ksp_type cg solve of App. B).
// Scalars live on the device (layout below); every kernel after convergence
// returns at once, so the host synchronises only every few iterations.
// ---------------------------------------------------------------------------
namespace {
enum { CG_DONE = 0, CG_ITS, CG_RZ, CG_RR, CG_PQ, CG_ALPHA, CG_BETA, CG_RZ2, CG_RR2, CG_BRK, CG_RZB, CG_NS };
// the two slots of <r,z>, alternating by iteration parity (CG_RZ holds the first one)
__device__ __forceinline__ int cg_rz(int par) { return par ? CG_RZB : CG_RZ; }

__global__ void __launch_bounds__(RED_THREADS) k_cg_init(const double *__restrict__ b, const double *__restrict__ dinv,
                                                         double *__restrict__ x, double *__restrict__ r, double *__restrict__ p,
                                                         double *__restrict__ partial, int64_t N) {
  __shared__ double sh[32];
  int64_t per = (N + gridDim.x - 1) / gridDim.x;
  int64_t a = blockIdx.x * per, e = min(N, a + per);
  double rz = 0.0, rr = 0.0;
  for (int64_t i = a + threadIdx.x; i < e; i += blockDim.x) {
    double bi = b[i], pi = dinv[i] * bi;
    x[i] = 0.0;
    r[i] = bi;
    p[i] = pi;
    rz = fma(bi, pi, rz);
    rr = fma(bi, bi, rr);
  }
  rz = block_sum(rz, sh);
  rr = block_sum(rr, sh);
  if (threadIdx.x == 0) {
    partial[2 * blockIdx.x] = rz;
    partial[2 * blockIdx.x + 1] = rr;
  }
}

// out[0], out[1] = column sums of partial[nb][2] in index order (one block)
__global__ void __launch_bounds__(RED_THREADS) k_reduce2(const double *__restrict__ partial, int nb, double *__restrict__ out0,
                                                         double *__restrict__ out1, const double *__restrict__ done) {
  __shared__ double sh[32];
  if (done && done[0] != 0.0) return;
  double a = 0.0, c = 0.0;
  for (int k = threadIdx.x; k < nb; k += blockDim.x) {
    a += partial[2 * k];
    c += partial[2 * k + 1];
  }
  a = block_sum(a, sh);
  c = block_sum(c, sh);
  if (threadIdx.x == 0) {
    *out0 = a;
    *out1 = c;
  }
}

__global__ void k_cg_check0(double *s, double tol) {
  for (int k = 0; k < CG_NS; k++)
    if (k != CG_RZ && k != CG_RR) s[k] = 0.0;
  if (!isfinite(s[CG_RR])) { s[CG_DONE] = 1.0; s[CG_BRK] = 1.0; }
  else if (!(sqrt(s[CG_RR]) > tol)) s[CG_DONE] = 1.0;
}

// Sum of partial[k * stride + off], k < nb, in a fixed order (the same in every block);
// valid in every thread of the block
__device__ double block_sum_strided(const double *__restrict__ partial, int nb, int stride, int off, double *sh) {
  __shared__ double res;
  double v = 0.0;
  for (int k = threadIdx.x; k < nb; k += blockDim.x) v += partial[(size_t)k * stride + off];
  v = block_sum(v, sh);
  if (threadIdx.x == 0) res = v;
  __syncthreads();
  return res;
}

// One CG iteration after the operator product q = A p, in two kernels whose every block
// forms the iteration's scalars from the previous kernel's per-block partials in the
// same fixed order (so all blocks agree bit for bit) and block 0 records them:
//   k_cg_xr: alpha = <r,z> / <p,q>; x += alpha p; r -= alpha q; partials of <r,z>, <r,r>
//   k_cg_p:  converged when ||r|| <= tol; else beta = <r,z>_new / <r,z>; p = D^-1 r + beta p
// <r,z> alternates between two slots by iteration parity: block 0 writes the new value
// while the other blocks still read the old one.
__global__ void __launch_bounds__(RED_THREADS) k_cg_xr(double *__restrict__ x, double *__restrict__ r, const double *__restrict__ p,
                                                       const double *__restrict__ q, const double *__restrict__ dinv,
                                                       double *__restrict__ s, const double *__restrict__ pq_part,
                                                       double *__restrict__ partial, int nb, int par, int64_t N) {
  __shared__ double sh[32];
  if (s[CG_DONE] != 0.0) return;
  const double pq = block_sum_strided(pq_part, nb, 1, 0, sh);
  if (!(pq > 0.0) || !isfinite(pq)) {  // every block takes this branch
    if (blockIdx.x == 0 && threadIdx.x == 0) { s[CG_DONE] = 1.0; s[CG_BRK] = 1.0; }
    return;
  }
  // alpha = <r,z> / <p,q> once per block (a FP64 division in every thread would cost the
  // narrow FP64 pipe as much as a vector pass)
  __shared__ double alpha_s;
  if (threadIdx.x == 0) alpha_s = s[cg_rz(par)] / pq;  // <r,z> of this iteration
  __syncthreads();
  const double alpha = alpha_s;
  if (blockIdx.x == 0 && threadIdx.x == 0) { s[CG_PQ] = pq; s[CG_ALPHA] = alpha; }
  int64_t per = (N + gridDim.x - 1) / gridDim.x;
  int64_t a = blockIdx.x * per, e = min(N, a + per);
  double rr = 0.0, rz = 0.0;
  for (int64_t i = a + threadIdx.x; i < e; i += blockDim.x) {
    x[i] = fma(alpha, p[i], x[i]);
    double ri = fma(-alpha, q[i], r[i]);
    r[i] = ri;
    rr = fma(ri, ri, rr);
    rz = fma(ri, dinv[i] * ri, rz);
  }
  rz = block_sum(rz, sh);
  rr = block_sum(rr, sh);
  if (threadIdx.x == 0) {
    partial[2 * blockIdx.x] = rz;
    partial[2 * blockIdx.x + 1] = rr;
  }
}

__global__ void __launch_bounds__(RED_THREADS) k_cg_p(double *__restrict__ p, const double *__restrict__ r,
                                                      const double *__restrict__ dinv, double *__restrict__ s,
                                                      const double *__restrict__ partial, int nb, int par, double tol, int64_t N) {
  __shared__ double sh[32];
  if (s[CG_DONE] != 0.0) return;
  const double rz_new = block_sum_strided(partial, nb, 2, 0, sh);
  const double rr = block_sum_strided(partial, nb, 2, 1, sh);
  // the convergence test and beta once per block (thread 0), shared
  __shared__ double beta_s;
  __shared__ int conv_s;
  if (threadIdx.x == 0) {
    conv_s = isfinite(rr) && sqrt(rr) <= tol;
    beta_s = rz_new / s[cg_rz(par)];
  }
  __syncthreads();
  const bool bad = !isfinite(rr), conv = conv_s != 0;
  const double beta = beta_s;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    s[CG_ITS] += 1.0;
    s[CG_RR] = rr;
    s[CG_BETA] = beta;
    s[cg_rz(par ^ 1)] = rz_new;  // the next iteration's <r,z>
    if (bad) { s[CG_DONE] = 1.0; s[CG_BRK] = 1.0; }
    else if (conv) s[CG_DONE] = 1.0;
  }
  if (bad || conv) return;  // every block takes the same branch
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x)
    p[i] = fma(beta, p[i], dinv[i] * r[i]);
}
}  // namespace

// Returns 0 on convergence, 1 when the cap was hit, 2 on breakdown/NaN, -1 on a CUDA error.
int cg_solve(iga_s *h, const void *vals, int is_f32, const double *b, double *x, double tol_abs, int maxit, int *its,
             cudaError_t *cerr) {
  const int64_t N = h->N;
  double *s = h->ctl;
  double *dinv = h->wk + 4 * N, *r = h->wk + 5 * N, *p = h->wk + 6 * N, *q = h->wk + 7 * N;
  int eg = grid_for(N, 256, 4 * 152);
  *cerr = cudaSuccess;
  jacobi_scaling(h, vals, is_f32, dinv);
  IGA_LAUNCH(h, KC_VEC, (k_cg_init<<<RED_BLOCKS, RED_THREADS, 0, h->stream>>>(b, dinv, x, r, p, h->red, N)));
  IGA_LAUNCH(h, KC_GMRES_SCALAR, (k_reduce2<<<1, RED_THREADS, 0, h->stream>>>(h->red, RED_BLOCKS, s + CG_RZ, s + CG_RR, nullptr)));
  IGA_LAUNCH(h, KC_GMRES_SCALAR, (k_cg_check0<<<1, 1, 0, h->stream>>>(s, tol_abs)));
  const double *done = s + CG_DONE;
  const int batch = 16;
  int enq = 0;
  while (enq < maxit) {
    for (int k = 0; k < batch && enq < maxit; k++, enq++) {
      const int par = enq & 1;  // <r,z> slot of this iteration
      double *pq_part = h->red, *rz_part = h->red + RED_BLOCKS;
      apply_op(h, vals, is_f32, p, q, done);
      IGA_LAUNCH(h, KC_VEC, (k_dot_partial<<<RED_BLOCKS, RED_THREADS, 0, h->stream>>>(p, q, pq_part, N, done)));
      IGA_LAUNCH(h, KC_VEC, (k_cg_xr<<<RED_BLOCKS, RED_THREADS, 0, h->stream>>>(x, r, p, q, dinv, s, pq_part, rz_part, RED_BLOCKS,
                                                                                  par, N)));
      IGA_LAUNCH(h, KC_VEC, (k_cg_p<<<RED_BLOCKS, RED_THREADS, 0, h->stream>>>(p, r, dinv, s, rz_part, RED_BLOCKS, par, tol_abs, N)));
    }
    cudaMemcpyAsync(h->ctl_host, s, CG_NS * sizeof(double), cudaMemcpyDeviceToHost, h->stream);
    cudaError_t ce = cudaStreamSynchronize(h->stream);
    if (ce) { *cerr = ce; return -1; }
    if (h->ctl_host[CG_DONE] != 0.0) break;
  }
  cudaError_t ce = cudaGetLastError();
  if (ce) { *cerr = ce; return -1; }
  *its = (int)h->ctl_host[CG_ITS];
  if (h->ctl_host[CG_BRK] != 0.0) return 2;
  return h->ctl_host[CG_DONE] != 0.0 ? 0 : 1;
}
