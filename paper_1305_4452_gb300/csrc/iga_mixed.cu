// Mixed-precision Jacobian of libiga: element matrices contracted on the tensor
// cores with BF16 or TF32 operands and FP32 accumulation.
//
// Per element (Sec. 2.7: matrices "assembled in a similar fashion" to Algorithm 3)
//     E_ab = sum_q sum_{mu,nu} Q_{mu nu}(q) D_mu M_a(q) D_nu M_b(q)
//          = (Bt^T C)_ab,   Bt[(mu,q), a] = D_mu M_a(q),   C[(mu,q), b] = sum_nu Q_{mu nu}(q) Bt[(nu,q), b]
// is one dense (nen x 4nq) x (4nq x nen) product (27 x 108 x 27 for p = 2 in 3D,
// 64 x 256 x 64 for p = 3).  One warp forms Bt and C for its element in shared
// memory (FP32 arithmetic from the FP32 copies of the basis tables and geometry
// factors, with u and exp(u) at the Gauss points in FP32), rounds them to the
// operand type, and runs mma.sync m16n8k16 (BF16) or m16n8k8 (TF32) with FP32
// accumulators.  E goes to an element-matrix buffer; a gather kernel then adds,
// for every CSR entry, the entries of the elements shared by its row and column
// in a fixed order (no atomics), applies w_A w_B and the Dirichlet rows/columns,
// and writes FP32 values.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <float.h>
#include <stdint.h>

#include "iga_exp.h"
#include "iga_internal.h"

namespace {

template <int DIM> __host__ __device__ constexpr int ipow(int b) { return DIM == 2 ? b * b : b * b * b; }
__host__ __device__ constexpr int rup(int x, int m) { return (x + m - 1) / m * m; }


template <int DIM, int P>
__global__ void k_geom32(const double *__restrict__ geom, GeomLayout gl, float *__restrict__ g32, int64_t nelem) {
  constexpr int NQ = ipow<DIM>(P + 1);
  using L = G32<DIM>;
  int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= nelem * NQ) return;
  int64_t e = t / NQ;
  int qp = (int)(t % NQ);
  const double *rec = geom + (size_t)e * gl.nf * NQ + qp;
  float *o = g32 + (size_t)e * L::NF * NQ + qp;
  o[L::INVW * NQ] = (float)rec[gl.invW * NQ];
  o[L::GSG * NQ] = (float)rec[gl.gSg * NQ];
  o[L::JWW2 * NQ] = (float)rec[gl.jwW2 * NQ];
  for (int k = 0; k < L::NS; k++) o[(L::S + k) * NQ] = (float)rec[(gl.S + k) * NQ];
  for (int k = 0; k < DIM; k++) o[(L::NSG + k) * NQ] = (float)rec[(gl.Sg + k) * NQ];
}

__global__ void k_to_f32(const double *__restrict__ x, float *__restrict__ y, int64_t n) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) y[i] = (float)x[i];
}

enum { OP_BF16 = 0, OP_TF32 = 1 };

template <int OP> struct Op;
template <> struct Op<OP_BF16> {
  using T = __nv_bfloat16;
  static constexpr int KSTEP = 16, PAD = 8;
  __device__ static T cvt(float x) { return __float2bfloat16_rn(x); }
};
template <> struct Op<OP_TF32> {
  using T = uint32_t;
  static constexpr int KSTEP = 8, PAD = 4;
  __device__ static T cvt(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return r;
  }
};

template <int DIM, int P, int OP> struct TcShape {
  static constexpr int N1 = P + 1, Q = P + 1;
  static constexpr int NEN = ipow<DIM>(N1), NQ = ipow<DIM>(Q);
  static constexpr int M = rup(NEN, 16);             // rows (test functions), padded
  static constexpr int NN = rup(NEN, 8);             // columns (trial functions), padded
  static constexpr int K = rup((DIM + 1) * NQ, Op<OP>::KSTEP);
  static constexpr int LD = K + Op<OP>::PAD;         // row stride of the K-contiguous operands
  static constexpr int TAB = DIM * Q * N1 * 2;       // FP32 tables
  static constexpr int NSLOT = G32<DIM>::NF;
  // per-warp shared memory (bytes)
  static constexpr size_t OPS = (size_t)(M + NN) * LD * sizeof(typename Op<OP>::T);
  static constexpr size_t F32 = (size_t)(TAB + NEN + 2 * NQ * (DIM == 3 ? 2 : 1) + NSLOT * NQ + NQ) * sizeof(float);
  static constexpr size_t PER = (OPS + F32 + 15) / 16 * 16;
};

template <int OP>
__device__ __forceinline__ void mma_tile(float *d, const uint32_t *a, const uint32_t *b);
template <>
__device__ __forceinline__ void mma_tile<OP_BF16>(float *d, const uint32_t *a, const uint32_t *b) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}
template <>
__device__ __forceinline__ void mma_tile<OP_TF32>(float *d, const uint32_t *a, const uint32_t *b) {
  asm volatile(
      "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// One warp per element; WPB warps per CTA.
template <int DIM, int P, int OP, int WPB>
__global__ void __launch_bounds__(32 * WPB) k_elem_tc(DirArgs d0, DirArgs d1, DirArgs d2, const float *__restrict__ tab0,
                                                      const float *__restrict__ tab1, const float *__restrict__ tab2,
                                                      const double *__restrict__ U, const double *__restrict__ wts,
                                                      const float *__restrict__ g32, float lambda, float cs, float cr,
                                                      float *__restrict__ Ebuf, int64_t nelem) {
  using S = TcShape<DIM, P, OP>;
  using T = typename Op<OP>::T;
  using GL = G32<DIM>;
  constexpr int N1 = S::N1, Q = S::Q, NEN = S::NEN, NQ = S::NQ;
  extern __shared__ __align__(16) unsigned char smem[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t e = (int64_t)blockIdx.x * WPB + warp;
  if (e >= nelem) return;  // whole warp leaves together (no block-wide barrier below)
  unsigned char *base = smem + (size_t)warp * S::PER;
  T *As = reinterpret_cast<T *>(base);           // [M][LD]   A = Bt^T  (test functions x (mu,q))
  T *Bs = As + (size_t)S::M * S::LD;              // [NN][LD]  B^T = C^T (trial functions x (mu,q))
  float *tab = reinterpret_cast<float *>(Bs + (size_t)S::NN * S::LD);  // [DIM][Q][N1][2]
  float *Ue = tab + S::TAB;                       // [NEN]
  float *w1 = Ue + NEN;                           // interpolation scratch
  float *w2 = w1 + NQ;
  float *gq = w2 + NQ * (DIM == 3 ? 1 : 0) + NQ;  // [NSLOT][NQ] geometry slots
  float *q00 = gq + S::NSLOT * NQ;                // [NQ]
  const int e0 = (int)(e % d0.nel), e1 = (int)((e / d0.nel) % d1.nel), e2 = (DIM == 3) ? (int)(e / ((int64_t)d0.nel * d1.nel)) : 0;
  for (int k = lane; k < S::TAB; k += 32) {
    int ax = k / (Q * N1 * 2), r = k % (Q * N1 * 2);
    const float *src = ax == 0 ? tab0 + (size_t)e0 * Q * N1 * 2 : (ax == 1 ? tab1 + (size_t)e1 * Q * N1 * 2 : tab2 + (size_t)e2 * Q * N1 * 2);
    tab[k] = src[r];
  }
  const int f0 = d0.first[e0], f1 = d1.first[e1], f2 = (DIM == 3) ? d2.first[e2] : 0;
  for (int a = lane; a < NEN; a += 32) {
    int a0 = a % N1, a1 = (a / N1) % N1, a2 = (DIM == 3) ? a / (N1 * N1) : 0;
    int64_t G = (f0 + a0) + (int64_t)d0.n * ((f1 + a1) + (int64_t)d1.n * (f2 + a2));
    Ue[a] = (U && cr != 0.f) ? (float)(U[G] * (wts ? wts[G] : 1.0)) : 0.f;
  }
  const float *grec = g32 + (size_t)e * GL::NF * NQ;
  for (int k = lane; k < GL::NF * NQ; k += 32) gq[k] = grec[k];
  __syncwarp();
#define TB(ax, g, a, s) tab[(((ax) * Q + (g)) * N1 + (a)) * 2 + (s)]
  // u~ at the Gauss points (sum factorisation, values only), then Q00
  if (DIM == 3) {
    for (int r = lane; r < N1 * N1 * Q; r += 32) {  // [a2][a1][g0]
      int a2 = r / (N1 * Q), a1 = (r / Q) % N1, g0 = r % Q;
      float acc = 0.f;
      for (int a0 = 0; a0 < N1; a0++) acc = fmaf(TB(0, g0, a0, 0), Ue[(a2 * N1 + a1) * N1 + a0], acc);
      w1[r] = acc;
    }
    __syncwarp();
    for (int r = lane; r < N1 * Q * Q; r += 32) {  // [a2][g1][g0]
      int a2 = r / (Q * Q), g1 = (r / Q) % Q, g0 = r % Q;
      float acc = 0.f;
      for (int a1 = 0; a1 < N1; a1++) acc = fmaf(TB(1, g1, a1, 0), w1[(a2 * N1 + a1) * Q + g0], acc);
      w2[r] = acc;
    }
    __syncwarp();
  } else {
    for (int r = lane; r < N1 * Q; r += 32) {  // [a1][g0]
      int a1 = r / Q, g0 = r % Q;
      float acc = 0.f;
      for (int a0 = 0; a0 < N1; a0++) acc = fmaf(TB(0, g0, a0, 0), Ue[a1 * N1 + a0], acc);
      w2[r] = acc;
    }
    __syncwarp();
  }
  for (int qp = lane; qp < NQ; qp += 32) {
    float ut = 0.f;
    if (DIM == 3) {
      int g2 = qp / (Q * Q), g1 = (qp / Q) % Q, g0 = qp % Q;
      for (int a2 = 0; a2 < N1; a2++) ut = fmaf(TB(2, g2, a2, 0), w2[(a2 * Q + g1) * Q + g0], ut);
    } else {
      int g1 = qp / Q, g0 = qp % Q;
      for (int a1 = 0; a1 < N1; a1++) ut = fmaf(TB(1, g1, a1, 0), w2[a1 * Q + g0], ut);
    }
    float v = cs * gq[GL::GSG * NQ + qp];
    if (cr != 0.f) v -= cr * gq[GL::JWW2 * NQ + qp] * lambda * expf(ut * gq[GL::INVW * NQ + qp]);
    q00[qp] = v;
  }
  __syncwarp();
  // operands: A[a][(mu,q)] = D_mu M_a(q);  B^T[b][(mu,q)] = sum_nu Q_{mu nu}(q) D_nu M_b(q)
  // one (function, Gauss point) pair per iteration: its DIM+1 basis products and
  // the DIM+1 entries of Q D are written to the K-slots mu*NQ + q of row a
  for (int idx = lane; idx < NEN * NQ; idx += 32) {
    int a = idx / NQ, qp = idx % NQ;
    int a0 = a % N1, a1 = (a / N1) % N1, a2 = (DIM == 3) ? a / (N1 * N1) : 0;
    int g0 = qp % Q, g1 = (qp / Q) % Q, g2 = (DIM == 3) ? qp / (Q * Q) : 0;
    float b0 = TB(0, g0, a0, 0), b1 = TB(1, g1, a1, 0), b2 = (DIM == 3) ? TB(2, g2, a2, 0) : 1.f;
    float db0 = TB(0, g0, a0, 1), db1 = TB(1, g1, a1, 1), db2 = (DIM == 3) ? TB(2, g2, a2, 1) : 0.f;
    float D[4] = {b0 * b1 * b2, db0 * b1 * b2, b0 * db1 * b2, b0 * b1 * db2};
    const float *g = gq + qp;
    float vb[4];
    if (DIM == 3) {
      // S slots 00,11,22,01,02,12; Q_0a = nSg_a; Q_ab = S_ab
      float s00 = g[(GL::S + 0) * NQ], s11 = g[(GL::S + 1) * NQ], s22 = g[(GL::S + 2) * NQ];
      float s01 = g[(GL::S + 3) * NQ], s02 = g[(GL::S + 4) * NQ], s12 = g[(GL::S + 5) * NQ];
      float n0 = g[(GL::NSG + 0) * NQ], n1 = g[(GL::NSG + 1) * NQ], n2 = g[(GL::NSG + 2) * NQ];
      float qq = q00[qp];
      vb[0] = qq * D[0] + n0 * D[1] + n1 * D[2] + n2 * D[3];
      vb[1] = n0 * D[0] + s00 * D[1] + s01 * D[2] + s02 * D[3];
      vb[2] = n1 * D[0] + s01 * D[1] + s11 * D[2] + s12 * D[3];
      vb[3] = n2 * D[0] + s02 * D[1] + s12 * D[2] + s22 * D[3];
    } else {
      float s00 = g[(GL::S + 0) * NQ], s11 = g[(GL::S + 1) * NQ], s01 = g[(GL::S + 2) * NQ];
      float n0 = g[(GL::NSG + 0) * NQ], n1 = g[(GL::NSG + 1) * NQ];
      float qq = q00[qp];
      vb[0] = qq * D[0] + n0 * D[1] + n1 * D[2];
      vb[1] = n0 * D[0] + s00 * D[1] + s01 * D[2];
      vb[2] = n1 * D[0] + s01 * D[1] + s11 * D[2];
    }
#pragma unroll
    for (int mu = 0; mu <= DIM; mu++) {
      As[(size_t)a * S::LD + mu * NQ + qp] = Op<OP>::cvt(D[mu]);
      Bs[(size_t)a * S::LD + mu * NQ + qp] = Op<OP>::cvt(vb[mu]);
    }
  }
  // zero padding: columns (DIM+1)*NQ .. K-1 of every row, and rows NEN.. of both operands
  constexpr int KV = (DIM + 1) * NQ;
  if constexpr (S::K > KV) {
    for (int idx = lane; idx < NEN * (S::K - KV); idx += 32) {
      int a = idx / (S::K - KV), k = KV + idx % (S::K - KV);
      As[(size_t)a * S::LD + k] = Op<OP>::cvt(0.f);
      Bs[(size_t)a * S::LD + k] = Op<OP>::cvt(0.f);
    }
  }
  for (int idx = lane; idx < (S::M - NEN) * S::K; idx += 32) {
    int a = NEN + idx / S::K, k = idx % S::K;
    As[(size_t)a * S::LD + k] = Op<OP>::cvt(0.f);
    if (a < S::NN) Bs[(size_t)a * S::LD + k] = Op<OP>::cvt(0.f);
  }
#undef TB
  __syncwarp();
  // E = A (M x K) * B (K x NN), FP32 accumulators; tiles m16 x n8
  constexpr int MT = S::M / 16, NT = S::NN / 8;
  const int g = lane >> 2, t = lane & 3;
  float *Eo = Ebuf + (size_t)e * NEN * NEN;
  for (int mt = 0; mt < MT; mt++) {
    float acc[NT][4];
#pragma unroll
    for (int nt = 0; nt < NT; nt++) acc[nt][0] = acc[nt][1] = acc[nt][2] = acc[nt][3] = 0.f;
    for (int k0 = 0; k0 < S::K; k0 += Op<OP>::KSTEP) {
      uint32_t af[4];
      if (OP == OP_BF16) {
        const T *r0 = As + (size_t)(mt * 16 + g) * S::LD + k0 + 2 * t;
        const T *r1 = r0 + 8 * S::LD;
        af[0] = *reinterpret_cast<const uint32_t *>(r0);
        af[1] = *reinterpret_cast<const uint32_t *>(r1);
        af[2] = *reinterpret_cast<const uint32_t *>(r0 + 8);
        af[3] = *reinterpret_cast<const uint32_t *>(r1 + 8);
      } else {
        const T *r0 = As + (size_t)(mt * 16 + g) * S::LD + k0 + t;
        const T *r1 = r0 + 8 * S::LD;
        af[0] = *reinterpret_cast<const uint32_t *>(r0);
        af[1] = *reinterpret_cast<const uint32_t *>(r1);
        af[2] = *reinterpret_cast<const uint32_t *>(r0 + 4);
        af[3] = *reinterpret_cast<const uint32_t *>(r1 + 4);
      }
#pragma unroll
      for (int nt = 0; nt < NT; nt++) {
        uint32_t bf[2];
        if (OP == OP_BF16) {
          const T *c0 = Bs + (size_t)(nt * 8 + g) * S::LD + k0 + 2 * t;
          bf[0] = *reinterpret_cast<const uint32_t *>(c0);
          bf[1] = *reinterpret_cast<const uint32_t *>(c0 + 8);
        } else {
          const T *c0 = Bs + (size_t)(nt * 8 + g) * S::LD + k0 + t;
          bf[0] = *reinterpret_cast<const uint32_t *>(c0);
          bf[1] = *reinterpret_cast<const uint32_t *>(c0 + 4);
        }
        mma_tile<OP>(acc[nt], af, bf);
      }
    }
#pragma unroll
    for (int nt = 0; nt < NT; nt++) {
      int r0 = mt * 16 + g, c = nt * 8 + 2 * t;
      if (r0 < NEN) {
        if (c < NEN) Eo[(size_t)r0 * NEN + c] = acc[nt][0];
        if (c + 1 < NEN) Eo[(size_t)r0 * NEN + c + 1] = acc[nt][1];
      }
      if (r0 + 8 < NEN) {
        if (c < NEN) Eo[(size_t)(r0 + 8) * NEN + c] = acc[nt][2];
        if (c + 1 < NEN) Eo[(size_t)(r0 + 8) * NEN + c + 1] = acc[nt][3];
      }
    }
  }
}

__device__ __forceinline__ bool on_dirichlet(const BndArgs &b, int dim, const int *i, const int *n) {
  bool on = false;
  for (int ax = 0; ax < dim; ax++) {
    if (b.flag[ax][0] && i[ax] == 0) on = true;
    if (b.flag[ax][1] && i[ax] == n[ax] - 1) on = true;
  }
  return on;
}

// One warp per CSR row A.  For every element containing A (e2, e1, e0 ascending)
// the warp reads that element's row a(A) -- NEN contiguous floats -- and adds each
// value into the row accumulator in shared memory at the position of its column;
// within one element the columns are distinct, so every entry is summed in element
// order.  The finished row (weights, Dirichlet) is written contiguously.
template <int DIM, int P, typename T = float>
__global__ void __launch_bounds__(256) k_gather_elem(DirArgs d0, DirArgs d1, DirArgs d2, const T *__restrict__ Ebuf,
                                                     const int64_t *__restrict__ rowptr, const double *__restrict__ wts,
                                                     BndArgs bnd, T *__restrict__ vals, int64_t N) {
  constexpr int N1 = P + 1, NEN = ipow<DIM>(N1), RMAX = ipow<DIM>(2 * P + 1);
  __shared__ T rowacc[8][RMAX];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t A = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  if (A >= N) return;
  T *acc = rowacc[warp];
  int I[3] = {(int)(A % d0.n), (int)((A / d0.n) % d1.n), (DIM == 3) ? (int)(A / ((int64_t)d0.n * d1.n)) : 0};
  int n[3] = {d0.n, d1.n, d2.n};
  int l[3] = {d0.l[I[0]], d1.l[I[1]], DIM == 3 ? d2.l[I[2]] : 0};
  int w[3] = {d0.r[I[0]] - l[0] + 1, d1.r[I[1]] - l[1] + 1, DIM == 3 ? d2.r[I[2]] - l[2] + 1 : 1};
  const int len = w[0] * w[1] * w[2];
  for (int k = lane; k < len; k += 32) acc[k] = (T)0;
  __syncwarp();
  const int lo2 = (DIM == 3) ? d2.node_e0[I[2]] : 0, hi2 = (DIM == 3) ? lo2 + d2.node_ne[I[2]] : 1;
  const int lo1 = d1.node_e0[I[1]], hi1 = lo1 + d1.node_ne[I[1]];
  const int lo0 = d0.node_e0[I[0]], hi0 = lo0 + d0.node_ne[I[0]];
  for (int e2 = lo2; e2 < hi2; e2++) {
    const int f2 = (DIM == 3) ? d2.first[e2] : 0;
    for (int e1 = lo1; e1 < hi1; e1++) {
      const int f1 = d1.first[e1];
      for (int e0 = lo0; e0 < hi0; e0++) {
        const int f0 = d0.first[e0];
        const int64_t e = e0 + (int64_t)d0.nel * (e1 + (int64_t)d1.nel * e2);
        const int a = (I[0] - f0) + N1 * ((I[1] - f1) + N1 * (I[2] - f2));
        const T *Er = Ebuf + (size_t)e * NEN * NEN + (size_t)a * NEN;
        for (int b = lane; b < NEN; b += 32) {
          int b0 = b % N1, b1 = (b / N1) % N1, b2 = (DIM == 3) ? b / (N1 * N1) : 0;
          int pos = ((f2 + b2 - l[2]) * w[1] + (f1 + b1 - l[1])) * w[0] + (f0 + b0 - l[0]);
          acc[pos] += Er[b];
        }
        __syncwarp();
      }
    }
  }
  const bool rowfix = on_dirichlet(bnd, DIM, I, n);
  const T wA = wts ? (T)wts[A] : (T)1;
  const int64_t r0 = rowptr[A];
  for (int k = lane; k < len; k += 32) {
    int J[3] = {l[0] + k % w[0], l[1] + (k / w[0]) % w[1], l[2] + k / (w[0] * w[1])};
    int64_t B = J[0] + (int64_t)d0.n * (J[1] + (int64_t)d1.n * J[2]);
    T v = acc[k];
    if (wts) v *= wA * (T)wts[B];
    if (rowfix || on_dirichlet(bnd, DIM, J, n)) v = (A == B) ? (T)1 : (T)0;
    vals[r0 + k] = v;
  }
}

// ---------------------------------------------------------------------------
// Local numerical differentiation (Sec. 2.8, Eq. fdjac): per element, per Gauss
// point q and element value k, the integrand F_q(U_e + delta e_k) - F_q(U_e) over
// delta, delta = sqrt(eps) sqrt(1 + ||U_e||_2), summed over q into the element
// matrix E[a][k] (weights included), then gathered per row like the tensor-core
// element matrices.  The integrand is the factored form of the residual
// (F_q,a = w_a (grad M_a . v + M_a s), v = S (grad u~ - u~ g), s = -g . v -
// jw/W lambda e^(u~/W)) re-evaluated at the perturbed u~' = u~ + delta w_k M_k.
// One CTA of 128 threads per element: unperturbed values per point, then chunks
// of FD_QC points: the perturbed (v' - v, s' - s) per (point, k) in shared
// memory, and each thread accumulates its (a, k) pairs over the points in order.
// ---------------------------------------------------------------------------
constexpr int FD_QC = 8;
template <int DIM, int P>
struct FdShape {
  static constexpr int NEN = ipow<DIM>(P + 1);
  static constexpr int THREADS = NEN >= 64 ? 256 : 128;  // (a, k) pairs per thread stay <= 16
};

template <int DIM, int P>
__global__ void __launch_bounds__(FdShape<DIM, P>::THREADS) k_elem_fd(DirArgs d0, DirArgs d1, DirArgs d2,
                                                                      const double *__restrict__ U, const double *__restrict__ wts,
                                                                      const double *__restrict__ geom, GeomLayout gl,
                                                                      double lambda, double *__restrict__ E, int64_t nelem) {
  constexpr int N1 = P + 1, Q = P + 1, NEN = ipow<DIM>(N1), NQ = ipow<DIM>(Q);
  constexpr int T = FdShape<DIM, P>::THREADS;
  constexpr int PAIRS = NEN * NEN, PPT = (PAIRS + T - 1) / T;
  __shared__ double tab[3][Q][N1][2];
  __shared__ double wa[NEN], ua[NEN];
  __shared__ double ut[NQ], gut[NQ][3], vq[NQ][3], sq[NQ];
  __shared__ double dv[FD_QC][NEN][3], ds[FD_QC][NEN];
  __shared__ double delta_s;
  const int64_t e = blockIdx.x;
  if (e >= nelem) return;
  const int tid = threadIdx.x;
  const int e0 = (int)(e % d0.nel), e1 = (int)((e / d0.nel) % d1.nel), e2 = DIM == 3 ? (int)(e / ((int64_t)d0.nel * d1.nel)) : 0;
  for (int k = tid; k < DIM * Q * N1 * 2; k += blockDim.x) {
    const int ax = k / (Q * N1 * 2), r = k % (Q * N1 * 2);
    const DirArgs &d = ax == 0 ? d0 : (ax == 1 ? d1 : d2);
    const int ee = ax == 0 ? e0 : (ax == 1 ? e1 : e2);
    (&tab[ax][0][0][0])[r] = d.tab[(size_t)ee * Q * N1 * 2 + r];
  }
  for (int a = tid; a < NEN; a += blockDim.x) {
    const int a0 = a % N1, a1 = (a / N1) % N1, a2 = DIM == 3 ? a / (N1 * N1) : 0;
    const int64_t G = (d0.first[e0] + a0) + (int64_t)d0.n * ((d1.first[e1] + a1) + (int64_t)d1.n * ((DIM == 3 ? d2.first[e2] : 0) + a2));
    ua[a] = U[G];
    wa[a] = wts ? wts[G] : 1.0;
  }
  __syncthreads();
  if (tid == 0) {
    double nrm = 0.0;
    for (int a = 0; a < NEN; a++) nrm += ua[a] * ua[a];
    delta_s = sqrt(DBL_EPSILON) * sqrt(1.0 + sqrt(nrm));
  }
  // M_a and grad M_a at point q from the tables
  auto basis = [&](int a, int q, double &m, double *dm) {
    const int a0 = a % N1, a1 = (a / N1) % N1, a2 = DIM == 3 ? a / (N1 * N1) : 0;
    const int g0 = q % Q, g1 = (q / Q) % Q, g2 = DIM == 3 ? q / (Q * Q) : 0;
    const double b0 = tab[0][g0][a0][0], db0 = tab[0][g0][a0][1], b1 = tab[1][g1][a1][0], db1 = tab[1][g1][a1][1];
    if (DIM == 3) {
      const double b2 = tab[2][g2][a2][0], db2 = tab[2][g2][a2][1];
      m = b0 * b1 * b2;
      dm[0] = db0 * b1 * b2;
      dm[1] = b0 * db1 * b2;
      dm[2] = b0 * b1 * db2;
    } else {
      m = b0 * b1;
      dm[0] = db0 * b1;
      dm[1] = b0 * db1;
    }
  };
  // v = S (grad u~ - u~ g), s = -g . v - jw/W lambda e^(u~ / W) at point q for given u~, grad u~
  auto integrand = [&](int q, double u, const double *gu, double *v, double &sv) {
    const double *rec = geom + (size_t)e * gl.nf * NQ + q;
    double r[3];
    for (int a = 0; a < DIM; a++) r[a] = gu[a] - u * rec[(gl.g + a) * NQ];
    if (DIM == 2) {
      const double s00 = rec[gl.S * NQ], s11 = rec[(gl.S + 1) * NQ], s01 = rec[(gl.S + 2) * NQ];
      v[0] = s00 * r[0] + s01 * r[1];
      v[1] = s01 * r[0] + s11 * r[1];
    } else {
      const double s00 = rec[gl.S * NQ], s11 = rec[(gl.S + 1) * NQ], s22 = rec[(gl.S + 2) * NQ];
      const double s01 = rec[(gl.S + 3) * NQ], s02 = rec[(gl.S + 4) * NQ], s12 = rec[(gl.S + 5) * NQ];
      v[0] = s00 * r[0] + s01 * r[1] + s02 * r[2];
      v[1] = s01 * r[0] + s11 * r[1] + s12 * r[2];
      v[2] = s02 * r[0] + s12 * r[1] + s22 * r[2];
    }
    sv = -rec[gl.jwW * NQ] * lambda * iga_exp(u * rec[gl.invW * NQ]);
    for (int a = 0; a < DIM; a++) sv -= rec[(gl.g + a) * NQ] * v[a];
  };
  for (int q = tid; q < NQ; q += blockDim.x) {
    double u = 0.0, gu[3] = {0.0, 0.0, 0.0};
    for (int a = 0; a < NEN; a++) {
      double m, dm[3];
      basis(a, q, m, dm);
      const double c = wa[a] * ua[a];
      u = fma(c, m, u);
      for (int i = 0; i < DIM; i++) gu[i] = fma(c, dm[i], gu[i]);
    }
    double v[3], sv;
    integrand(q, u, gu, v, sv);
    ut[q] = u;
    sq[q] = sv;
    for (int i = 0; i < DIM; i++) {
      gut[q][i] = gu[i];
      vq[q][i] = v[i];
    }
  }
  __syncthreads();
  const double delta = delta_s;
  double acc[PPT];
#pragma unroll
  for (int j = 0; j < PPT; j++) acc[j] = 0.0;
  for (int q0 = 0; q0 < NQ; q0 += FD_QC) {
    const int nq = min(FD_QC, NQ - q0);
    for (int idx = tid; idx < nq * NEN; idx += blockDim.x) {
      const int qq = idx / NEN, k = idx % NEN, q = q0 + qq;
      double m, dm[3];
      basis(k, q, m, dm);
      const double c = delta * wa[k];
      double gu[3], v[3], sv;
      for (int i = 0; i < DIM; i++) gu[i] = gut[q][i] + c * dm[i];
      integrand(q, ut[q] + c * m, gu, v, sv);
      for (int i = 0; i < DIM; i++) dv[qq][k][i] = v[i] - vq[q][i];
      ds[qq][k] = sv - sq[q];
    }
    __syncthreads();
#pragma unroll
    for (int j = 0; j < PPT; j++) {
      const int pr = tid + T * j;
      if (pr < PAIRS) {
        const int a = pr / NEN, k = pr % NEN;
        for (int qq = 0; qq < nq; qq++) {
          double m, dm[3];
          basis(a, q0 + qq, m, dm);
          double t = m * ds[qq][k];
          for (int i = 0; i < DIM; i++) t = fma(dm[i], dv[qq][k][i], t);
          acc[j] += t;
        }
      }
    }
    __syncthreads();
  }
#pragma unroll
  for (int j = 0; j < PPT; j++) {
    const int pr = tid + T * j;
    if (pr < PAIRS) {
      const int a = pr / NEN, k = pr % NEN;
      E[(size_t)e * PAIRS + (size_t)a * NEN + k] = wa[a] * acc[j] / delta;
    }
  }
}

#define DISPATCH_TC(DIM_, P_, CALL)                                      \
  do {                                                                   \
    if ((DIM_) == 2) {                                                   \
      switch (P_) {                                                      \
        case 1: { constexpr int D = 2, PP = 1; CALL; } break;            \
        case 2: { constexpr int D = 2, PP = 2; CALL; } break;            \
        case 3: { constexpr int D = 2, PP = 3; CALL; } break;            \
        case 4: { constexpr int D = 2, PP = 4; CALL; } break;            \
      }                                                                  \
    } else {                                                             \
      switch (P_) {                                                      \
        case 1: { constexpr int D = 3, PP = 1; CALL; } break;            \
        case 2: { constexpr int D = 3, PP = 2; CALL; } break;            \
        case 3: { constexpr int D = 3, PP = 3; CALL; } break;            \
      }                                                                  \
    }                                                                    \
  } while (0)

template <int DIM, int P, int OP>
cudaError_t run_tc(iga_s *h, const double *U, float cs, float cr) {
  using S = TcShape<DIM, P, OP>;
  constexpr int WPB = (S::PER * 2 <= 200 * 1024) ? ((S::PER * 4 <= 200 * 1024) ? 4 : 2) : 1;
  size_t sm = S::PER * WPB;
  auto kern = k_elem_tc<DIM, P, OP, WPB>;
  cudaError_t ce = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (ce) return ce;
  DirArgs a0 = dir_args(h->ddev[0]), a1 = dir_args(h->ddev[1]), a2 = dir_args(h->ddev[2]);
  unsigned grid = (unsigned)((h->nelem + WPB - 1) / WPB);
  IGA_LAUNCH(h, KC_ELEM_TC, (kern<<<grid, 32 * WPB, sm, h->stream>>>(a0, a1, a2, h->tab32[0], h->tab32[1], h->tab32[2], U,
                                                                       h->weights, h->geom32, (float)h->lambda, cs, cr,
                                                                       h->Ebuf, h->nelem)));
  return cudaGetLastError();
}

}  // namespace

bool mixed_supported(int dim, int p) { return dim == 2 ? (p >= 1 && p <= 4) : (p >= 1 && p <= 3); }

// Lazily build the FP32 tables and geometry slots and the element-matrix buffer.
static cudaError_t mixed_prepare(iga_s *h) {
  cudaError_t ce;
  if (!h->geom32) {
    int nq = (h->dim == 3) ? h->q * h->q * h->q : h->q * h->q;
    int nf = (h->dim == 3) ? G32<3>::NF : G32<2>::NF;
    ce = cudaMalloc((void **)&h->geom32, (size_t)h->nelem * nf * nq * sizeof(float));
    if (ce) return ce;
    int64_t tot = h->nelem * nq;
    unsigned grid = (unsigned)((tot + 255) / 256);
    // every degree (the element GEMM takes 3D p = 4, which the per-element kernels do not)
    if (h->dim == 3 && h->p == 4)
      IGA_LAUNCH(h, KC_GEOM, (k_geom32<3, 4><<<grid, 256, 0, h->stream>>>(h->geom, h->gl, h->geom32, h->nelem)));
    else
      IGA_LAUNCH(h, KC_GEOM, DISPATCH_TC(h->dim, h->p, (k_geom32<D, PP><<<grid, 256, 0, h->stream>>>(h->geom, h->gl, h->geom32, h->nelem))));
    for (int ax = 0; ax < h->dim; ax++) {
      size_t n = h->dir[ax].tab.size();
      ce = cudaMalloc((void **)&h->tab32[ax], n * sizeof(float));
      if (ce) return ce;
      IGA_LAUNCH(h, KC_VEC, (k_to_f32<<<(unsigned)((n + 255) / 256), 256, 0, h->stream>>>(h->ddev[ax].tab, h->tab32[ax], (int64_t)n)));
    }
  }
  return cudaGetLastError();
}

static cudaError_t ebuf_prepare(iga_s *h) {
  if (!h->Ebuf) {
    int nen = (h->dim == 3) ? (h->p + 1) * (h->p + 1) * (h->p + 1) : (h->p + 1) * (h->p + 1);
    cudaError_t ce = cudaMalloc((void **)&h->Ebuf, (size_t)h->nelem * nen * nen * sizeof(float));
    if (ce) return ce;
  }
  return cudaSuccess;
}

bool tc_jacobian_supported(iga_s *h, int prec) {
  if (h->inner) return false;
  return elem_gemm_supported(h, prec) || mixed_supported(h->dim, h->p);
}

// Jacobian by local numerical differentiation (FP64 values), same degrees as the
// tensor-core path; the element matrices go to a library-owned FP64 buffer.
cudaError_t launch_jacobian_fd(iga_s *h, const double *U, double *vals) {
  if (!mixed_supported(h->dim, h->p)) return cudaErrorNotSupported;
  const int nen = (h->dim == 3) ? (h->p + 1) * (h->p + 1) * (h->p + 1) : (h->p + 1) * (h->p + 1);
  if (!h->Ebuf64) {
    cudaError_t ce = cudaMalloc((void **)&h->Ebuf64, (size_t)h->nelem * nen * nen * sizeof(double));
    if (ce) return ce;
  }
  DirArgs a0 = dir_args(h->ddev[0]), a1 = dir_args(h->ddev[1]), a2 = dir_args(h->ddev[2]);
  IGA_LAUNCH(h, KC_ELEM_TC, DISPATCH_TC(h->dim, h->p, (k_elem_fd<D, PP><<<(unsigned)h->nelem, FdShape<D, PP>::THREADS, 0, h->stream>>>(
                                                          a0, a1, a2, U, h->weights, h->geom, h->gl, h->lambda, h->Ebuf64, h->nelem))));
  unsigned grid = (unsigned)((h->N * 32 + 255) / 256);
  IGA_LAUNCH(h, KC_ELEM_GATHER, DISPATCH_TC(h->dim, h->p, (k_gather_elem<D, PP, double><<<grid, 256, 0, h->stream>>>(
                                                              a0, a1, a2, h->Ebuf64, h->rowptr, nullptr, h->bnd, vals, h->N))));
  return cudaGetLastError();
}

// Full mixed-precision Jacobian into FP32 CSR values (prec: IGA_JAC_TF32 / IGA_JAC_BF16).
cudaError_t launch_jacobian_mixed(iga_s *h, const double *U, float *vals, int prec) {
  cudaError_t ce = mixed_prepare(h);
  if (ce) return ce;
  // repeated 1D tables: the element matrices as one tensor-core GEMM across elements
  if (elem_gemm_supported(h, prec)) return launch_jacobian_elem_gemm(h, U, vals, prec);
  if (!mixed_supported(h->dim, h->p)) return cudaErrorNotSupported;
  if ((ce = ebuf_prepare(h))) return ce;
  if (prec == IGA_JAC_BF16) {
    DISPATCH_TC(h->dim, h->p, ce = (run_tc<D, PP, OP_BF16>(h, U, 1.f, 1.f)));
  } else {
    DISPATCH_TC(h->dim, h->p, ce = (run_tc<D, PP, OP_TF32>(h, U, 1.f, 1.f)));
  }
  if (ce) return ce;
  DirArgs a0 = dir_args(h->ddev[0]), a1 = dir_args(h->ddev[1]), a2 = dir_args(h->ddev[2]);
  unsigned grid = (unsigned)((h->N * 32 + 255) / 256);
  IGA_LAUNCH(h, KC_ELEM_GATHER, DISPATCH_TC(h->dim, h->p, (k_gather_elem<D, PP><<<grid, 256, 0, h->stream>>>(a0, a1, a2, h->Ebuf, h->rowptr, h->weights, h->bnd, vals, h->N))));
  return cudaGetLastError();
}
