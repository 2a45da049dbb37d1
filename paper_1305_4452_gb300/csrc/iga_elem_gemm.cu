// Element matrices of the reduced-precision Jacobian as one GEMM across elements
// on the 5th-generation tensor cores (tcgen05.mma, BF16 or TF32 operands, FP32
// accumulator in tensor memory).
//
// With Q_{mu nu}(e, q) the per-Gauss-point coefficients (geometry, kappa and the
// reaction term at U, mu, nu = 0 for values and 1..DIM for derivatives) and
// D_mu M_a(q) the tensor-product B-spline values and first derivatives,
//     E_ab(e) = sum_q sum_{mu,nu} Q_{mu nu}(e, q) D_mu M_a(q) D_nu M_b(q)
// (the element matrix of Eq. (jacobian), Sec. 2.7, before the weights w_a w_b).
// D_mu M_a(q) depends on the element only through its three 1D tables, and the
// elements of a uniform knot vector share them except for p elements at each end
// per direction.  For elements of one such type, with k = (slot s = (mu <= nu), q)
// and the pairs (a, b),
//     E(e, ab) = sum_k Qv(e, k) T(k, ab),       Qv(e, (s, q)) = Q_{mu nu}(e, q),
//     T((s, q), ab) = D_mu M_a D_nu M_b + [mu != nu] D_nu M_a D_mu M_b,
// a dense (elements x K) x (K x pairs) product: M = 128 elements of one type per
// tile, N = 128 pairs, K = slots x NQ (padded to 64).  E is symmetric (Q is), so only
// the pairs a <= b are formed, packed row by row.  Identity maps with unit
// weights have g = 0 and a diagonal S, so only the DIM+1 slots mu = nu are nonzero.
//
// k_elem_gemm, one CTA per (128 elements, 128 pairs) tile and group of element tiles,
// 256 threads:
//   - the T tile of the CTA's pair range comes from a per-mesh cache built once by the
//     same kernel in build mode (when the cache takes at most 1 GB), else two threads per
//     pair row compute it from the type's 1D tables; it stays in shared memory for the
//     CTA's group of element tiles.  When the T tile of the whole K does not fit (TF32 at
//     p = 4, general maps at p = 4), K runs in passes of at most EG_PASS_CHUNKS chunks:
//     the group (at most EG_PASS_GROUP element tiles) keeps one accumulator per tile in
//     tensor memory, each pass loads its part of T and adds its chunks' MMAs to every
//     tile's accumulator, and the epilogues follow the last pass;
//   - two threads per row copy an element row of each Qv chunk (cp.async, 16 B) into the
//     canonical K-major layout without swizzling (8-row x 16-byte core matrices, 128 B
//     apart along M/N, 2 KB apart along K), two stages, the next chunk's copy issued
//     before the wait for the current one;
//   - thread 0 issues the chunk's four tcgen05.mma (32 bytes of K each) and commits
//     them to the stage's barrier, which frees the stage two chunks later;
//   - after the last chunk warp w reads accumulator rows 32 (w % 4) .. + 31 (half the
//     columns each) with
//     tcgen05.ld and writes them to the element-matrix buffer E[slot][packed (a, b)].
// T is the same for every element of a type, so its rounding error would perturb the
// assembled matrix systematically (row sums of the stiffness part no longer vanish,
// which slows Newton on fine meshes); where shared memory allows, T is kept as a
// rounded part plus its rounded remainder and each chunk runs the MMAs on both with
// the same Qv operand (about 16 significant bits for BF16, 21 for TF32).
// Every barrier wait is bounded in time; the decision to stop is taken by thread 0
// and shared through shared memory, so all threads leave the loop together.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "iga_internal.h"
#include "iga_tc.h"
#include "iga_interp.h"

namespace {

constexpr int GT = 128;          // elements (M) and pairs (N) per tile
constexpr int KB = 128;          // bytes of K per chunk and row
constexpr int STAGE = GT * KB;   // bytes of one operand chunk
constexpr uint32_t LBO = 16 * 128;  // next 16 bytes of K: 16 row groups of 128 B
constexpr int EG_GROUP_MAX = 32;    // m-tiles per CTA at most (one T tile computed per CTA)
constexpr int EG_PASS_CHUNKS = 10;  // T chunks resident per K pass when the whole K does not fit
constexpr int EG_PASS_GROUP = 4;    // m-tiles per CTA with K passes: 4 accumulators of 128 columns

enum { EG_BF16 = 0, EG_TF32 = 1 };

// (mu, nu) of each slot: the DIM+1 diagonal slots first, then mu < nu
struct Slots {
  int n;
  int mu[10], nu[10];
};
__host__ __device__ inline Slots make_slots(int dim, bool general) {
  Slots s;
  s.n = 0;
  for (int m = 0; m <= dim; m++) { s.mu[s.n] = m; s.nu[s.n] = m; s.n++; }
  if (general)
    for (int m = 0; m <= dim; m++)
      for (int v = m + 1; v <= dim; v++) { s.mu[s.n] = m; s.nu[s.n] = v; s.n++; }
  return s;
}

struct GemmArgs {
  const void *Qv;          // [slots_total][Kp] operand values (BF16, or TF32 in FP32 containers)
  float *E;                // [nsym][N]: E_ab(e), a <= b, in slab pk(a, b) at column A(e, a)
  const int *elem_of_slot; // [slots_total] element of each slot, -1 for padding
  const int *first[3];     // first function of each element per direction
  const int *pair_off;     // [nsym][2]: offsets of a and of b from the element's first function, natural order
  int nel0, nel1;
  int64_t N, N0, N1;        // functions in all, along x, along y
  const float *tab[3];     // FP32 1D tables [nel][q][p+1][2]
  const int *group;        // [ngroups][6]: first m-tile, m-tiles, element of the type per direction, type
  const uint8_t *Tc;       // T tiles built once per mesh ([type][n_tile][tile_bytes]), or null
  uint8_t *Tout;           // build mode: write the T tiles here and stop
  int64_t tile_bytes;
  const int *pair_ab;      // [nsym]: a | b << 16, a <= b, row by row
  int dim, p, nq, nsym, nen, Kp, n_tiles, m_tiles, general;
  int split;  // 1: T = T_hi + T_lo, both in the operand type (two MMAs per chunk on the same Qv)
  int npass;  // K passes (1: the T tile of the whole K is resident)
  int *err;
  uint64_t limit_ns;  // bound of each pipeline wait (the drain after a stop keeps MBAR_LIMIT_NS)
  int stall;          // failure-detection test: wait once on a barrier phase that nothing completes
};

__device__ __forceinline__ uint32_t op_bits(float x, int op) {
  if (op == EG_BF16) {
    __nv_bfloat16 h = __float2bfloat16_rn(x);
    return (uint32_t)*reinterpret_cast<uint16_t *>(&h);
  }
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return r;
}

// Shared memory of k_elem_gemm: the T tile for the whole K (one STAGE per chunk; twice
// with the split into a rounded part and its rounded remainder), two A stages, the 1D
// tables, the slot table, barriers and flags.
__host__ __device__ constexpr size_t eg_smem(int nchunks, int split) {
  return (size_t)(nchunks * (1 + split) + 2) * STAGE + 3 * 5 * 5 * 2 * sizeof(float) + (32 + 3 * GT) * sizeof(int) +
         2 * sizeof(uint64_t) + 16;
}

template <int OP>
__global__ void __launch_bounds__(256) k_elem_gemm(GemmArgs g) {
  constexpr int ES = OP == EG_BF16 ? 2 : 4;  // operand bytes
  constexpr int KC = KB / ES;                // K values per chunk
  constexpr int PER = 16 / ES;               // values per 16 bytes
  const int nchunks = g.Kp / KC;
  const int npass = g.npass, pcs = (nchunks + npass - 1) / npass;  // K passes, chunks per pass
  extern __shared__ __align__(128) uint8_t sm[];
  uint8_t *Ts = sm;                                    // [pcs][STAGE]  T rounded (this pass's chunks)
  uint8_t *Tl = sm + (size_t)pcs * STAGE;              // [pcs][STAGE]  remainder (split, one pass only)
  uint8_t *As = sm + (size_t)pcs * (1 + g.split) * STAGE;  // [2][STAGE]
  float *tab = reinterpret_cast<float *>(As + 2 * STAGE);  // [3][q][p+1][2]
  int *smu = reinterpret_cast<int *>(tab + 3 * 5 * 5 * 2), *snu = smu + 16;
  int *spair = smu + 32;  // [GT][3]: this pair tile's (a | b << 16, offset of a, offset of b)
  uint64_t *done = reinterpret_cast<uint64_t *>(spair + 3 * GT);
  uint32_t *slot = reinterpret_cast<uint32_t *>(done + 2);
  volatile int *abort_s = reinterpret_cast<volatile int *>(slot + 1);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int r128 = tid & 127, half = tid >> 7;  // operand row of this thread, and which half of its 8 16-byte chunks
  const int grp = blockIdx.x / g.n_tiles, n_tile = blockIdx.x % g.n_tiles;
  const int m_first = g.group[grp * 6 + 0], m_count = g.group[grp * 6 + 1];
  const int q = g.p + 1, n1 = g.p + 1;
  const int tsz = q * n1 * 2;

  // tensor memory: one 128-column accumulator, or one per m-tile of the group with K passes
  const uint32_t tcols = npass > 1 ? (uint32_t)(EG_PASS_GROUP * GT) : (uint32_t)GT;
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(slot)), "r"(tcols) : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(su32(done)) : "memory");
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(su32(done + 1)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    *abort_s = 0;
    const Slots S = make_slots(g.dim, g.general != 0);
    for (int k = 0; k < 16; k++) {
      smu[k] = k < S.n ? S.mu[k] : 0;
      snu[k] = k < S.n ? S.nu[k] : 0;
    }
    smu[15] = S.n;
  }
  for (int k = tid; k < 3 * tsz; k += blockDim.x) {
    const int ax = k / tsz, r = k - ax * tsz;
    tab[k] = ax < g.dim ? g.tab[ax][(size_t)g.group[grp * 6 + 2 + ax] * tsz + r] : (r % 2 == 0 ? 1.f : 0.f);
  }
  for (int c = tid; c < GT; c += blockDim.x) {
    const int n = n_tile * GT + c;
    spair[3 * c] = n < g.nsym ? g.pair_ab[n] : -1;
    spair[3 * c + 1] = n < g.nsym ? g.pair_off[2 * n] : 0;
    spair[3 * c + 2] = n < g.nsym ? g.pair_off[2 * n + 1] : 0;
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *slot;
  const int nslot = smu[15];
  const int KV = nslot * g.nq;

  // ---- T tile of this pair range for chunks [c_lo, c_hi) of K (all of K in one pass):
  // copied from the per-mesh cache, or built here (once per group and pass) from the
  // type's 1D tables ----
  const int64_t tile_off = ((int64_t)g.group[grp * 6 + 5] * g.n_tiles + n_tile) * g.tile_bytes;
  auto load_T = [&](int c_lo, int c_hi) {
  if (g.Tc) {
    // one pass: the whole cached tile (with the remainder part when split); passes: this
    // pass's chunks of the rounded part
    const int64_t x0 = (int64_t)c_lo * STAGE, x1 = npass > 1 ? (int64_t)c_hi * STAGE : g.tile_bytes;
    for (int64_t x = x0 + (int64_t)tid * 16; x < x1; x += 16 * (int64_t)blockDim.x)
      cp16(su32(Ts) + (uint32_t)(x - x0), g.Tc + tile_off + x, true);
    cp_commit();
    cp_wait<0>();
  } else {
    const int npair = n_tile * GT + r128;
    int a0 = 0, a1 = 0, a2 = 0, b0 = 0, b1 = 0, b2 = 0;
    const bool pvalid = npair < g.nsym;
    if (pvalid) {
      const int ab = g.pair_ab[npair];
      const int ia = ab & 0xFFFF, ib = ab >> 16;
      a0 = ia % n1;
      a1 = (ia / n1) % n1;
      a2 = g.dim == 3 ? ia / (n1 * n1) : 0;
      b0 = ib % n1;
      b1 = (ib / n1) % n1;
      b2 = g.dim == 3 ? ib / (n1 * n1) : 0;
    }
#define TB(ax, gq, aa, s) tab[(((ax) * q + (gq)) * n1 + (aa)) * 2 + (s)]
    const uint32_t rowoff = (uint32_t)((r128 >> 3) * 128 + (r128 & 7) * 16);
    for (int c = c_lo; c < c_hi; c++) {
      const uint32_t bdst = su32(Ts + (size_t)(c - c_lo) * STAGE) + rowoff, ldst = su32(Tl + (size_t)(c - c_lo) * STAGE) + rowoff;
      for (int kc = half * 4; kc < half * 4 + 4; kc++) {
        int k = c * KC + kc * PER, sl = k / g.nq, qp = k - sl * g.nq;  // K index, its slot and Gauss point
        uint32_t w[4] = {0u, 0u, 0u, 0u}, wl[4] = {0u, 0u, 0u, 0u};
#pragma unroll
        for (int j = 0; j < PER; j++, k++) {
          float v = 0.f;
          if (pvalid && k < KV) {
            const int mu = smu[sl], nu = snu[sl];
            const int g0 = qp % q, g1 = (qp / q) % q, g2 = g.dim == 3 ? qp / (q * q) : 0;
            const float Dam = TB(0, g0, a0, mu == 1) * TB(1, g1, a1, mu == 2) * TB(2, g2, a2, mu == 3);
            const float Dbn = TB(0, g0, b0, nu == 1) * TB(1, g1, b1, nu == 2) * TB(2, g2, b2, nu == 3);
            v = Dam * Dbn;
            if (mu != nu) {
              const float Dan = TB(0, g0, a0, nu == 1) * TB(1, g1, a1, nu == 2) * TB(2, g2, a2, nu == 3);
              const float Dbm = TB(0, g0, b0, mu == 1) * TB(1, g1, b1, mu == 2) * TB(2, g2, b2, mu == 3);
              v += Dan * Dbm;
            }
          }
          if (++qp == g.nq) {
            qp = 0;
            sl++;
          }
          const uint32_t bits = op_bits(v, OP);
          // the rounding error of T is the same in every element of the type: without the
          // split it is a systematic perturbation of the assembled matrix
          const float hv = ES == 2 ? __uint_as_float(bits << 16) : __uint_as_float(bits);
          const uint32_t lbits = g.split ? op_bits(v - hv, OP) : 0u;
          if (ES == 2) {
            w[j >> 1] |= bits << (16 * (j & 1));
            wl[j >> 1] |= lbits << (16 * (j & 1));
          } else {
            w[j] = bits;
            wl[j] = lbits;
          }
        }
        asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(bdst + kc * LBO), "r"(w[0]), "r"(w[1]), "r"(w[2]),
                     "r"(w[3])
                     : "memory");
        if (g.split)
          asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(ldst + kc * LBO), "r"(wl[0]), "r"(wl[1]), "r"(wl[2]),
                       "r"(wl[3])
                       : "memory");
      }
    }
#undef TB
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  __syncthreads();
  if (g.Tout) {  // build mode: the tile (this pass's part of it) goes to the per-mesh cache
    const int64_t x0 = (int64_t)c_lo * STAGE, x1 = npass > 1 ? (int64_t)c_hi * STAGE : g.tile_bytes;
    for (int64_t x = x0 + (int64_t)tid * 16; x < x1; x += 16 * (int64_t)blockDim.x)
      *reinterpret_cast<uint4 *>(g.Tout + tile_off + x) = *reinterpret_cast<const uint4 *>(Ts + (x - x0));
    __syncthreads();  // the next pass rebuilds Ts
  }
  };

  const uint32_t idesc = (1u << 4) | ((OP == EG_BF16 ? 1u : 2u) << 7) | ((OP == EG_BF16 ? 1u : 2u) << 10) |
                         ((uint32_t)(GT >> 3) << 17) | ((uint32_t)(GT >> 4) << 24);
  const uint32_t rowoff = (uint32_t)((r128 >> 3) * 128 + (r128 & 7) * 16);
  int it = 0;     // chunk counter over all m-tiles (stage it & 1)
  int last = -1;  // thread 0: the last chunk whose MMAs were committed
  // copy chunk c of m-tile mt_ of the Qv operand into stage st_ (this thread's 64 bytes of
  // its row), as one cp.async group
  auto issue = [&](int mt_, int c_, int st_) {
    const uint8_t *qr = reinterpret_cast<const uint8_t *>(g.Qv) + ((size_t)mt_ * GT + r128) * g.Kp * ES + (size_t)c_ * KB;
    const uint32_t adst = su32(As + st_ * STAGE) + rowoff;
#pragma unroll
    for (int kc = half * 4; kc < half * 4 + 4; kc++) cp16(adst + kc * LBO, qr + kc * 16, true);
    cp_commit();
  };
  // failure-detection test: barrier 1's first phase completes only at the first commit to
  // stage 1, which never comes before this wait, so the wait gives up after limit_ns and the
  // kernel stops before it has issued any copy or MMA
  if (g.stall) {
    if (tid == 0 && !mbar_wait(su32(done + 1), 0, abort_s, 0, g.limit_ns)) *abort_s = 1;
    __syncthreads();
  }
  // E_ab (a <= b) goes to slab pk(a, b) at column A(e, a): for consecutive elements
  // along x the lanes write consecutive floats; warp w reads tensor-memory lanes
  // 32 (w % 4) .. + 31, columns 64 (w / 4) .. + 63 of the m-tile's accumulator
  auto epilogue = [&](int mt, uint32_t acc_tm) {
    tc_fence_after();
    const int quarter = warp & 3, ch = warp >> 2;
    const int row = quarter * 32 + lane;
    const int e = g.elem_of_slot[(size_t)mt * GT + row];
    int64_t abase = 0;
    if (e >= 0) {
      const int e0 = e % g.nel0, e1 = (e / g.nel0) % g.nel1, e2 = g.dim == 3 ? e / (g.nel0 * g.nel1) : 0;
      abase = g.first[0][e0] + g.N0 * ((int64_t)g.first[1][e1] + (int64_t)g.N1 * (g.dim == 3 ? g.first[2][e2] : 0));
    }
    for (int c0 = ch * (GT / 2); c0 < (ch + 1) * (GT / 2); c0 += 16) {
      float v[16];
      tmem_ld16(acc_tm + ((uint32_t)(quarter * 32) << 16) + (uint32_t)c0, v);
      if (e < 0) continue;
#pragma unroll
      for (int u = 0; u < 16; u++) {
        if (spair[3 * (c0 + u)] < 0) break;
        g.E[(size_t)(n_tile * GT + c0 + u) * g.N + abase + spair[3 * (c0 + u) + 1]] = v[u];
      }
    }
    tc_fence_before();
    __syncthreads();  // the accumulator is read before later MMAs overwrite it
  };
  // K in npass passes; within a pass two stages in flight: the copy of the next chunk (the
  // next m-tile's first chunk of the pass after a tile's last) is issued before the wait for
  // the current one, and runs during the MMAs and the epilogue
  for (int h = 0; h < npass && !*abort_s; h++) {
    const int c_lo = h * pcs, c_hi = min(nchunks, c_lo + pcs);
    if (h > 0) {
      // the previous pass's MMAs read Ts: its last commit precedes the rebuild
      if (tid == 0 && last >= 0 && !mbar_wait(su32(done + (last & 1)), (last >> 1) & 1, abort_s, 0, g.limit_ns)) *abort_s = 1;
      __syncthreads();
      if (*abort_s) break;
    }
    load_T(c_lo, c_hi);
    if (m_count > 0 && !*abort_s) issue(m_first, c_lo, it & 1);
    for (int mi = 0; mi < m_count && !*abort_s; mi++) {
      const int mt = m_first + mi;
      const uint32_t acc_tm = tmem + (npass > 1 ? (uint32_t)(mi * GT) : 0u);
      for (int c = c_lo; c < c_hi; c++, it++) {
        const int st = it & 1;
        if ((c + 1 < c_hi) || (mi + 1 < m_count)) {
          // the other stage is free once the MMAs of chunk it - 1, which read it, are complete
          if (it >= 1) {
            if (tid == 0 && !mbar_wait(su32(done + (st ^ 1)), ((it - 1) >> 1) & 1, abort_s, 0, g.limit_ns)) *abort_s = 1;
            __syncthreads();
            if (*abort_s) break;
          }
          if (c + 1 < c_hi) issue(mt, c + 1, st ^ 1);
          else issue(mt + 1, c_lo, st ^ 1);
          cp_wait<1>();  // this chunk's copies have landed; the next chunk's may be in flight
        } else {
          cp_wait<0>();
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        if (tid == 0) {
          tc_fence_after();
          const uint64_t ad = sdesc(su32(As + st * STAGE), LBO, 128);
          for (int part = 0; part <= g.split; part++) {
            const uint64_t bd = sdesc(su32((part ? Tl : Ts) + (size_t)(c - c_lo) * STAGE), LBO, 128);
#pragma unroll
            for (int kk = 0; kk < 4; kk++) {
              const uint32_t acc = (c > 0 || kk > 0 || part > 0) ? 1u : 0u;
              const uint64_t a_k = ad + (uint64_t)((kk * 2 * LBO) >> 4), b_k = bd + (uint64_t)((kk * 2 * LBO) >> 4);
              if constexpr (OP == EG_BF16)
                asm volatile(
                    "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(acc_tm),
                    "l"(a_k), "l"(b_k), "r"(idesc), "r"(acc)
                    : "memory");
              else
                asm volatile(
                    "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(acc_tm),
                    "l"(a_k), "l"(b_k), "r"(idesc), "r"(acc)
                    : "memory");
            }
          }
          asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(su32(done + st))
                       : "memory");
          last = it;
        }
      }
      if (*abort_s) break;
      if (npass == 1) {
        // this m-tile's accumulator is complete once its last commit has arrived
        if (tid == 0 && !mbar_wait(su32(done + ((it - 1) & 1)), ((it - 1) >> 1) & 1, abort_s, 0, g.limit_ns)) *abort_s = 1;
        __syncthreads();
        if (*abort_s) break;
        epilogue(mt, acc_tm);
      }
    }
  }
  if (npass > 1 && m_count > 0 && !*abort_s) {
    // every accumulator of the group is complete once the last pass's last commit has arrived
    if (tid == 0 && !mbar_wait(su32(done + ((it - 1) & 1)), ((it - 1) >> 1) & 1, abort_s, 0, g.limit_ns)) *abort_s = 1;
    __syncthreads();
    for (int mi = 0; mi < m_count && !*abort_s; mi++) epilogue(m_first + mi, tmem + (uint32_t)(mi * GT));
  }
  cp_wait<0>();  // after a stop a prefetched chunk may still be in flight
  // after a stop, wait (bounded) for the last committed MMAs before freeing the tensor memory
  if (tid == 0 && *abort_s) {
    if (last >= 0) (void)mbar_wait(su32(done + (last & 1)), (last >> 1) & 1, nullptr);
    atomicExch(g.err, 1);
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(tcols) : "memory");
}

// Qv[slot(e)][(s, q)] = Q_{mu nu}(e, q) in the operand type from the FP32 geometry
// factors (geom32) and U: Q_00 = gSg - jw/W^2 lambda e^u (u~ interpolated and the exponential taken in
// FP32), Q_0a = nSg_a, Q_ab = S_ab.  One thread per Gauss point, EB elements per block.
template <int DIM, int P, int OP>
__global__ void __launch_bounds__(128) k_qv(DirArgs d0, DirArgs d1, DirArgs d2, const double *__restrict__ U,
                                            const double *__restrict__ wts, const float *__restrict__ g32,
                                            float lambda, const int *__restrict__ slot_of_elem, void *__restrict__ Qv, int Kp,
                                            int general, int64_t nelem) {
  using IS = InterpF32<DIM, P>;
  constexpr int nq = IS::NQ;
  __shared__ float ue[IS::EB * IS::NEN], tb[IS::EB * DIM * IS::Q * IS::N1];
  const int64_t e_first = (int64_t)blockIdx.x * IS::EB;
  const float ut = interp_u_block<DIM, P>(d0, d1, d2, U, wts, e_first, nelem, ue, tb);
  const int le = threadIdx.x / nq, qp = threadIdx.x - le * nq;
  const int64_t e = e_first + le;
  if (le >= IS::EB || e >= nelem) return;
  using GL = G32<DIM>;
  const float *rec = g32 + (size_t)e * GL::NF * nq + qp;
  const float q00 = rec[GL::GSG * nq] - rec[GL::JWW2 * nq] * lambda * __expf(ut * rec[GL::INVW * nq]);
  const Slots S = make_slots(DIM, general != 0);
  const size_t row = (size_t)slot_of_elem[e] * Kp;
#pragma unroll
  for (int s = 0; s < (DIM == 3 ? 10 : 6); s++) {
    if (s >= S.n) break;
    const int mu = S.mu[s], nu = S.nu[s];
    float v;
    if (mu == 0 && nu == 0) v = q00;
    else if (mu == 0) v = rec[(GL::NSG + nu - 1) * nq];
    else {
      // S slots: 2D 00, 11, 01; 3D 00, 11, 22, 01, 02, 12
      const int i = mu - 1, j = nu - 1;
      const int si = (i == j) ? i : (DIM == 2 ? 2 : (i == 0 ? (j == 1 ? 3 : 4) : 5));
      v = rec[(GL::S + si) * nq];
    }
    const uint32_t bits = op_bits(v, OP);
    if (OP == EG_BF16) reinterpret_cast<uint16_t *>(Qv)[row + (size_t)s * nq + qp] = (uint16_t)bits;
    else reinterpret_cast<uint32_t *>(Qv)[row + (size_t)s * nq + qp] = bits;
  }
}

// The same Qv for elements of at most 27 Gauss points (2D, or 3D with p <= 2), in two
// phases per block of 128 elements: one thread per element forms u~ at its points
// (interp_u_elem, the same operations per point as interp_u_block) into shared memory,
// then one thread per (element, point) of the block's contiguous range reads the FP32
// geometry factors (coalesced) and writes the element's Qv row entries.
template <int DIM, int P, int OP>
__global__ void __launch_bounds__(128) k_qv_e(DirArgs d0, DirArgs d1, DirArgs d2, const double *__restrict__ U,
                                              const double *__restrict__ wts, const float *__restrict__ g32,
                                              float lambda, const int *__restrict__ slot_of_elem, void *__restrict__ Qv, int Kp,
                                              int general, int64_t nelem) {
  constexpr int Q = P + 1, EB = 128, nq = DIM == 3 ? Q * Q * Q : Q * Q;
  __shared__ float ut_s[EB * nq];
  const int64_t e_first = (int64_t)blockIdx.x * EB, e = e_first + threadIdx.x;
  if (e < nelem) interp_u_elem<DIM, P>(d0, d1, d2, U, wts, e, ut_s + threadIdx.x * nq);
  __syncthreads();
  using GL = G32<DIM>;
  const Slots S = make_slots(DIM, general != 0);
  const int nb = (int)min((int64_t)EB, nelem - e_first);
  for (int k = threadIdx.x; k < nb * nq; k += EB) {
    const int le = k / nq, qp = k - le * nq;
    const int64_t ee = e_first + le;
    const float *rec = g32 + (size_t)ee * GL::NF * nq + qp;
    const float q00 = rec[GL::GSG * nq] - rec[GL::JWW2 * nq] * lambda * __expf(ut_s[k] * rec[GL::INVW * nq]);
    const size_t row = (size_t)slot_of_elem[ee] * Kp;
#pragma unroll
    for (int s = 0; s < (DIM == 3 ? 10 : 6); s++) {
      if (s >= S.n) break;
      const int mu = S.mu[s], nu = S.nu[s];
      float v;
      if (mu == 0 && nu == 0) v = q00;
      else if (mu == 0) v = rec[(GL::NSG + nu - 1) * nq];
      else {
        // S slots: 2D 00, 11, 01; 3D 00, 11, 22, 01, 02, 12
        const int i = mu - 1, j = nu - 1;
        const int si = (i == j) ? i : (DIM == 2 ? 2 : (i == 0 ? (j == 1 ? 3 : 4) : 5));
        v = rec[(GL::S + si) * nq];
      }
      const uint32_t bits = op_bits(v, OP);
      if (OP == EG_BF16) reinterpret_cast<uint16_t *>(Qv)[row + (size_t)s * nq + qp] = (uint16_t)bits;
      else reinterpret_cast<uint32_t *>(Qv)[row + (size_t)s * nq + qp] = bits;
    }
  }
}

template <int DIM> __host__ __device__ constexpr int ipow3(int b) { return DIM == 2 ? b * b : b * b * b; }

// One thread per CSR row A (consecutive rows across a warp) and, in 3D, per axis-2
// column offset s2 = blockIdx.y of the row (the row's columns J2 = l(I2) + s2): the
// thread owns the w0 w1 columns of that slice, not the row's w0 w1 w2.  For every element
// e containing A (e2, e1, e0 ascending) whose axis-2 functions include J2, with a the
// local index of A in e, it reads E_ab for the b of e in the slice -- slab pk(a, b) at
// column A for b >= a, slab pk(b, a) at column A(e, b) = A + off(b) - off(a) for b < a;
// both coalesced across the warp's rows -- and adds it at the column of e's function b,
// in a per-thread accumulator in shared memory (each column's terms in element order);
// then w_A w_B and the Dirichlet rows and columns.
template <int DIM, int P, int TPB>
__global__ void __launch_bounds__(TPB) k_gather_rows(DirArgs d0, DirArgs d1, DirArgs d2, const float *__restrict__ E,
                                                     const int2 *__restrict__ gtab_g, const int64_t *__restrict__ rowptr,
                                                     const double *__restrict__ wts, BndArgs bnd, float *__restrict__ vals,
                                                     int64_t N, int slice_major) {
  constexpr int N1 = P + 1, NEN = ipow3<DIM>(N1), RMAX = (2 * P + 1) * (2 * P + 1);
  constexpr int NB = N1 * N1;  // functions of an element in one axis-2 slice (2D: all)
  constexpr int LD = TPB + 1;  // accumulator stride: conflict-free by thread and by column
  constexpr int TABOFF = (RMAX * LD + 1) / 2 * 2;  // the int2 table starts on an 8-byte boundary
  constexpr bool TAB_SMEM = NEN * NEN * 8 <= 8 * 1024;  // p = 2: small enough not to cost occupancy
  extern __shared__ float acc_all[];  // [RMAX][TPB + 1] (+ pad to 8 bytes), then the (pk, column shift) table
  __shared__ int64_t r0_s[TPB];       // each row slice's first CSR position (-1: nothing to store)
  __shared__ int len_s[TPB];
  const int t = threadIdx.x;
  const int2 *gtab = gtab_g;
  if (TAB_SMEM) {
    int2 *st = reinterpret_cast<int2 *>(acc_all + TABOFF);
    for (int k = t; k < NEN * NEN; k += TPB) st[k] = gtab_g[k];
    __syncthreads();
    gtab = st;
  }
  // slice_major: blockIdx.x is the axis-2 slice and blockIdx.y the row chunk, so that the
  // slices of a row chunk run together and the mirrored reads of the element matrices
  // (rows a few axis-2 layers apart) find them in L2
  const int64_t A = (int64_t)(slice_major ? blockIdx.y : blockIdx.x) * TPB + t;
  float *acc = acc_all + t;
  const int64_t Ac = A < N ? A : N - 1;
  const int I0 = (int)(Ac % d0.n), I1 = (int)((Ac / d0.n) % d1.n), I2 = (DIM == 3) ? (int)(Ac / ((int64_t)d0.n * d1.n)) : 0;
  const int l0 = d0.l[I0], l1 = d1.l[I1], l2 = DIM == 3 ? d2.l[I2] : 0;
  const int w0 = d0.r[I0] - l0 + 1, w1 = d1.r[I1] - l1 + 1, w2 = DIM == 3 ? d2.r[I2] - l2 + 1 : 1;
  const int s2 = DIM == 3 ? (int)(slice_major ? blockIdx.x : blockIdx.y) : 0;
  const bool active = A < N && s2 < w2;  // no early return: the block stores together at the end
  const int J2 = l2 + s2;
  const int len = w0 * w1;
  r0_s[t] = -1;
  len_s[t] = 0;
  if (active) {
    for (int k = 0; k < len; k++) acc[k * LD] = 0.f;
    const int lo2 = (DIM == 3) ? d2.node_e0[I2] : 0, hi2 = (DIM == 3) ? lo2 + d2.node_ne[I2] : 1;
    const int lo1 = d1.node_e0[I1], hi1 = lo1 + d1.node_ne[I1];
    const int lo0 = d0.node_e0[I0], hi0 = lo0 + d0.node_ne[I0];
    for (int e2 = lo2; e2 < hi2; e2++) {
      const int f2 = (DIM == 3) ? d2.first[e2] : 0;
      const int b2 = J2 - f2;  // e's axis-2 function at column J2
      if (DIM == 3 && (b2 < 0 || b2 > P)) continue;
      for (int e1 = lo1; e1 < hi1; e1++) {
        const int f1 = d1.first[e1];
        for (int e0 = lo0; e0 < hi0; e0++) {
          const int f0 = d0.first[e0];
          const int a = (I0 - f0) + N1 * ((I1 - f1) + N1 * (I2 - f2));
          const int base = (f1 - l1) * w0 + (f0 - l0);
          const int2 *ga = gtab + a * NEN + (DIM == 3 ? b2 * NB : 0);
          // the slice's values are loaded before any is added: independent loads in flight
          constexpr int CH = NB <= 64 ? NB : 25;
          for (int bc = 0; bc < NB; bc += CH) {
            float ev[CH];
#pragma unroll
            for (int u = 0; u < CH; u++) {
              const int b = bc + u;
              float x = 0.f;
              if (b < NB) {
                const int2 pc = ga[b];  // packed slab of (min(a,b), max(a,b)); column shift off(b) - off(a) for b < a
                x = __ldg(E + (size_t)pc.x * N + A + pc.y);
              }
              ev[u] = x;
            }
#pragma unroll
            for (int u = 0; u < CH; u++) {
              const int b = bc + u;
              if (b >= NB) break;
              const int b0 = b % N1, b1 = b / N1;
              acc[(base + b1 * w0 + b0) * LD] += ev[u];
            }
          }
        }
      }
    }
    bool rowfix = (bnd.flag[0][0] && I0 == 0) || (bnd.flag[0][1] && I0 == d0.n - 1) || (bnd.flag[1][0] && I1 == 0) ||
                  (bnd.flag[1][1] && I1 == d1.n - 1);
    if (DIM == 3) rowfix |= (bnd.flag[2][0] && I2 == 0) || (bnd.flag[2][1] && I2 == d2.n - 1);
    bool fix2 = false;  // the slice's axis-2 column is a Dirichlet one
    if (DIM == 3) fix2 = (bnd.flag[2][0] && J2 == 0) || (bnd.flag[2][1] && J2 == d2.n - 1);
    const float wA = wts ? (float)wts[A] : 1.f;
    for (int k = 0; k < len; k++) {
      const int J0 = l0 + k % w0, J1 = l1 + k / w0;
      const int64_t B = J0 + (int64_t)d0.n * (J1 + (int64_t)d1.n * J2);
      const bool colfix = fix2 || (bnd.flag[0][0] && J0 == 0) || (bnd.flag[0][1] && J0 == d0.n - 1) ||
                          (bnd.flag[1][0] && J1 == 0) || (bnd.flag[1][1] && J1 == d1.n - 1);
      float v = acc[k * LD];
      if (wts) v *= wA * (float)wts[B];
      if (rowfix || colfix) v = (A == B) ? 1.f : 0.f;
      acc[k * LD] = v;
    }
    r0_s[t] = rowptr[A] + (int64_t)s2 * len;
    len_s[t] = len;
  }
  __syncthreads();
  // each row slice is a run of len consecutive CSR values: a warp stores the runs of its
  // own 32 rows one after the other, a lane per value (coalesced)
  const int lane = t & 31, w = t >> 5;
  for (int rr = 0; rr < 32; rr++) {
    const int tt = w * 32 + rr;
    const int64_t r0 = r0_s[tt];
    if (r0 < 0) continue;
    const int n = len_s[tt];
    for (int k = lane; k < n; k += 32) vals[r0 + k] = acc_all[k * LD + tt];
  }
}

}  // namespace

// Host-side plan: element types per direction (elements whose FP64 1D tables agree
// to 1e-12 relative), elements sorted by type into 128-element tiles, the symmetric
// pair list, and the operand and result buffers.
struct ElemGemmPlan {
  bool ok = false;
  int general = 0, nq = 0, nsym = 0, Kp = 0, n_tiles = 0, m_tiles = 0;
  int ngroups = 0, ntypes = 0;
  int *tgroup = nullptr;                 // [ntypes][6]: build groups of the T-tile cache
  uint8_t *Tc[2] = {nullptr, nullptr};   // T-tile cache per operand type (null: built in the GEMM)
  bool tc_tried[2] = {false, false};
  int *slot_of_elem = nullptr, *elem_of_slot = nullptr, *group = nullptr, *pair_ab = nullptr, *pair_off = nullptr,
      *err = nullptr;
  int *group4 = nullptr;                 // [ngroups4][6]: groups of at most EG_PASS_GROUP m-tiles (K passes)
  int ngroups4 = 0;
  int2 *gtab = nullptr;  // [nen][nen]: packed slab of (min, max), and the column shift off(b) - off(a) when b < a
  void *Qv[2] = {nullptr, nullptr};  // BF16, TF32 operand buffers
  float *E = nullptr;
};

static std::vector<int> dir_types(const Dir &D, std::vector<int> &rep) {
  const size_t tsz = (size_t)D.q * (D.p + 1) * 2;
  std::vector<int> type(D.nel, -1);
  rep.clear();
  for (int e = 0; e < D.nel; e++) {
    const double *te = &D.tab[(size_t)e * tsz];
    for (size_t t = 0; t < rep.size() && type[e] < 0; t++) {
      const double *tr = &D.tab[(size_t)rep[t] * tsz];
      bool same = true;
      for (size_t k = 0; k < tsz && same; k++) same = std::fabs(te[k] - tr[k]) <= 1e-12 * (1.0 + std::fabs(tr[k]));
      if (same) type[e] = (int)t;
    }
    if (type[e] < 0) {
      type[e] = (int)rep.size();
      rep.push_back(e);
    }
  }
  return type;
}

static void plan_free(ElemGemmPlan *P) {
  void *ps[] = {P->slot_of_elem, P->elem_of_slot, P->group, P->pair_ab, P->pair_off, P->err, P->Qv[0], P->Qv[1], P->E, P->gtab,
                P->tgroup, P->Tc[0], P->Tc[1], P->group4};
  for (void *p : ps)
    if (p) cudaFree(p);
}

void elem_gemm_release(iga_s *h) {
  if (!h->egemm) return;
  plan_free(h->egemm);
  delete h->egemm;
  h->egemm = nullptr;
}

static cudaError_t elem_gemm_prepare(iga_s *h) {
  if (h->egemm) return h->egemm->ok ? cudaSuccess : cudaErrorNotSupported;
  ElemGemmPlan *P = new ElemGemmPlan();
  h->egemm = P;
  const int dim = h->dim, p = h->p, n1 = p + 1;
  const int nen = dim == 3 ? n1 * n1 * n1 : n1 * n1;
  P->nq = dim == 3 ? h->q * h->q * h->q : h->q * h->q;
  P->general = (h->has_geom || h->has_w) ? 1 : 0;
  const Slots S = make_slots(dim, P->general != 0);
  P->Kp = (S.n * P->nq + 63) / 64 * 64;
  P->nsym = nen * (nen + 1) / 2;  // the upper triangle a <= b, row by row
  P->n_tiles = (P->nsym + GT - 1) / GT;
  // types and tiles
  std::vector<int> rep[3], ty[3];
  for (int ax = 0; ax < 3; ax++) {
    if (ax < dim) ty[ax] = dir_types(h->dir[ax], rep[ax]);
    else { ty[ax].assign(1, 0); rep[ax].assign(1, 0); }
  }
  const int nt0 = (int)rep[0].size(), nt1 = (int)rep[1].size(), nt2 = (int)rep[2].size();
  const int64_t ntypes = (int64_t)nt0 * nt1 * nt2;
  std::vector<int64_t> count(ntypes, 0);
  const int nel0 = h->dir[0].nel, nel1 = h->dir[1].nel;
  auto type_of = [&](int64_t e) {
    const int e0 = (int)(e % nel0), e1 = (int)((e / nel0) % nel1), e2 = (int)(e / ((int64_t)nel0 * nel1));
    return (int64_t)ty[0][e0] + nt0 * ((int64_t)ty[1][e1] + (int64_t)nt1 * ty[2][dim == 3 ? e2 : 0]);
  };
  for (int64_t e = 0; e < h->nelem; e++) count[type_of(e)]++;
  std::vector<int64_t> first_slot(ntypes, 0);
  int64_t m_tiles = 0;
  for (int64_t t = 0; t < ntypes; t++) {
    first_slot[t] = m_tiles * GT;
    m_tiles += (count[t] + GT - 1) / GT;
  }
  // tiles beyond four times the elements (knot vectors with few repeated spans): not worth it
  if (m_tiles * GT > 4 * h->nelem + 64 * GT) return cudaErrorNotSupported;
  P->m_tiles = (int)m_tiles;
  std::vector<int> slot(h->nelem), groups, groups4, tgroups;
  std::vector<int64_t> next = first_slot;
  for (int64_t e = 0; e < h->nelem; e++) {
    const int64_t t = type_of(e);
    slot[e] = (int)next[t]++;
  }
  // work groups: up to G consecutive m-tiles of one type share the T tile; G as large
  // as keeps about two waves of CTAs (three per SM) on the GPU
  int nsm = 152, dev = 0;
  if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  const int64_t EG_GROUP = std::max<int64_t>(1, std::min<int64_t>(EG_GROUP_MAX, m_tiles * P->n_tiles / (2 * 3 * (int64_t)nsm)));
  for (int64_t t = 0; t < ntypes; t++) {
    const int t0 = (int)(t % nt0), t1 = (int)((t / nt0) % nt1), t2 = (int)(t / ((int64_t)nt0 * nt1));
    const int64_t m0 = first_slot[t] / GT, m1 = (first_slot[t] + count[t] + GT - 1) / GT;
    for (int64_t m = m0; m < m1; m += EG_GROUP) {
      groups.push_back((int)m);
      groups.push_back((int)std::min<int64_t>(EG_GROUP, m1 - m));
      groups.push_back(rep[0][t0]);
      groups.push_back(rep[1][t1]);
      groups.push_back(rep[2][t2]);
      groups.push_back((int)t);
    }
    for (int64_t m = m0; m < m1; m += EG_PASS_GROUP) {
      groups4.push_back((int)m);
      groups4.push_back((int)std::min<int64_t>(EG_PASS_GROUP, m1 - m));
      groups4.push_back(rep[0][t0]);
      groups4.push_back(rep[1][t1]);
      groups4.push_back(rep[2][t2]);
      groups4.push_back((int)t);
    }
    tgroups.push_back(0);  // one group per type without element tiles: builds the type's T tiles
    tgroups.push_back(0);
    tgroups.push_back(rep[0][t0]);
    tgroups.push_back(rep[1][t1]);
    tgroups.push_back(rep[2][t2]);
    tgroups.push_back((int)t);
  }
  P->ngroups = (int)(groups.size() / 6);
  P->ngroups4 = (int)(groups4.size() / 6);
  P->ntypes = (int)ntypes;
  std::vector<int> pairs, poff;
  const int64_t n0f = h->dir[0].n, n1f = h->dir[1].n;
  auto off = [&](int a) {
    const int a0 = a % n1, a1 = (a / n1) % n1, a2 = dim == 3 ? a / (n1 * n1) : 0;
    return (int)(a0 + n0f * (a1 + n1f * a2));
  };
  for (int a = 0; a < nen; a++)
    for (int b = a; b < nen; b++) {
      pairs.push_back(a | (b << 16));
      poff.push_back(off(a));
      poff.push_back(off(b));
    }
  std::vector<int2> gt((size_t)nen * nen);
  for (int a = 0; a < nen; a++)
    for (int b = 0; b < nen; b++) {
      const int lo = std::min(a, b), hi = std::max(a, b);
      gt[(size_t)a * nen + b] = make_int2(lo * nen - lo * (lo - 1) / 2 + (hi - lo), b < a ? off(b) - off(a) : 0);
    }
  std::vector<int> eos((size_t)m_tiles * GT, -1);
  for (int64_t e = 0; e < h->nelem; e++) eos[slot[e]] = (int)e;
  const size_t slots_total = (size_t)m_tiles * GT;
  cudaError_t ce;
  if ((ce = cudaMalloc((void **)&P->slot_of_elem, slot.size() * sizeof(int)))) return ce;
  if ((ce = cudaMemcpy(P->slot_of_elem, slot.data(), slot.size() * sizeof(int), cudaMemcpyHostToDevice))) return ce;
  if ((ce = cudaMalloc((void **)&P->group, groups.size() * sizeof(int)))) return ce;
  if ((ce = cudaMemcpy(P->group, groups.data(), groups.size() * sizeof(int), cudaMemcpyHostToDevice))) return ce;
  if ((ce = cudaMalloc((void **)&P->group4, groups4.size() * sizeof(int)))) return ce;
  if ((ce = cudaMemcpy(P->group4, groups4.data(), groups4.size() * sizeof(int), cudaMemcpyHostToDevice))) return ce;
  if ((ce = cudaMalloc((void **)&P->tgroup, tgroups.size() * sizeof(int)))) return ce;
  if ((ce = cudaMemcpy(P->tgroup, tgroups.data(), tgroups.size() * sizeof(int), cudaMemcpyHostToDevice))) return ce;
  if ((ce = cudaMalloc((void **)&P->pair_ab, pairs.size() * sizeof(int)))) return ce;
  if ((ce = cudaMemcpy(P->pair_ab, pairs.data(), pairs.size() * sizeof(int), cudaMemcpyHostToDevice))) return ce;
  if ((ce = cudaMalloc((void **)&P->pair_off, poff.size() * sizeof(int)))) return ce;
  if ((ce = cudaMemcpy(P->pair_off, poff.data(), poff.size() * sizeof(int), cudaMemcpyHostToDevice))) return ce;
  if ((ce = cudaMalloc((void **)&P->gtab, gt.size() * sizeof(int2)))) return ce;
  if ((ce = cudaMemcpy(P->gtab, gt.data(), gt.size() * sizeof(int2), cudaMemcpyHostToDevice))) return ce;
  if ((ce = cudaMalloc((void **)&P->elem_of_slot, eos.size() * sizeof(int)))) return ce;
  if ((ce = cudaMemcpy(P->elem_of_slot, eos.data(), eos.size() * sizeof(int), cudaMemcpyHostToDevice))) return ce;
  if ((ce = cudaMalloc((void **)&P->err, sizeof(int)))) return ce;
  if ((ce = cudaMemset(P->err, 0, sizeof(int)))) return ce;
  if ((ce = cudaMalloc((void **)&P->E, (size_t)P->nsym * h->N * sizeof(float)))) return ce;
  (void)slots_total;
  P->ok = true;
  return cudaSuccess;
}

static cudaError_t qv_buffer(iga_s *h, int op, void **out) {
  ElemGemmPlan *P = h->egemm;
  const size_t es = op == EG_BF16 ? 2 : 4;
  if (!P->Qv[op]) {
    const size_t bytes = (size_t)P->m_tiles * GT * P->Kp * es;
    cudaError_t ce = cudaMalloc(&P->Qv[op], bytes);
    if (ce) return ce;
    ce = cudaMemsetAsync(P->Qv[op], 0, bytes, h->stream);  // padding rows and K columns stay zero
    if (ce) return ce;
  }
  *out = P->Qv[op];
  return cudaSuccess;
}

#define EG_DISPATCH(DIM_, P_, CALL)                         \
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

// K passes of the element GEMM for an operand type: one when the T tile of the whole K
// fits in shared memory, else as few as keep EG_PASS_CHUNKS chunks resident.
static int eg_passes(int nch) {
  if (eg_smem(nch, 0) <= 200 * 1024) return 1;
  return (nch + EG_PASS_CHUNKS - 1) / EG_PASS_CHUNKS;
}

// The element-type plan exists (knot vectors whose spans repeat enough) and either the T
// tile of the whole K fits in shared memory for the operand type, or it does not and the
// per-element contraction (iga_mixed.cu: 2D p <= 4, 3D p <= 3) cannot take the case: then
// K runs in passes (3D p = 4 in TF32, and with a general map in BF16 too).
bool elem_gemm_supported(iga_s *h, int prec) {
  if (elem_gemm_prepare(h) != cudaSuccess) return false;
  const int es = prec == IGA_JAC_BF16 ? 2 : 4;
  return eg_passes(h->egemm->Kp * es / KB) == 1 || !mixed_supported(h->dim, h->p);
}

// vals (FP32, CSR) = the Jacobian with BF16 (prec IGA_JAC_BF16) or TF32 element
// contractions: Q00 at U in FP64 (launch_q00), the operand rows, the GEMM, the gather.
// h->tab32 must hold the FP32 tables.
cudaError_t launch_jacobian_elem_gemm(iga_s *h, const double *U, float *vals, int prec) {
  if (!elem_gemm_supported(h, prec)) return cudaErrorNotSupported;
  cudaError_t ce;
  ElemGemmPlan *P = h->egemm;
  const int op = prec == IGA_JAC_BF16 ? EG_BF16 : EG_TF32;
  void *Qv = nullptr;
  if ((ce = qv_buffer(h, op, &Qv))) return ce;
  h->q00_valid = false;
  DirArgs a0 = dir_args(h->ddev[0]), a1 = dir_args(h->ddev[1]), a2 = dir_args(h->ddev[2]);
  IGA_LAUNCH(h, KC_Q00, EG_DISPATCH(h->dim, h->p, ({
    using IS = InterpF32<D, PP>;
    const unsigned gq = (unsigned)((h->nelem + IS::EB - 1) / IS::EB);
    constexpr int PE = (D == 2 || PP <= 2) ? PP : 2;  // small elements: one thread per element
    const unsigned ge = (unsigned)((h->nelem + 127) / 128);
    if (D == 2 || PP <= 2) {
      if (op == EG_BF16)
        k_qv_e<D, PE, EG_BF16><<<ge, 128, 0, h->stream>>>(a0, a1, a2, U, h->weights, h->geom32, (float)h->lambda,
                                                          P->slot_of_elem, Qv, P->Kp, P->general, h->nelem);
      else
        k_qv_e<D, PE, EG_TF32><<<ge, 128, 0, h->stream>>>(a0, a1, a2, U, h->weights, h->geom32, (float)h->lambda,
                                                          P->slot_of_elem, Qv, P->Kp, P->general, h->nelem);
    } else if (op == EG_BF16)
      k_qv<D, PP, EG_BF16><<<gq, IS::THREADS, 0, h->stream>>>(a0, a1, a2, U, h->weights, h->geom32, (float)h->lambda,
                                                              P->slot_of_elem, Qv, P->Kp, P->general, h->nelem);
    else
      k_qv<D, PP, EG_TF32><<<gq, IS::THREADS, 0, h->stream>>>(a0, a1, a2, U, h->weights, h->geom32, (float)h->lambda,
                                                              P->slot_of_elem, Qv, P->Kp, P->general, h->nelem);
  })));
  GemmArgs g;
  g.Qv = Qv;
  g.E = P->E;
  g.elem_of_slot = P->elem_of_slot;
  for (int ax = 0; ax < 3; ax++) g.first[ax] = ax < h->dim ? h->ddev[ax].first : nullptr;
  g.pair_off = P->pair_off;
  g.nel0 = h->dir[0].nel;
  g.nel1 = h->dir[1].nel;
  g.N = h->N;
  g.N0 = h->dir[0].n;
  g.N1 = h->dir[1].n;
  g.nen = h->dim == 3 ? (h->p + 1) * (h->p + 1) * (h->p + 1) : (h->p + 1) * (h->p + 1);
  for (int ax = 0; ax < 3; ax++) g.tab[ax] = ax < h->dim ? h->tab32[ax] : nullptr;
  g.group = P->group;
  g.pair_ab = P->pair_ab;
  g.dim = h->dim;
  g.p = h->p;
  g.nq = P->nq;
  g.nsym = P->nsym;
  g.Kp = P->Kp;
  g.n_tiles = P->n_tiles;
  g.m_tiles = P->m_tiles;
  g.general = P->general;
  g.err = P->err;
  g.limit_ns = h->wait_limit_ns;
  g.stall = 0;
  const int nch = P->Kp * (op == EG_BF16 ? 2 : 4) / KB;
  g.npass = eg_passes(nch);
  const int pcs = (nch + g.npass - 1) / g.npass;
  g.split = (g.npass == 1 && eg_smem(nch, 1) <= 200 * 1024) ? 1 : 0;
  const size_t smem = eg_smem(pcs, g.split);
  g.tile_bytes = (int64_t)nch * (1 + g.split) * STAGE;
  g.Tc = nullptr;
  g.Tout = nullptr;
  if (op == EG_BF16) cudaFuncSetAttribute(k_elem_gemm<EG_BF16>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  else cudaFuncSetAttribute(k_elem_gemm<EG_TF32>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  // the T tiles depend on the mesh only: built once (when they take at most 1 GB) and copied by the GEMM
  if (!P->tc_tried[op]) {
    P->tc_tried[op] = true;
    const int64_t bytes = (int64_t)P->ntypes * P->n_tiles * g.tile_bytes;
    if (bytes <= (int64_t)1 << 30 && cudaMalloc((void **)&P->Tc[op], bytes) == cudaSuccess) {
      GemmArgs gb = g;
      gb.group = P->tgroup;
      gb.Tout = P->Tc[op];
      const unsigned gridb = (unsigned)((int64_t)P->ntypes * P->n_tiles);
      if (op == EG_BF16) IGA_LAUNCH(h, KC_ELEM_TC, (k_elem_gemm<EG_BF16><<<gridb, 256, smem, h->stream>>>(gb)));
      else IGA_LAUNCH(h, KC_ELEM_TC, (k_elem_gemm<EG_TF32><<<gridb, 256, smem, h->stream>>>(gb)));
      if ((ce = cudaGetLastError())) return ce;
    } else {
      cudaGetLastError();  // a failed allocation only means no cache
      P->Tc[op] = nullptr;
    }
  }
  g.Tc = P->Tc[op];
  g.stall = h->stall_next ? 1 : 0;
  h->stall_next = false;
  // with K passes a CTA keeps one accumulator per m-tile: groups of at most EG_PASS_GROUP
  if (g.npass > 1) g.group = P->group4;
  const unsigned grid = (unsigned)((int64_t)(g.npass > 1 ? P->ngroups4 : P->ngroups) * P->n_tiles);
  if (op == EG_BF16) {
    IGA_LAUNCH(h, KC_ELEM_TC, (k_elem_gemm<EG_BF16><<<grid, 256, smem, h->stream>>>(g)));
  } else {
    IGA_LAUNCH(h, KC_ELEM_TC, (k_elem_gemm<EG_TF32><<<grid, 256, smem, h->stream>>>(g)));
  }
  if ((ce = cudaGetLastError())) return ce;
  IGA_LAUNCH(h, KC_ELEM_GATHER, EG_DISPATCH(h->dim, h->p, ({
    constexpr int RMAX = (2 * PP + 1) * (2 * PP + 1);  // columns of a thread's slice
    constexpr int TPB = 128;
    constexpr int NENc = ipow3<D>(PP + 1);
    const size_t sm = (size_t)((RMAX * (TPB + 1) + 1) / 2 * 2) * sizeof(float) +
                      (NENc * NENc * 8 <= 8 * 1024 ? (size_t)NENc * NENc * 8 : 0);
    if (sm > 48 * 1024) cudaFuncSetAttribute(k_gather_rows<D, PP, TPB>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    const unsigned chunks = (unsigned)((h->N + TPB - 1) / TPB);
    const int slice_major = (D == 3 && chunks <= 65535u) ? 1 : 0;
    const dim3 gg = slice_major ? dim3(2 * PP + 1, chunks) : dim3(chunks, D == 3 ? 2 * PP + 1 : 1);
    k_gather_rows<D, PP, TPB><<<gg, TPB, sm, h->stream>>>(a0, a1, a2, P->E, P->gtab, h->rowptr, h->weights, h->bnd, vals,
                                                          h->N, slice_major);
  })));
  return cudaGetLastError();
}

// Error flag of the element GEMM (a pipeline wait that gave up): read on the handle's
// stream (which this synchronises) and cleared for the next launch.
bool elem_gemm_failed(iga_s *h) {
  if (!h->egemm || !h->egemm->err) return false;
  int v = 0;
  if (cudaMemcpyAsync(&v, h->egemm->err, sizeof(int), cudaMemcpyDeviceToHost, h->stream) != cudaSuccess) return false;
  if (cudaStreamSynchronize(h->stream) != cudaSuccess) return false;
  if (v) {
    cudaMemsetAsync(h->egemm->err, 0, sizeof(int), h->stream);
    cudaStreamSynchronize(h->stream);
  }
  return v != 0;
}
