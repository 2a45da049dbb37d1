// 3x3 dilated convolutions of the neural operator as implicit GEMMs on the
// 5th-generation tensor cores (tcgen05.mma, BF16 operands, FP32 accumulator in
// tensor memory).
//
//   out[p][n] = sum_{tap < 9} sum_{c < CIN} in[p + sign * off(tap)][c] * Wk[n][tap][c]
//
// p runs over the B*H*W pixels (NHWC rows of CIN BF16 values), off(tap) =
// dil * (tap/3 - 1, tap%3 - 1) in (y, x), and a source pixel outside the grid
// reads zero ("same" padding).  sign = +1 is the forward convolution; sign = -1
// with Wk[ci][tap][co] = W[co][tap][ci] is its input gradient (the transposed
// convolution).  The GEMM is M = 128 pixels per tile, N = NOUT, K = 9 * CIN.
//
// One persistent CTA per SM, warp-specialised (416 threads):
//   - warps 8-11 (producers): thread j gathers pixel row j of the shifted, dilated
//     input for each (tile, tap) with 16-byte cp.async copies (zero-filled outside
//     the grid) into an 8-stage ring; once its copies of a stage have landed it
//     fences them into the async proxy and arrives on the stage's "full" barrier;
//     it refills a stage after the stage's "empty" barrier reports the MMAs that
//     read it complete;
//   - warp 12 (MMA): allocates tensor memory; one thread waits for "full", issues
//     the tap's CIN/16 tcgen05.mma instructions (K = 16, FP32 accumulator in
//     TMEM) and commits them to "empty"; after the ninth tap it commits the
//     accumulator to "acc full";
//   - warps 0-7 (epilogue): warp w reads accumulator rows 32 (w % 4) .. + 31
//     (pixels of the tile; a warp may only address its quarter of the TMEM
//     lanes), columns of half w / 4, with tcgen05.ld, applies the fused epilogue
//     (bias + SiLU, or the SiLU derivative of the layer below), stores, and
//     arrives on "acc empty".
//   Two accumulators in TMEM (2 x NOUT columns) let the epilogue of one tile
//   overlap the MMAs of the next; the layer's weights stay in shared memory.
// Operand tiles use the canonical K-major layout without swizzling: 8-row x
// 16-byte core matrices, 128 bytes apart along M/N (SBO) and one column of
// core matrices per 8 K values (LBO).  Every mbarrier wait is bounded in time
// (globaltimer); on timeout the kernel raises an error flag, every role stops,
// the MMA thread waits (bounded) for its last commit, and the tensor memory is
// freed before the kernel returns.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>

#include "iga_internal.h"
#include "iga_conv_tc.h"
#include "iga_tc.h"

namespace {

typedef __nv_bfloat16 bf16;

// logistic function with the fast exponential and division intrinsics (the
// activations are rounded to BF16 afterwards)
__device__ __forceinline__ float sigm(float z) { return __fdividef(1.f, 1.f + __expf(-z)); }

__device__ __forceinline__ uint32_t pack2(float a, float b) {
  __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
  return *reinterpret_cast<uint32_t *>(&h);
}

constexpr int CONV_EPI_WARPS = 8;  // two per quarter of the TMEM lanes, each half the columns
constexpr int CONV_PRODUCER0 = CONV_EPI_WARPS;       // first producer warp (4 producer warps)
constexpr int CONV_MMA_WARP = CONV_EPI_WARPS + 4;
constexpr int CONV_THREADS = 32 * (CONV_EPI_WARPS + 5);
constexpr int CONV_STAGES = 8;
constexpr int CONV_LAG = 5;        // copy groups a producer keeps in flight beyond the one it signals

template <int CIN, int NOUT>
struct ConvSmem {
  static constexpr uint32_t SBO = 128;                 // next 8 rows (M or N)
  static constexpr uint32_t LBO_A = 128 * 16;          // next 8 K values of an A tile (16 row groups)
  static constexpr uint32_t LBO_W = 128 * (NOUT / 8);  // next 8 K values of the weight tile
  static constexpr uint32_t A_BYTES = 128 * CIN * 2;
  static constexpr uint32_t W_BYTES = NOUT * 9 * CIN * 2;
  static constexpr uint32_t BAR = W_BYTES + CONV_STAGES * A_BYTES;
  // barriers: full[S], empty[S], acc_full[2], acc_empty[2]; the TMEM slot and the abort
  // flag; the bias
  static constexpr uint32_t BIAS = BAR + 8 * (2 * CONV_STAGES + 4) + 16;
  static constexpr uint32_t TOTAL = BIAS + 4 * NOUT;
  static constexpr uint32_t TMEM_COLS = 2 * NOUT < 32 ? 32 : 2 * NOUT;  // two accumulators
};

// columns [cb, cb + CW) of accumulator row p (taddr: the row's lane, column 0)
template <int CIN, int NOUT, int EPI, int CW>
__device__ __forceinline__ void conv_epilogue(const ConvArgs &a, uint32_t taddr, int p, int cb, const float *bias_s) {
  if constexpr (EPI == CONV_EPI_LAST) {
    float v[16];
    tmem_ld16(taddr, v);
    if (p < a.P) a.z[p] = v[0] + bias_s[0];
  } else {
#pragma unroll
  for (int c0 = cb; c0 < cb + CW; c0 += 16) {
    float v[16];
    tmem_ld16(taddr + c0, v);
    if (p >= a.P) continue;
    float d[16];
    if constexpr (EPI == CONV_EPI_FWD_SILU) {
#pragma unroll
      for (int j = 0; j < 16; j++) d[j] = v[j] + bias_s[c0 + j];
      if (a.z) {
        float4 *z4 = reinterpret_cast<float4 *>(a.z + (size_t)p * NOUT + c0);
#pragma unroll
        for (int q = 0; q < 4; q++) z4[q] = make_float4(d[4 * q], d[4 * q + 1], d[4 * q + 2], d[4 * q + 3]);
      }
#pragma unroll
      for (int j = 0; j < 16; j++) d[j] = d[j] * sigm(d[j]);
    } else {  // CONV_EPI_BWD_SILU: d = v * SiLU'(z of the layer below)
      const float4 *zp = reinterpret_cast<const float4 *>(a.zprev + (size_t)p * NOUT + c0);
#pragma unroll
      for (int q = 0; q < 4; q++) {
        const float4 z = zp[q];
        const float zz[4] = {z.x, z.y, z.z, z.w};
#pragma unroll
        for (int u = 0; u < 4; u++) {
          const float sg = sigm(zz[u]);
          d[4 * q + u] = v[4 * q + u] * sg * (1.f + zz[u] * (1.f - sg));
        }
      }
      float4 *z4 = reinterpret_cast<float4 *>(a.z + (size_t)p * NOUT + c0);
#pragma unroll
      for (int q = 0; q < 4; q++) z4[q] = make_float4(d[4 * q], d[4 * q + 1], d[4 * q + 2], d[4 * q + 3]);
    }
    uint4 o[2];
    uint32_t *ow = reinterpret_cast<uint32_t *>(o);
#pragma unroll
    for (int j = 0; j < 8; j++) ow[j] = pack2(d[2 * j], d[2 * j + 1]);
    uint4 *dst = reinterpret_cast<uint4 *>(a.act + (size_t)p * NOUT + c0);
    dst[0] = o[0];
    dst[1] = o[1];
  }
  }
}

template <int CIN, int NOUT, int EPI>
__global__ void __launch_bounds__(CONV_THREADS, 1) k_conv_tc(ConvArgs a) {
  using SM = ConvSmem<CIN, NOUT>;
  constexpr int KCH = CIN / 8, KSTEPS = CIN / 16, S = CONV_STAGES, LAG = CONV_LAG;
  static_assert(CIN % 16 == 0 && NOUT % 16 == 0 && NOUT <= 128, "tile shape");
  extern __shared__ __align__(128) uint8_t sm[];
  uint8_t *Ws = sm;
  uint8_t *As = sm + SM::W_BYTES;
  uint64_t *full = reinterpret_cast<uint64_t *>(sm + SM::BAR);
  uint64_t *empty = full + S;
  uint64_t *accf = empty + S;
  uint64_t *acce = accf + 2;
  uint32_t *slot = reinterpret_cast<uint32_t *>(acce + 2);
  volatile int *abort_s = reinterpret_cast<volatile int *>(slot + 1);
  float *bias_s = reinterpret_cast<float *>(sm + SM::BIAS);
  const int tid = threadIdx.x, warp = tid >> 5;
  const int ntiles = (a.P + 127) / 128;
  const int my_tiles = (int)blockIdx.x < ntiles ? (ntiles - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;
  const int total_it = my_tiles * 9;

  // the layer's weights, resident for the whole kernel
  for (int c = tid; c < NOUT * 9 * KCH; c += CONV_THREADS) {
    const int n = c % NOUT, kc = c / NOUT;
    cp16(su32(Ws + (n / 8) * SM::SBO + kc * SM::LBO_W + (n % 8) * 16), a.wk + (size_t)n * 9 * CIN + kc * 8, true);
  }
  cp_commit();
  for (int c = tid; c < NOUT; c += CONV_THREADS) bias_s[c] = a.bias ? a.bias[c] : 0.f;
  if (warp == CONV_MMA_WARP) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(slot)), "r"(SM::TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 0) {
    for (int i = 0; i < S; i++) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 128;" ::"r"(su32(full + i)) : "memory");
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(su32(empty + i)) : "memory");
    }
    for (int i = 0; i < 2; i++) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(su32(accf + i)) : "memory");
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(su32(acce + i)), "n"(32 * CONV_EPI_WARPS) : "memory");
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    *abort_s = 0;
  }
  cp_wait<0>();
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *slot;

  if (warp >= CONV_PRODUCER0 && warp < CONV_MMA_WARP) {
    // ---------------- producers ----------------
    const int j = tid - 32 * CONV_PRODUCER0;  // pixel row within the tile
    const int HW = a.H * a.W;
    int pb = 0, py = 0, px = 0;                // this row's pixel (image, y, x) in the current tile
    bool pin = false;
    int it = 0;
    for (; it < total_it; it++) {
      const int s = it % S;
      if (it >= S && !mbar_wait(su32(empty + s), ((it / S) - 1) & 1, abort_s)) {
        atomicExch(a.err, 1);
        *abort_s = 1;
        break;
      }
      const int tl = it / 9, tap = it - tl * 9;
      if (tap == 0) {
        const int p = ((int)blockIdx.x + tl * (int)gridDim.x) * 128 + j;
        pin = p < a.P;
        if (pin) {
          pb = p / HW;
          const int r = p - pb * HW;
          py = r / a.W;
          px = r - py * a.W;
        }
      }
      const int sy = py + (tap / 3 - 1) * a.dil * a.sign, sx = px + (tap % 3 - 1) * a.dil * a.sign;
      const bool valid = pin && sy >= 0 && sy < a.H && sx >= 0 && sx < a.W;
      const bf16 *src = valid ? a.in + ((size_t)pb * HW + (size_t)sy * a.W + sx) * CIN : a.in;
      const uint32_t dst = su32(As + s * SM::A_BYTES + (j / 8) * SM::SBO + (j % 8) * 16);
#pragma unroll
      for (int kc = 0; kc < KCH; kc++) cp16(dst + kc * SM::LBO_A, src + kc * 8, valid);
      cp_commit();
      if (it >= LAG) {
        cp_wait<LAG>();  // the copies of iteration it - LAG have landed
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        mbar_arrive(su32(full + (it - LAG) % S));
      }
    }
    cp_wait<0>();
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    for (int k = (it > LAG ? it - LAG : 0); k < it; k++) mbar_arrive(su32(full + k % S));
  } else if (warp == CONV_MMA_WARP) {
    // ---------------- MMA issuer ----------------
    if ((tid & 31) == 0) {
      const uint32_t idesc =
          (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(NOUT >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
      const uint64_t adesc0 = sdesc(su32(As), SM::LBO_A, SM::SBO), bdesc0 = sdesc(su32(Ws), SM::LBO_W, SM::SBO);
      int last = -1;  // last iteration whose MMAs were committed
      for (int it = 0; it < total_it; it++) {
        const int s = it % S, tl = it / 9, tap = it - tl * 9, buf = tl & 1;
        if (tap == 0 && tl >= 2 && !mbar_wait(su32(acce + buf), ((tl / 2) - 1) & 1, abort_s)) {
          atomicExch(a.err, 1);
          *abort_s = 1;
          break;
        }
        if (!mbar_wait(su32(full + s), (it / S) & 1, abort_s)) {
          atomicExch(a.err, 1);
          *abort_s = 1;
          break;
        }
        tc_fence_after();
        // descriptors by addition to the start-address field (bytes / 16)
        const uint64_t ad0 = adesc0 + (uint64_t)((s * SM::A_BYTES) >> 4);
        const uint64_t bd0 = bdesc0 + (uint64_t)((tap * KSTEPS * 2 * SM::LBO_W) >> 4);
        const uint32_t d = tmem + (uint32_t)(buf * NOUT);
#pragma unroll
        for (int k = 0; k < KSTEPS; k++) {
          const uint32_t acc = (tap > 0 || k > 0) ? 1u : 0u;
          asm volatile(
              "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
              "l"(ad0 + (uint64_t)((k * 2 * SM::LBO_A) >> 4)), "l"(bd0 + (uint64_t)((k * 2 * SM::LBO_W) >> 4)), "r"(idesc),
              "r"(acc)
              : "memory");
        }
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(su32(empty + s))
                     : "memory");
        if (tap == 8)
          asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(su32(accf + buf))
                       : "memory");
        last = it;
      }
      // after a failure, let the MMAs already issued finish before the memory is freed
      if (*abort_s && last >= 0) mbar_wait(su32(empty + last % S), (last / S) & 1, nullptr);
    }
    __syncwarp();
  } else {
    // ---------------- epilogue: warp w reads TMEM lanes 32 (w % 4) .. + 31 ----------------
    constexpr int CW = NOUT / 2 < 16 ? 16 : NOUT / 2;  // columns per warp
    const int quarter = warp & 3, cb = (warp >> 2) * CW;
    for (int tl = 0; tl < my_tiles; tl++) {
      const int buf = tl & 1;
      if (!mbar_wait(su32(accf + buf), (tl / 2) & 1, abort_s)) {
        atomicExch(a.err, 1);
        *abort_s = 1;
        break;
      }
      tc_fence_after();
      const int p = ((int)blockIdx.x + tl * (int)gridDim.x) * 128 + quarter * 32 + (tid & 31);
      if (cb < NOUT)
        conv_epilogue<CIN, NOUT, EPI, CW>(a, tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(buf * NOUT), p, cb, bias_s);
      tc_fence_before();
      mbar_arrive(su32(acce + buf));
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == CONV_MMA_WARP) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(SM::TMEM_COLS) : "memory");
  }
}

// ---------------------------------------------------------------------------
// Weight gradient of the convolution on the tensor cores:
//   dW[co][tap][ci] = sum_p dZ[p][co] * X[p + off(tap)][ci]
// as D[(tap, ci)][co] = sum_p A[(tap, ci)][p] B[co][p] with the pixels as K.
// Both operands keep their natural NHWC layout in the canonical MN-major form
// (core matrix = 8 pixels x 16 bytes of 8 consecutive channels; LBO = stride
// between 8-pixel groups, SBO = stride between 8-channel groups), so the
// producers copy 16-byte channel chunks without transposing.  M = 9 * CIN rows
// in ceil(9 CIN / 128) tiles of 128 (the tail rows are zero), N = NOUT, one
// TMEM accumulator per M tile.  Each CTA reduces a contiguous pixel range
// (split K) in steps of 32 pixels through a 4-stage ring (producer warps 4-7,
// MMA warp 8), then warps 0-3 write its partial dW; k_wgrad_sum adds the
// partials of all CTAs in index order.
// ---------------------------------------------------------------------------
constexpr int WG_THREADS = 288;
constexpr int WG_STAGES = 4;
constexpr int WG_BK = 32;  // pixels per stage

template <int CIN, int NOUT>
struct WgSmem {
  static constexpr int MT = (9 * CIN + 127) / 128;        // M tiles
  static constexpr uint32_t A_TILE = 128 * WG_BK * 2;     // one M tile of a stage
  static constexpr uint32_t A_BYTES = MT * A_TILE;
  static constexpr uint32_t B_BYTES = NOUT * WG_BK * 2;
  static constexpr uint32_t STAGE = A_BYTES + B_BYTES;
  static constexpr uint32_t CK_A = 128 * 16;              // next 8 pixels of an A tile (16 channel groups)
  static constexpr uint32_t CK_B = 128 * (NOUT / 8);      // next 8 pixels of the B tile
  static constexpr uint32_t BAR = WG_STAGES * STAGE;
  static constexpr uint32_t TOTAL = BAR + 8 * (2 * WG_STAGES + 1) + 16;
  static constexpr uint32_t COLS = MT * NOUT;
  static constexpr uint32_t TMEM_COLS = COLS <= 32 ? 32 : COLS <= 64 ? 64 : COLS <= 128 ? 128 : COLS <= 256 ? 256 : 512;
};

template <int CIN, int NOUT>
__global__ void __launch_bounds__(WG_THREADS, 1) k_conv_wgrad_tc(WgradArgs a) {
  using SM = WgSmem<CIN, NOUT>;
  constexpr int S = WG_STAGES, LAG = 2, MT = SM::MT;
  constexpr int NCH_A = 9 * (CIN / 8) * WG_BK;  // 16-byte chunks of A per stage
  constexpr int NCH_B = (NOUT / 8) * WG_BK;
  static_assert(SM::COLS <= 512, "accumulators exceed tensor memory");
  extern __shared__ __align__(128) uint8_t sm[];
  uint64_t *full = reinterpret_cast<uint64_t *>(sm + SM::BAR);
  uint64_t *empty = full + S;
  uint64_t *done_bar = empty + S;
  uint32_t *slot = reinterpret_cast<uint32_t *>(done_bar + 1);
  volatile int *abort_s = reinterpret_cast<volatile int *>(slot + 1);
  const int tid = threadIdx.x, warp = tid >> 5;
  // this CTA's pixel range, in whole steps
  const int nsteps_all = (a.P + WG_BK - 1) / WG_BK;
  const int per = (nsteps_all + (int)gridDim.x - 1) / (int)gridDim.x;
  const int s0 = (int)blockIdx.x * per;
  const int nsteps = max(0, min(per, nsteps_all - s0));

  // zero the M tail rows of every stage once (never written by the producers)
  if (9 * CIN < MT * 128) {
    for (int st = 0; st < S; st++) {
      uint8_t *tile = sm + st * SM::STAGE + (MT - 1) * SM::A_TILE;
      const int r0 = 9 * CIN - (MT - 1) * 128;  // first unused row of the last tile (multiple of 16)
      for (int c = tid; c < (128 - r0) / 8 * (WG_BK / 8) * 8; c += WG_THREADS) {
        const int g = r0 / 8 + c / (WG_BK), k = c % WG_BK;
        *reinterpret_cast<uint4 *>(tile + g * 128 + (k / 8) * SM::CK_A + (k % 8) * 16) = make_uint4(0, 0, 0, 0);
      }
    }
  }
  if (warp == 8) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(slot)), "r"(SM::TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 0) {
    for (int i = 0; i < S; i++) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 128;" ::"r"(su32(full + i)) : "memory");
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(su32(empty + i)) : "memory");
    }
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(su32(done_bar)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    *abort_s = 0;
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *slot;
  const int HW = a.H * a.W;

  if (warp >= 4 && warp < 8) {
    // ---------------- producers ----------------
    const int j = tid - 128;
    int it = 0;
    for (; it < nsteps; it++) {
      const int s = it % S;
      if (it >= S && !mbar_wait(su32(empty + s), ((it / S) - 1) & 1, abort_s)) {
        atomicExch(a.err, 1);
        *abort_s = 1;
        break;
      }
      const int pbase = (s0 + it) * WG_BK;
      uint8_t *st = sm + s * SM::STAGE;
      // A: chunk c -> (tap, channel group g, pixel k), pixel fastest
      for (int c = j; c < NCH_A; c += 128) {
        const int k = c % WG_BK, rest = c / WG_BK, g = rest % (CIN / 8), tap = rest / (CIN / 8);
        const int p = pbase + k;
        bool valid = false;
        const bf16 *src = a.x;
        if (p < a.P) {
          const int b = p / HW, r = p - b * HW, y = r / a.W, xx = r - y * a.W;
          const int sy = y + (tap / 3 - 1) * a.dil, sx = xx + (tap % 3 - 1) * a.dil;
          if (sy >= 0 && sy < a.H && sx >= 0 && sx < a.W) {
            valid = true;
            src = a.x + ((size_t)b * HW + (size_t)sy * a.W + sx) * CIN + g * 8;
          }
        }
        const int m = tap * CIN + g * 8;  // first row of the chunk
        cp16(su32(st + (m / 128) * SM::A_TILE + ((m % 128) / 8) * 128 + (k / 8) * SM::CK_A + (k % 8) * 16), src, valid);
      }
      // B: chunk c -> (channel group g, pixel k)
      for (int c = j; c < NCH_B; c += 128) {
        const int k = c % WG_BK, g = c / WG_BK;
        const int p = pbase + k;
        const bool valid = p < a.P && g * 8 < a.ldz;
        const bf16 *src = valid ? a.dz + (size_t)p * a.ldz + g * 8 : a.dz;
        cp16(su32(st + SM::A_BYTES + g * 128 + (k / 8) * SM::CK_B + (k % 8) * 16), src, valid);
      }
      cp_commit();
      if (it >= LAG) {
        cp_wait<LAG>();
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        mbar_arrive(su32(full + (it - LAG) % S));
      }
    }
    cp_wait<0>();
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    for (int k = (it > LAG ? it - LAG : 0); k < it; k++) mbar_arrive(su32(full + k % S));
  } else if (warp == 8) {
    // ---------------- MMA issuer ----------------
    if ((tid & 31) == 0) {
      // FP32 accumulator, BF16 A and B, both MN-major, N = NOUT, M = 128
      const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | (1u << 15) | (1u << 16) |
                             ((uint32_t)(NOUT >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
      const uint64_t adesc0 = sdesc(su32(sm), SM::CK_A, 128), bdesc0 = sdesc(su32(sm + SM::A_BYTES), SM::CK_B, 128);
      int last = -1;
      for (int it = 0; it < nsteps; it++) {
        const int s = it % S;
        if (!mbar_wait(su32(full + s), (it / S) & 1, abort_s)) {
          atomicExch(a.err, 1);
          *abort_s = 1;
          break;
        }
        tc_fence_after();
        const uint64_t soff = (uint64_t)((s * SM::STAGE) >> 4);
#pragma unroll
        for (int mt = 0; mt < MT; mt++)
#pragma unroll
          for (int kk = 0; kk < WG_BK / 16; kk++) {
            const uint64_t ad = adesc0 + soff + (uint64_t)((mt * SM::A_TILE + 2 * kk * SM::CK_A) >> 4);
            const uint64_t bd = bdesc0 + soff + (uint64_t)((2 * kk * SM::CK_B) >> 4);
            const uint32_t acc = (it > 0 || kk > 0) ? 1u : 0u;
            asm volatile(
                "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(
                    tmem + (uint32_t)(mt * NOUT)),
                "l"(ad), "l"(bd), "r"(idesc), "r"(acc)
                : "memory");
          }
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(su32(empty + s))
                     : "memory");
        last = it;
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(su32(done_bar))
                   : "memory");
      if (*abort_s && last >= 0) mbar_wait(su32(empty + last % S), (last / S) & 1, nullptr);
    }
    __syncwarp();
  } else if (warp < 4) {
    // ---------------- partial dW of this CTA (rows of TMEM lane quarter `warp`) ----------------
    const bool ok = mbar_wait(su32(done_bar), 0, abort_s, 256);
    if (!ok) {
      atomicExch(a.err, 1);
      *abort_s = 1;
    }
    tc_fence_after();
    float *out = a.part + (size_t)blockIdx.x * NOUT * 9 * CIN;
    const int lane_row = warp * 32 + (tid & 31);
#pragma unroll 1
    for (int mt = 0; mt < MT; mt++) {
      const int m = mt * 128 + lane_row;  // (tap, ci)
#pragma unroll 1
      for (int c0 = 0; c0 < NOUT; c0 += 16) {
        float v[16];
        if (ok && nsteps > 0) tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(mt * NOUT + c0), v);
        else
          for (int q = 0; q < 16; q++) v[q] = 0.f;
        if (m < 9 * CIN)
          for (int q = 0; q < 16; q++) out[(size_t)(c0 + q) * 9 * CIN + m] = v[q];
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 8) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(SM::TMEM_COLS) : "memory");
  }
}

// out[i] = sum over the nparts partials in index order, for i < n; the partial
// layout is [part][co][tap][ci] with co < NOUT, of which the first cout rows are
// the parameters (out: [cout][9][cin] with cin <= CIN, the padded channels dropped)
__global__ void k_wgrad_sum(const float *__restrict__ part, int nparts, int NOUT, int CIN, int cout, int cin,
                            float *__restrict__ out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= cout * 9 * cin) return;
  const int co = i / (9 * cin), r = i % (9 * cin), tap = r / cin, ci = r % cin;
  const size_t src = ((size_t)co * 9 + tap) * CIN + ci, stride = (size_t)NOUT * 9 * CIN;
  float acc = 0.f;
  for (int k = 0; k < nparts; k++) acc += part[k * stride + src];
  out[i] = acc;
}

template <int CIN, int NOUT>
cudaError_t launch_wgrad(const WgradArgs &a, cudaStream_t stream) {
  using SM = WgSmem<CIN, NOUT>;
  auto kern = k_conv_wgrad_tc<CIN, NOUT>;
  cudaError_t ce = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SM::TOTAL);
  if (ce) return ce;
  kern<<<a.nparts, WG_THREADS, SM::TOTAL, stream>>>(a);
  ce = cudaGetLastError();
  if (ce) return ce;
  const int n = a.cout * 9 * a.cin;
  k_wgrad_sum<<<(n + 255) / 256, 256, 0, stream>>>(a.part, a.nparts, NOUT, CIN, a.cout, a.cin, a.dw);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// 64-channel inputs: the shifted input of a tap is a TMA box.
// Tiles are 16 x 8 pixel boxes of one image (M = 128 rows, row m = pixel
// (y0 + m / 16, x0 + m % 16)); a tap's A tile is the box at (x0 + dx, y0 + dy),
// loaded by cp.async.bulk.tensor from a 4D tensor map {C, W, H, B} with 128-byte
// swizzle, the parts outside the grid filled with zeros by the copy engine (the
// "same" padding, negative coordinates included).  One thread issues the loads
// (arrive.expect_tx on the stage's "full" barrier), one thread the MMAs, and
// 8 epilogue warps drain the two TMEM accumulators as in k_conv_tc; boxes that
// overhang the grid compute rows that the epilogue does not store.
// ---------------------------------------------------------------------------
constexpr int TMA_THREADS = 32 * (CONV_EPI_WARPS + 2);  // + producer warp + MMA warp
constexpr int TMA_STAGES = 8;
constexpr int TMA_BX = 16, TMA_BY = 8;

template <int NOUT>
struct TmaSmem {
  static constexpr uint32_t A_BYTES = 128 * 64 * 2;       // one box: 128 pixels x 128 B
  static constexpr uint32_t W_BYTES = NOUT * 9 * 64 * 2;
  static constexpr uint32_t LBO_W = 128 * (NOUT / 8);
  static constexpr uint32_t A0 = 0;                        // stages first (1024-aligned)
  static constexpr uint32_t W0 = TMA_STAGES * A_BYTES;
  static constexpr uint32_t BAR = W0 + W_BYTES;
  static constexpr uint32_t BIAS = BAR + 8 * (2 * TMA_STAGES + 4) + 16;
  static constexpr uint32_t TOTAL = BIAS + 4 * NOUT + 1024;  // + alignment slack
  static constexpr uint32_t TMEM_COLS = 2 * NOUT < 32 ? 32 : 2 * NOUT;
};

template <int NOUT, int EPI>
__global__ void __launch_bounds__(TMA_THREADS, 1) k_conv_tma(const __grid_constant__ CUtensorMap tmap, ConvArgs a) {
  using SM = TmaSmem<NOUT>;
  constexpr int S = TMA_STAGES, KSTEPS = 4;
  extern __shared__ uint8_t smraw[];
  uint8_t *sm = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smraw) + 1023) & ~(uintptr_t)1023);
  uint8_t *As = sm + SM::A0;
  uint8_t *Ws = sm + SM::W0;
  uint64_t *full = reinterpret_cast<uint64_t *>(sm + SM::BAR);
  uint64_t *empty = full + S;
  uint64_t *accf = empty + S;
  uint64_t *acce = accf + 2;
  uint32_t *slot = reinterpret_cast<uint32_t *>(acce + 2);
  volatile int *abort_s = reinterpret_cast<volatile int *>(slot + 1);
  float *bias_s = reinterpret_cast<float *>(sm + SM::BIAS);
  const int tid = threadIdx.x, warp = tid >> 5;
  const int PRODUCER = CONV_EPI_WARPS, MMA = CONV_EPI_WARPS + 1;
  const int TXN = (a.W + TMA_BX - 1) / TMA_BX, TYN = (a.H + TMA_BY - 1) / TMA_BY;
  const int nimg = a.P / (a.H * a.W);
  const int ntiles = nimg * TXN * TYN;
  const int my_tiles = (int)blockIdx.x < ntiles ? (ntiles - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;
  const int total_it = my_tiles * 9;

  for (int c = tid; c < NOUT * 9 * 8; c += TMA_THREADS) {
    const int n = c % NOUT, kc = c / NOUT;
    cp16(su32(Ws + (n / 8) * 128 + kc * SM::LBO_W + (n % 8) * 16), a.wk + (size_t)n * 9 * 64 + kc * 8, true);
  }
  cp_commit();
  for (int c = tid; c < NOUT; c += TMA_THREADS) bias_s[c] = a.bias ? a.bias[c] : 0.f;
  if (warp == MMA) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(slot)), "r"(SM::TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 0) {
    for (int i = 0; i < S; i++) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(su32(full + i)) : "memory");
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(su32(empty + i)) : "memory");
    }
    for (int i = 0; i < 2; i++) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(su32(accf + i)) : "memory");
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(su32(acce + i)), "n"(32 * CONV_EPI_WARPS) : "memory");
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    *abort_s = 0;
  }
  cp_wait<0>();
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *slot;

  if (warp == PRODUCER) {
    if ((tid & 31) == 0) {
      for (int it = 0; it < total_it; it++) {
        const int s = it % S;
        if (it >= S && !mbar_wait(su32(empty + s), ((it / S) - 1) & 1, abort_s)) {
          atomicExch(a.err, 1);
          *abort_s = 1;
          break;
        }
        const int tl = it / 9, tap = it - tl * 9;
        const int t = (int)blockIdx.x + tl * (int)gridDim.x;
        const int tx = t % TXN, ty = (t / TXN) % TYN, b = t / (TXN * TYN);
        const int x = tx * TMA_BX + (tap % 3 - 1) * a.dil * a.sign, y = ty * TMA_BY + (tap / 3 - 1) * a.dil * a.sign;
        asm volatile("{\n .reg .b64 st;\n mbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n}\n" ::"r"(su32(full + s)),
                     "r"(SM::A_BYTES)
                     : "memory");
        asm volatile(
            "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5}], [%6];" ::"r"(
                su32(As + s * SM::A_BYTES)),
            "l"(&tmap), "r"(0), "r"(x), "r"(y), "r"(b), "r"(su32(full + s))
            : "memory");
      }
    }
    __syncwarp();
  } else if (warp == MMA) {
    if ((tid & 31) == 0) {
      const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(NOUT >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
      const uint64_t adesc0 = sdesc_sw128(su32(As)), bdesc0 = sdesc(su32(Ws), SM::LBO_W, 128);
      int last = -1;
      for (int it = 0; it < total_it; it++) {
        const int s = it % S, tl = it / 9, tap = it - tl * 9, buf = tl & 1;
        if (tap == 0 && tl >= 2 && !mbar_wait(su32(acce + buf), ((tl / 2) - 1) & 1, abort_s)) {
          atomicExch(a.err, 1);
          *abort_s = 1;
          break;
        }
        if (!mbar_wait(su32(full + s), (it / S) & 1, abort_s)) {
          atomicExch(a.err, 1);
          *abort_s = 1;
          break;
        }
        tc_fence_after();
        // descriptors by addition: +32 B along K inside the swizzle atom is +2 in the
        // start-address field; the weights advance by 2 * LBO_W per K step
        const uint64_t ad0 = adesc0 + (uint64_t)((s * SM::A_BYTES) >> 4);
        const uint64_t bd0 = bdesc0 + (uint64_t)((tap * KSTEPS * 2 * SM::LBO_W) >> 4);
        const uint32_t d = tmem + (uint32_t)(buf * NOUT);
#pragma unroll
        for (int k = 0; k < KSTEPS; k++) {
          const uint32_t acc = (tap > 0 || k > 0) ? 1u : 0u;
          asm volatile(
              "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
              "l"(ad0 + 2 * k), "l"(bd0 + (uint64_t)((k * 2 * SM::LBO_W) >> 4)), "r"(idesc), "r"(acc)
              : "memory");
        }
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(su32(empty + s))
                     : "memory");
        if (tap == 8)
          asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(su32(accf + buf))
                       : "memory");
        last = it;
      }
      if (*abort_s && last >= 0) mbar_wait(su32(empty + last % S), (last / S) & 1, nullptr);
    }
    __syncwarp();
  } else {
    constexpr int CW = NOUT / 2 < 16 ? 16 : NOUT / 2;
    const int quarter = warp & 3, cb = (warp >> 2) * CW;
    const int m = quarter * 32 + (tid & 31);
    for (int tl = 0; tl < my_tiles; tl++) {
      const int buf = tl & 1;
      if (!mbar_wait(su32(accf + buf), (tl / 2) & 1, abort_s)) {
        atomicExch(a.err, 1);
        *abort_s = 1;
        break;
      }
      tc_fence_after();
      const int t = (int)blockIdx.x + tl * (int)gridDim.x;
      const int tx = t % TXN, ty = (t / TXN) % TYN, b = t / (TXN * TYN);
      const int x = tx * TMA_BX + m % TMA_BX, y = ty * TMA_BY + m / TMA_BX;
      const int p = (x < a.W && y < a.H) ? (b * a.H + y) * a.W + x : a.P;  // a.P: not stored
      if (cb < NOUT)
        conv_epilogue<64, NOUT, EPI, CW>(a, tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(buf * NOUT), p, cb, bias_s);
      tc_fence_before();
      mbar_arrive(su32(acce + buf));
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == MMA) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(SM::TMEM_COLS) : "memory");
  }
}

typedef CUresult (*TensorMapEncodeTiled)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                         const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                         CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

TensorMapEncodeTiled tensor_map_encoder() {
  static TensorMapEncodeTiled fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    cudaDriverEntryPointQueryResult q;
    void *p = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<TensorMapEncodeTiled>(p);
  });
  return fn;
}

template <int NOUT, int EPI>
cudaError_t launch_tma(const ConvArgs &a, cudaStream_t stream) {
  using SM = TmaSmem<NOUT>;
  TensorMapEncodeTiled enc = tensor_map_encoder();
  if (!enc) return cudaErrorNotSupported;
  const int HW = a.H * a.W;
  if (a.P % HW) return cudaErrorInvalidValue;
  CUtensorMap tm;
  const cuuint64_t dims[4] = {64, (cuuint64_t)a.W, (cuuint64_t)a.H, (cuuint64_t)(a.P / HW)};
  const cuuint64_t strides[3] = {64 * 2, (cuuint64_t)a.W * 64 * 2, (cuuint64_t)HW * 64 * 2};
  const cuuint32_t box[4] = {64, TMA_BX, TMA_BY, 1}, es[4] = {1, 1, 1, 1};
  if (enc(&tm, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, const_cast<bf16 *>(a.in), dims, strides, box, es,
          CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
          CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
    return cudaErrorInvalidValue;
  auto kern = k_conv_tma<NOUT, EPI>;
  cudaError_t ce = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SM::TOTAL);
  if (ce) return ce;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int ntiles = (a.P / HW) * ((a.W + TMA_BX - 1) / TMA_BX) * ((a.H + TMA_BY - 1) / TMA_BY);
  const int grid = ntiles < sms ? ntiles : sms;
  if (grid < 1) return cudaSuccess;
  kern<<<grid, TMA_THREADS, SM::TOTAL, stream>>>(tm, a);
  return cudaGetLastError();
}

template <int CIN, int NOUT, int EPI>
cudaError_t launch_one(const ConvArgs &a, cudaStream_t stream) {
  using SM = ConvSmem<CIN, NOUT>;
  auto kern = k_conv_tc<CIN, NOUT, EPI>;
  cudaError_t ce = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SM::TOTAL);
  if (ce) return ce;
  int dev = 0, sms = 0, per_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  ce = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, CONV_THREADS, SM::TOTAL);
  if (ce) return ce;
  // tensor memory: at most 512 columns per SM are ever requested
  const int tmem_cap = 512 / (int)SM::TMEM_COLS;
  if (per_sm > tmem_cap) per_sm = tmem_cap;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  const int ntiles = (a.P + 127) / 128;
  int grid = sms * per_sm;
  if (grid > ntiles) grid = ntiles;
  if (grid < 1) return cudaSuccess;
  kern<<<grid, CONV_THREADS, SM::TOTAL, stream>>>(a);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_conv_tc(int cin, int nout, int epi, const ConvArgs &a, cudaStream_t stream) {
  if (a.P <= 0) return cudaSuccess;
#define CONV_CASE(CI, NO, EP) \
  if (cin == CI && nout == NO && epi == EP) return launch_one<CI, NO, EP>(a, stream);
  CONV_CASE(16, 16, CONV_EPI_FWD_SILU)
  CONV_CASE(16, 32, CONV_EPI_FWD_SILU)
  CONV_CASE(32, 32, CONV_EPI_FWD_SILU)
  CONV_CASE(16, 64, CONV_EPI_FWD_SILU)
  // 64-channel inputs: TMA-fed kernel
  if (cin == 64 && nout == 64 && epi == CONV_EPI_FWD_SILU) return launch_tma<64, CONV_EPI_FWD_SILU>(a, stream);
  if (cin == 64 && nout == 16 && epi == CONV_EPI_LAST) return launch_tma<16, CONV_EPI_LAST>(a, stream);
  if (cin == 64 && nout == 64 && epi == CONV_EPI_BWD_SILU) return launch_tma<64, CONV_EPI_BWD_SILU>(a, stream);
  CONV_CASE(16, 16, CONV_EPI_LAST)
  CONV_CASE(32, 16, CONV_EPI_LAST)
  CONV_CASE(16, 16, CONV_EPI_BWD_SILU)
  CONV_CASE(16, 32, CONV_EPI_BWD_SILU)
  CONV_CASE(32, 32, CONV_EPI_BWD_SILU)
  CONV_CASE(16, 64, CONV_EPI_BWD_SILU)
#undef CONV_CASE
  return cudaErrorInvalidValue;
}

cudaError_t launch_conv_wgrad_tc(int cinp, int noutp, const WgradArgs &a, cudaStream_t stream) {
  if (a.P <= 0) return cudaSuccess;
  if (a.nparts < 1 || a.nparts > 1024) return cudaErrorInvalidValue;
#define WG_CASE(CI, NO) \
  if (cinp == CI && noutp == NO) return launch_wgrad<CI, NO>(a, stream);
  WG_CASE(16, 16)
  WG_CASE(16, 32)
  WG_CASE(16, 64)
  WG_CASE(32, 32)
  WG_CASE(32, 16)
  WG_CASE(64, 64)
  WG_CASE(64, 16)
#undef WG_CASE
  return cudaErrorInvalidValue;
}
