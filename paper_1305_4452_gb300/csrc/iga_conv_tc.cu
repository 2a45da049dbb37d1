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
// One persistent CTA per SM, warp-specialised (288 threads):
//   - warps 4-7 (producers): thread j gathers pixel row j of the shifted, dilated
//     input for each (tile, tap) with 16-byte cp.async copies (zero-filled outside
//     the grid) into an 8-stage ring; once its copies of a stage have landed it
//     fences them into the async proxy and arrives on the stage's "full" barrier;
//     it refills a stage after the stage's "empty" barrier reports the MMAs that
//     read it complete;
//   - warp 8 (MMA): allocates tensor memory; one thread waits for "full", issues
//     the tap's CIN/16 tcgen05.mma instructions (K = 16, FP32 accumulator in
//     TMEM) and commits them to "empty"; after the ninth tap it commits the
//     accumulator to "acc full";
//   - warps 0-3 (epilogue): thread t reads accumulator row t (pixel t of the tile)
//     with tcgen05.ld, applies the fused epilogue (bias + SiLU, or the SiLU
//     derivative of the layer below), stores, and arrives on "acc empty".
//   Two accumulators in TMEM (2 x NOUT columns) let the epilogue of one tile
//   overlap the MMAs of the next; the layer's weights stay in shared memory.
// Operand tiles use the canonical K-major layout without swizzling: 8-row x
// 16-byte core matrices, 128 bytes apart along M/N (SBO) and one column of
// core matrices per 8 K values (LBO).  Every mbarrier wait is bounded in time
// (globaltimer); on timeout the kernel raises an error flag, every role stops,
// the MMA thread waits (bounded) for its last commit, and the tensor memory is
// freed before the kernel returns.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "iga_internal.h"
#include "iga_conv_tc.h"

namespace {

typedef __nv_bfloat16 bf16;

__device__ __forceinline__ uint32_t su32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// shared-memory matrix descriptor: start, leading (K) and stride (M/N) byte
// offsets, descriptor version 1, no swizzle
__device__ __forceinline__ uint64_t sdesc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((addr & 0x3FFFF) >> 4) | ((uint64_t)((lbo >> 4) & 0x3FFF) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFF) << 32) | (1ull << 46);
}

__device__ __forceinline__ uint64_t gtimer() {
  uint64_t t;
  asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ bool mbar_try(uint32_t mbar, uint32_t parity) {
  uint32_t ok;
  asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
               : "=r"(ok)
               : "r"(mbar), "r"(parity)
               : "memory");
  return ok != 0;
}

// wait for the phase with the given parity to complete; false after ~2 s, or
// at once when another role has given up (*abort set)
__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t parity, volatile int *abort) {
  if (mbar_try(mbar, parity)) return true;
  const uint64_t t0 = gtimer();
  for (uint32_t i = 1;; i++) {
    if (mbar_try(mbar, parity)) return true;
    if ((i & 63) == 0 && ((abort && *abort) || gtimer() - t0 > 2000000000ull)) return false;
  }
}

__device__ __forceinline__ void mbar_arrive(uint32_t mbar) {
  asm volatile("{\n .reg .b64 st;\n mbarrier.arrive.shared::cta.b64 st, [%0];\n}\n" ::"r"(mbar) : "memory");
}

__device__ __forceinline__ void cp16(uint32_t dst, const void *src, bool valid) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(src), "r"(valid ? 16 : 0) : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float *v) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int j = 0; j < 16; j++) v[j] = __uint_as_float(r[j]);
}

__device__ __forceinline__ float sigm(float z) { return 1.f / (1.f + expf(-z)); }

__device__ __forceinline__ uint32_t pack2(float a, float b) {
  __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
  return *reinterpret_cast<uint32_t *>(&h);
}

constexpr int CONV_THREADS = 288;  // 4 epilogue warps, 4 producer warps, 1 MMA warp
constexpr int CONV_STAGES = 8;
constexpr int CONV_LAG = 2;        // copy groups a producer keeps in flight beyond the one it signals

template <int CIN, int NOUT>
struct ConvSmem {
  static constexpr uint32_t SBO = 128;                 // next 8 rows (M or N)
  static constexpr uint32_t LBO_A = 128 * 16;          // next 8 K values of an A tile (16 row groups)
  static constexpr uint32_t LBO_W = 128 * (NOUT / 8);  // next 8 K values of the weight tile
  static constexpr uint32_t A_BYTES = 128 * CIN * 2;
  static constexpr uint32_t W_BYTES = NOUT * 9 * CIN * 2;
  static constexpr uint32_t BAR = W_BYTES + CONV_STAGES * A_BYTES;
  // barriers: full[S], empty[S], acc_full[2], acc_empty[2]; then the TMEM slot and the abort flag
  static constexpr uint32_t TOTAL = BAR + 8 * (2 * CONV_STAGES + 4) + 16;
  static constexpr uint32_t TMEM_COLS = 2 * NOUT < 32 ? 32 : 2 * NOUT;  // two accumulators
};

template <int CIN, int NOUT, int EPI>
__device__ __forceinline__ void conv_epilogue(const ConvArgs &a, uint32_t taddr, int p) {
  if constexpr (EPI == CONV_EPI_LAST) {
    float v[16];
    tmem_ld16(taddr, v);
    if (p < a.P) a.z[p] = v[0] + (a.bias ? a.bias[0] : 0.f);
  } else {
#pragma unroll
  for (int c0 = 0; c0 < NOUT; c0 += 16) {
    float v[16];
    tmem_ld16(taddr + c0, v);
    if (p >= a.P) continue;
    float d[16];
    if constexpr (EPI == CONV_EPI_FWD_SILU) {
#pragma unroll
      for (int j = 0; j < 16; j++) d[j] = v[j] + (a.bias ? a.bias[c0 + j] : 0.f);
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
    for (int i = 0; i < 2; i++) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(su32(accf + i)) : "memory");
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 128;" ::"r"(su32(acce + i)) : "memory");
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

  if (warp >= 4 && warp < 8) {
    // ---------------- producers ----------------
    const int j = tid - 128;  // pixel row within the tile
    const int HW = a.H * a.W;
    int it = 0;
    for (; it < total_it; it++) {
      const int s = it % S;
      if (it >= S && !mbar_wait(su32(empty + s), ((it / S) - 1) & 1, abort_s)) {
        atomicExch(a.err, 1);
        *abort_s = 1;
        break;
      }
      const int tl = it / 9, tap = it - tl * 9;
      const int p = ((int)blockIdx.x + tl * (int)gridDim.x) * 128 + j;
      const int dy = (tap / 3 - 1) * a.dil * a.sign, dx = (tap % 3 - 1) * a.dil * a.sign;
      bool valid = false;
      const bf16 *src = a.in;
      if (p < a.P) {
        const int b = p / HW, r = p - b * HW, y = r / a.W, x = r - y * a.W;
        const int sy = y + dy, sx = x + dx;
        if (sy >= 0 && sy < a.H && sx >= 0 && sx < a.W) {
          valid = true;
          src = a.in + ((size_t)b * HW + (size_t)sy * a.W + sx) * CIN;
        }
      }
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
  } else if (warp == 8) {
    // ---------------- MMA issuer ----------------
    if ((tid & 31) == 0) {
      const uint32_t idesc =
          (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(NOUT >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
      const uint32_t w0 = su32(Ws);
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
        const uint32_t a0 = su32(As + s * SM::A_BYTES), d = tmem + (uint32_t)(buf * NOUT);
#pragma unroll
        for (int k = 0; k < KSTEPS; k++) {
          const uint64_t ad = sdesc(a0 + 2 * k * SM::LBO_A, SM::LBO_A, SM::SBO);
          const uint64_t bd = sdesc(w0 + 2 * (tap * KSTEPS + k) * SM::LBO_W, SM::LBO_W, SM::SBO);
          const uint32_t acc = (tap > 0 || k > 0) ? 1u : 0u;
          asm volatile(
              "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
              "l"(ad), "l"(bd), "r"(idesc), "r"(acc)
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
    // ---------------- epilogue (warps 0-3: TMEM lanes 0-127) ----------------
    for (int tl = 0; tl < my_tiles; tl++) {
      const int buf = tl & 1;
      if (!mbar_wait(su32(accf + buf), (tl / 2) & 1, abort_s)) {
        atomicExch(a.err, 1);
        *abort_s = 1;
        break;
      }
      tc_fence_after();
      const int p = ((int)blockIdx.x + tl * (int)gridDim.x) * 128 + tid;
      conv_epilogue<CIN, NOUT, EPI>(a, tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(buf * NOUT), p);
      tc_fence_before();
      mbar_arrive(su32(acce + buf));
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 8) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(SM::TMEM_COLS) : "memory");
  }
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
  CONV_CASE(64, 64, CONV_EPI_FWD_SILU)
  CONV_CASE(16, 16, CONV_EPI_LAST)
  CONV_CASE(32, 16, CONV_EPI_LAST)
  CONV_CASE(64, 16, CONV_EPI_LAST)
  CONV_CASE(16, 16, CONV_EPI_BWD_SILU)
  CONV_CASE(16, 32, CONV_EPI_BWD_SILU)
  CONV_CASE(32, 32, CONV_EPI_BWD_SILU)
  CONV_CASE(16, 64, CONV_EPI_BWD_SILU)
  CONV_CASE(64, 64, CONV_EPI_BWD_SILU)
#undef CONV_CASE
  return cudaErrorInvalidValue;
}
