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
// One CTA of 128 threads per tile stream (persistent over tiles):
//   - the weights of the layer sit in shared memory for the whole kernel;
//   - every thread gathers its own pixel row of the shifted input for each tap
//     with 16-byte cp.async copies (zero-filled outside the grid) into a
//     4-stage ring of A tiles, three taps ahead of the tensor core;
//   - one thread issues the MMAs of a tap (CIN/16 instructions of K = 16) and
//     commits them to the stage's mbarrier, which frees the stage for reuse;
//   - after the ninth tap the accumulator (128 lanes x NOUT columns of TMEM) is
//     read back with tcgen05.ld, thread t owning pixel row t, and the epilogue
//     (bias + SiLU, or the SiLU derivative of the layer below) is fused.
// Operand tiles use the canonical K-major layout without swizzling: 8-row x
// 16-byte core matrices, 128 bytes apart along M/N (SBO) and one column of
// core matrices per 8 K values (LBO).  Every mbarrier wait is bounded; on
// timeout the kernel raises an error flag, drains its copies, frees its tensor
// memory and returns.
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

__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t parity) {
  for (int i = 0; i < (1 << 24); i++) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(mbar), "r"(parity)
        : "memory");
    if (ok) return true;
  }
  return false;
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

constexpr int CONV_THREADS = 128;
constexpr int CONV_STAGES = 4;

template <int CIN, int NOUT>
struct ConvSmem {
  static constexpr uint32_t SBO = 128;                 // next 8 rows (M or N)
  static constexpr uint32_t LBO_A = 128 * 16;          // next 8 K values of an A tile (16 row groups)
  static constexpr uint32_t LBO_W = 128 * (NOUT / 8);  // next 8 K values of the weight tile
  static constexpr uint32_t A_BYTES = 128 * CIN * 2;
  static constexpr uint32_t W_BYTES = NOUT * 9 * CIN * 2;
  static constexpr uint32_t BAR = W_BYTES + CONV_STAGES * A_BYTES;
  static constexpr uint32_t TOTAL = BAR + 8 * (CONV_STAGES + 1) + 16;
  static constexpr uint32_t TMEM_COLS = NOUT <= 32 ? 32 : (NOUT <= 64 ? 64 : 128);
};

template <int CIN, int NOUT, int EPI>
__global__ void __launch_bounds__(CONV_THREADS, 1) k_conv_tc(ConvArgs a) {
  using SM = ConvSmem<CIN, NOUT>;
  constexpr int KCH = CIN / 8, KSTEPS = CIN / 16, S = CONV_STAGES, DIST = S - 1;
  static_assert(CIN % 16 == 0 && NOUT % 16 == 0 && NOUT <= 128, "tile shape");
  extern __shared__ __align__(128) uint8_t sm[];
  uint8_t *Ws = sm;
  uint8_t *As = sm + SM::W_BYTES;
  uint64_t *mbar = reinterpret_cast<uint64_t *>(sm + SM::BAR);  // [S] stages, [S] accumulator
  uint32_t *slot = reinterpret_cast<uint32_t *>(mbar + S + 1);
  int *abort_s = reinterpret_cast<int *>(slot + 1);
  const int tid = threadIdx.x, warp = tid >> 5;
  const int HW = a.H * a.W;
  const int ntiles = (a.P + 127) / 128;
  const int my_tiles = (int)blockIdx.x < ntiles ? (ntiles - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;
  const int total_it = my_tiles * 9;

  // the layer's weights, resident for the whole kernel (joins the first copy group)
  for (int c = tid; c < NOUT * 9 * KCH; c += CONV_THREADS) {
    const int n = c % NOUT, kc = c / NOUT;
    cp16(su32(Ws + (n / 8) * SM::SBO + kc * SM::LBO_W + (n % 8) * 16), a.wk + (size_t)n * 9 * CIN + kc * 8, true);
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(slot)), "r"(SM::TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 0) {
    for (int i = 0; i <= S; i++) asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(su32(mbar + i)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    *abort_s = 0;
  }

  // gather of iteration it = (local tile, tap): thread t copies pixel row t
  auto load_it = [&](int it) {
    if (it < total_it) {
      const int tl = it / 9, tap = it - tl * 9;
      const int p = ((int)blockIdx.x + tl * (int)gridDim.x) * 128 + tid;
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
      const uint32_t dst = su32(As + (it % S) * SM::A_BYTES + (tid / 8) * SM::SBO + (tid % 8) * 16);
#pragma unroll
      for (int kc = 0; kc < KCH; kc++) cp16(dst + kc * SM::LBO_A, src + kc * 8, valid);
    }
    cp_commit();
  };
  for (int i = 0; i < DIST; i++) load_it(i);

  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *slot;
  // instruction descriptor: FP32 accumulator, BF16 A and B, both K-major, N, M = 128
  const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(NOUT >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);

  int issued = -1;  // last iteration whose MMAs were issued (uniform)
  bool failed = false;
  for (int it = 0; it < total_it; it++) {
    const int s = it % S, tl = it / 9, tap = it - tl * 9;
    cp_wait<DIST - 1>();
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    tc_fence_before();
    __syncthreads();
    if (*abort_s) { failed = true; break; }
    if (tid == 0) {
      tc_fence_after();
      const uint32_t a0 = su32(As + s * SM::A_BYTES), w0 = su32(Ws);
#pragma unroll
      for (int j = 0; j < KSTEPS; j++) {
        const uint64_t ad = sdesc(a0 + 2 * j * SM::LBO_A, SM::LBO_A, SM::SBO);
        const uint64_t bd = sdesc(w0 + 2 * (tap * KSTEPS + j) * SM::LBO_W, SM::LBO_W, SM::SBO);
        const uint32_t acc = (tap > 0 || j > 0) ? 1u : 0u;
        asm volatile(
            "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
            "l"(ad), "l"(bd), "r"(idesc), "r"(acc)
            : "memory");
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(su32(mbar + s)) : "memory");
      if (tap == 8)
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(su32(mbar + S)) : "memory");
    }
    issued = it;
    // the stage of iteration it-1 receives iteration it+DIST once its MMAs are done
    if (it >= 1 && !mbar_wait(su32(mbar + (it - 1) % S), ((it - 1) / S) & 1)) {
      atomicExch(a.err, 1);
      *abort_s = 1;
    }
    load_it(it + DIST);
    if (tap == 8) {
      if (!mbar_wait(su32(mbar + S), tl & 1)) {
        atomicExch(a.err, 1);
        *abort_s = 1;
        continue;
      }
      tc_fence_after();
      const int p = ((int)blockIdx.x + tl * (int)gridDim.x) * 128 + tid;
      const uint32_t trow = tmem + ((uint32_t)(warp * 32) << 16);
      if (EPI == CONV_EPI_LAST) {
        float v[16];
        tmem_ld16(trow, v);
        if (p < a.P) a.z[p] = v[0] + (a.bias ? a.bias[0] : 0.f);
      } else {
#pragma unroll
        for (int c0 = 0; c0 < NOUT; c0 += 16) {
          float v[16];
          tmem_ld16(trow + c0, v);
          if (p >= a.P) continue;
          if (EPI == CONV_EPI_FWD_SILU) {
#pragma unroll
            for (int j = 0; j < 16; j++) v[j] += a.bias ? a.bias[c0 + j] : 0.f;
            if (a.z) {
              float4 *z4 = reinterpret_cast<float4 *>(a.z + (size_t)p * NOUT + c0);
#pragma unroll
              for (int q = 0; q < 4; q++) z4[q] = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
            }
            uint4 o[2];
            uint32_t *ow = reinterpret_cast<uint32_t *>(o);
#pragma unroll
            for (int j = 0; j < 8; j++) ow[j] = pack2(v[2 * j] * sigm(v[2 * j]), v[2 * j + 1] * sigm(v[2 * j + 1]));
            uint4 *dst = reinterpret_cast<uint4 *>(a.act + (size_t)p * NOUT + c0);
            dst[0] = o[0];
            dst[1] = o[1];
          } else {  // CONV_EPI_BWD_SILU: d = v * SiLU'(z_below)
            const float4 *zp = reinterpret_cast<const float4 *>(a.zprev + (size_t)p * NOUT + c0);
            float d[16];
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
    }
  }
  // drain: outstanding copies, then (after a failure) the MMAs already issued
  cp_wait<0>();
  if (failed && issued >= 0) mbar_wait(su32(mbar + issued % S), (issued / S) & 1);
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
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
