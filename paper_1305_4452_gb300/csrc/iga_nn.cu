// Convolutional neural operator for Newton initial guesses (hand-written training
// and inference kernels).  Not in the paper: it maps (lambda, log-kappa field) on
// the control grid to an initial U for the kappa-weighted Bratu problem.
//
// Network: L layers of 3x3 convolutions with per-layer dilation and "same" zero
// padding on an H x W grid (NHWC activations), SiLU between layers, a linear last
// layer with one output channel, multiplied by a mask (zero on Dirichlet rows).
// The forward convolutions, the input-gradient (transposed) convolutions and the
// weight gradients run as implicit GEMMs on the tcgen05 tensor cores, with fused
// bias + SiLU and SiLU' epilogues (iga_conv_tc.cu).  Operands are BF16 with FP32
// accumulation.
// Master weights, Adam moments, gradients and the loss are FP32; activations are
// stored in BF16 for the GEMMs and FP32 where the backward pass needs them.  Every
// reduction (split-K weight gradients, bias gradients, loss) has a fixed order.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <string>
#include <utility>
#include <vector>

#include "iga_internal.h"
#include "iga_conv_tc.h"

typedef __nv_bfloat16 bf16;

namespace {

// out[i] = sum_z part[z][i] in z order
__global__ void k_sum_splits(const float *__restrict__ part, int nsplit, int64_t n, float *__restrict__ out, int accumulate) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  float s = 0.f;
  for (int z = 0; z < nsplit; z++) s += part[(int64_t)z * n + i];
  out[i] = accumulate ? out[i] + s : s;
}

// features x[p][c] (FP32, c < C) -> xp[p][16] BF16 zero-padded for the tensor-core
// convolution, and (training) x16[p][c] unpadded for the weight-gradient im2col
__global__ void k_pad_input(const float *__restrict__ x, int C, int64_t P, bf16 *__restrict__ xp, bf16 *__restrict__ x16) {
  int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= P * 16) return;
  const int64_t p = t / 16;
  const int c = (int)(t % 16);
  const float v = c < C ? x[p * C + c] : 0.f;
  xp[t] = __float2bfloat16(v);
  if (x16 && c < C) x16[p * C + c] = __float2bfloat16(v);
}

// per layer, from the FP32 master W[co][tap][ci]: wk[n][tap][c] = W[n][tap][c] padded to
// (NP outputs, CP inputs), and wt[ci][tap][co] = W[co][tap][ci] padded to CP2 = NP
// inputs (the transposed convolution's operand)
__global__ void k_prep_w(const float *__restrict__ w, int cin, int cout, int CP, int NP, bf16 *__restrict__ wk,
                         bf16 *__restrict__ wt) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t < NP * 9 * CP) {
    const int n = t / (9 * CP), r = t % (9 * CP), tap = r / CP, c = r % CP;
    wk[t] = __float2bfloat16((n < cout && c < cin) ? w[(n * 9 + tap) * cin + c] : 0.f);
  }
  if (wt && t < cin * 9 * NP) {
    const int ci = t / (9 * NP), r = t % (9 * NP), tap = r / NP, co = r % NP;
    wt[t] = __float2bfloat16(co < cout ? w[(co * 9 + tap) * cin + ci] : 0.f);
  }
}

// last layer's output gradient dz[p] (one channel) -> BF16 [p][1] for the weight
// gradient and [p][16] zero-padded for the transposed convolution
__global__ void k_pad_grad(const float *__restrict__ dz, int64_t P, bf16 *__restrict__ d1, bf16 *__restrict__ d16) {
  int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= P * 16) return;
  const int64_t p = t / 16;
  const int c = (int)(t % 16);
  const bf16 v = __float2bfloat16(dz[p]);
  d16[t] = c == 0 ? v : __float2bfloat16(0.f);
  if (c == 0) d1[p] = v;
}

// y[b][p] = mask[p] * z[b][p]  (last layer, one channel)
__global__ void k_output(const float *__restrict__ z, const float *__restrict__ mask, int64_t HW, int64_t n, float *__restrict__ y) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) y[i] = (mask ? mask[i % HW] : 1.f) * z[i];
}

// Loss = [ sum mask (y-t)^2 + beta * sum over grid edges (difference of (y-t))^2 ] / sum mask:
// the mean-squared error plus a discrete H1 seminorm of the error (beta >= 0), which
// weighs the oscillatory error components that dominate the initial Newton residual.
// Per-block partial sums of the numerator and of the mask count.
__global__ void __launch_bounds__(256) k_loss_partial(const float *__restrict__ y, const float *__restrict__ tgt,
                                                      const float *__restrict__ mask, int64_t HW, int64_t n, int Wd,
                                                      int Hh, float beta, float *__restrict__ part) {
  __shared__ float sh[2][8];
  int64_t per = (n + gridDim.x - 1) / gridDim.x;
  int64_t a = blockIdx.x * per, e = min(n, a + per);
  float s = 0.f, m = 0.f;
  for (int64_t i = a + threadIdx.x; i < e; i += blockDim.x) {
    float mk = mask ? mask[i % HW] : 1.f;
    float d = y[i] - tgt[i];
    s += mk * d * d;
    m += mk;
    if (beta != 0.f) {
      const int64_t pix = i % HW;
      const int xx = (int)(pix % Wd), yy = (int)(pix / Wd);
      if (xx + 1 < Wd) { float dd = (y[i + 1] - tgt[i + 1]) - d; s += beta * dd * dd; }
      if (yy + 1 < Hh) { float dd = (y[i + Wd] - tgt[i + Wd]) - d; s += beta * dd * dd; }
    }
  }
  for (int o = 16; o > 0; o >>= 1) {
    s += __shfl_down_sync(0xffffffffu, s, o);
    m += __shfl_down_sync(0xffffffffu, m, o);
  }
  if ((threadIdx.x & 31) == 0) {
    sh[0][threadIdx.x >> 5] = s;
    sh[1][threadIdx.x >> 5] = m;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    float ts = 0.f, tm = 0.f;
    for (int w = 0; w < 8; w++) { ts += sh[0][w]; tm += sh[1][w]; }
    part[2 * blockIdx.x] = ts;
    part[2 * blockIdx.x + 1] = tm;
  }
}

__global__ void k_loss_final(const float *__restrict__ part, int nb, float *__restrict__ out) {
  float s = 0.f, m = 0.f;
  for (int k = 0; k < nb; k++) { s += part[2 * k]; m += part[2 * k + 1]; }
  out[0] = s / fmaxf(m, 1.f);
  out[1] = m;
}

// dL/dz with y = mask * z: mask * [2 mask e + 2 beta (sum over neighbours (e - e_nb))] / count
__global__ void k_loss_grad(const float *__restrict__ y, const float *__restrict__ tgt, const float *__restrict__ mask,
                            int64_t HW, int64_t n, int Wd, int Hh, float beta, const float *__restrict__ lossv,
                            float *__restrict__ dz) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  float mk = mask ? mask[i % HW] : 1.f;
  float e = y[i] - tgt[i];
  float g = 2.f * mk * e;
  if (beta != 0.f) {
    const int64_t pix = i % HW;
    const int xx = (int)(pix % Wd), yy = (int)(pix / Wd);
    float lap = 0.f;
    if (xx + 1 < Wd) lap += e - (y[i + 1] - tgt[i + 1]);
    if (xx > 0) lap += e - (y[i - 1] - tgt[i - 1]);
    if (yy + 1 < Hh) lap += e - (y[i + Wd] - tgt[i + Wd]);
    if (yy > 0) lap += e - (y[i - Wd] - tgt[i - Wd]);
    g += 2.f * beta * lap;
  }
  dz[i] = mk * g / fmaxf(lossv[1], 1.f);
}

// db[c] = sum_p dz[p][c]: per-chunk partials then an ordered sum
__global__ void k_colsum_partial(const float *__restrict__ dz, int64_t P, int C, int64_t chunk, float *__restrict__ part) {
  int c = threadIdx.x;
  if (c >= C) return;
  int64_t a = blockIdx.x * chunk, e = min(P, a + chunk);
  float s = 0.f;
  for (int64_t p = a; p < e; p++) s += dz[p * C + c];
  part[(int64_t)blockIdx.x * C + c] = s;
}

__global__ void k_adam(float *__restrict__ w, const float *__restrict__ gr, float *__restrict__ m, float *__restrict__ v,
                       int64_t n, float lr, float b1, float b2, float eps, float c1, float c2) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  float gi = gr[i];
  float mi = b1 * m[i] + (1.f - b1) * gi;
  float vi = b2 * v[i] + (1.f - b2) * gi * gi;
  m[i] = mi;
  v[i] = vi;
  float wi = w[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
  w[i] = wi;
}

// splitmix64-based uniform init in [-a, a]
__global__ void k_init_uniform(float *__restrict__ w, int64_t n, uint64_t seed, float a) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  uint64_t z = seed + (uint64_t)(i + 1) * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  z = z ^ (z >> 31);
  double u = (double)(z >> 11) * (1.0 / 9007199254740992.0);
  w[i] = (float)((2.0 * u - 1.0) * a);
}

inline unsigned g1(int64_t n) { return (unsigned)((n + 255) / 256); }

}  // namespace

struct NNLayer {
  int cin, cout, dil;
  int64_t woff, boff;  // offsets in the flat parameter vector
  int cp, np;          // tensor-core operand widths: inputs and outputs padded to >= 16
  bf16 *wk = nullptr;  // [np][9][cp] forward operand
  bf16 *wt = nullptr;  // [cin][9][np] transposed-convolution operand (layers > 0)
};

struct iga_nn_s {
  int H = 0, W = 0, cin = 0, hidden = 0, L = 0, maxB = 0;
  cudaStream_t stream = nullptr;
  std::vector<NNLayer> layers;
  int64_t nparams = 0;
  float *w = nullptr, *g = nullptr, *m = nullptr, *v = nullptr;  // FP32 master, grad, Adam
  bf16 *wops = nullptr;       // BF16 tensor-core operands of all layers (NNLayer::wk, wt)
  std::vector<bf16 *> X;      // inputs of each layer, BF16 [P][Cin]
  bf16 *X0p = nullptr;        // network input padded to 16 channels
  std::vector<float *> Z;     // pre-activations FP32 [P][Cout]
  float *wpart = nullptr;     // per-CTA partial weight gradients [nparts][64][9][64]
  int nparts = 0;
  float *dZ = nullptr, *dZ2 = nullptr;  // output gradients FP32 [P][Cmax] (ping-pong)
  bf16 *dZb = nullptr, *dZb2 = nullptr; // their BF16 copies
  bf16 *dZb16 = nullptr;      // last layer's gradient padded to 16 channels
  int *tc_err = nullptr;      // tensor-core wait timeout flag (device)
  int *tc_err_h = nullptr;    // pinned mirror
  float *part = nullptr;      // split-K / column-sum / loss partials
  float *y = nullptr, *lossv = nullptr, *lossh = nullptr;
  int64_t part_n = 0;
  int adam_t = 0;
  float h1 = 0.f;  // weight of the discrete H1 term of the loss
  std::string err;
};

static void nn_release(iga_nn_s *n) {
  void *ps[] = {n->w, n->g, n->m, n->v, n->wops, n->X0p, n->wpart, n->dZ, n->dZ2, n->dZb, n->dZb2, n->dZb16,
                n->part, n->y, n->lossv, n->tc_err};
  for (void *p : ps)
    if (p) cudaFree(p);
  for (auto p : n->X) if (p) cudaFree(p);
  for (auto p : n->Z) if (p) cudaFree(p);
  if (n->lossh) cudaFreeHost(n->lossh);
  if (n->tc_err_h) cudaFreeHost(n->tc_err_h);
}

#define NCK(call)                                                              \
  do {                                                                         \
    cudaError_t ce_ = (call);                                                  \
    if (ce_ != cudaSuccess) {                                                  \
      n->err = iga_format("%s: %s", #call, cudaGetErrorString(ce_));           \
      return ce_ == cudaErrorMemoryAllocation ? IGA_ENOMEM : IGA_ECUDA;        \
    }                                                                          \
  } while (0)

static thread_local std::string g_nn_err;

extern "C" iga_status iga_nn_create(int height, int width, int in_channels, int hidden, int layers, const int *dilations,
                                    int max_batch, uint64_t seed, void *stream, iga_nn_t *out) {
  if (!out) return IGA_EINVAL;
  *out = nullptr;
  if (height < 1 || width < 1 || in_channels < 1 || in_channels > 16 || (hidden != 16 && hidden != 32 && hidden != 64) ||
      layers < 2 || layers > 16 || max_batch < 1 || !dilations || (int64_t)max_batch * height * width > (1 << 28)) {
    g_nn_err = "bad network shape (in_channels 1..16, hidden 16, 32 or 64, 2..16 layers, at most 2^28 pixels)";
    return IGA_EINVAL;
  }
  iga_nn_s *n = new iga_nn_s();
  n->H = height; n->W = width; n->cin = in_channels; n->hidden = hidden; n->L = layers; n->maxB = max_batch;
  n->stream = (cudaStream_t)stream;
  int64_t off = 0;
  int cmax = std::max(in_channels, hidden);
  for (int l = 0; l < layers; l++) {
    NNLayer ly;
    ly.cin = (l == 0) ? in_channels : hidden;
    ly.cout = (l == layers - 1) ? 1 : hidden;
    ly.dil = dilations[l];
    if (ly.dil < 1 || ly.dil > height) {
      g_nn_err = "dilations must be in [1, height]";
      delete n;
      return IGA_EINVAL;
    }
    ly.woff = off;
    off += (int64_t)ly.cout * 9 * ly.cin;
    ly.boff = off;
    off += ly.cout;
    ly.cp = (l == 0) ? 16 : hidden;
    ly.np = (l == layers - 1) ? 16 : hidden;
    n->layers.push_back(ly);
  }
  n->nparams = off;
  auto fail = [&](iga_status st) {
    g_nn_err = n->err;
    nn_release(n);
    delete n;
    return st;
  };
#define NCK2(call)                                                        \
  do {                                                                    \
    cudaError_t ce_ = (call);                                             \
    if (ce_ != cudaSuccess) {                                             \
      n->err = iga_format("%s: %s", #call, cudaGetErrorString(ce_));      \
      return fail(ce_ == cudaErrorMemoryAllocation ? IGA_ENOMEM : IGA_ECUDA); \
    }                                                                     \
  } while (0)
  const int64_t P = (int64_t)max_batch * height * width;
  NCK2(cudaMalloc((void **)&n->w, off * sizeof(float)));
  NCK2(cudaMalloc((void **)&n->g, off * sizeof(float)));
  NCK2(cudaMalloc((void **)&n->m, off * sizeof(float)));
  NCK2(cudaMalloc((void **)&n->v, off * sizeof(float)));
  int64_t wops = 0;
  for (auto &ly : n->layers) wops += (int64_t)9 * (ly.np * ly.cp + ly.cin * ly.np);
  NCK2(cudaMalloc((void **)&n->wops, wops * sizeof(bf16)));
  {
    bf16 *q = n->wops;
    for (int l = 0; l < layers; l++) {
      NNLayer &ly = n->layers[l];
      ly.wk = q;
      q += (int64_t)9 * ly.np * ly.cp;
      ly.wt = l > 0 ? q : nullptr;
      q += (int64_t)9 * ly.cin * ly.np;
    }
  }
  NCK2(cudaMalloc((void **)&n->X0p, P * 16 * sizeof(bf16)));
  NCK2(cudaMalloc((void **)&n->tc_err, sizeof(int)));
  NCK2(cudaMemsetAsync(n->tc_err, 0, sizeof(int), n->stream));
  NCK2(cudaMallocHost((void **)&n->tc_err_h, sizeof(int)));
  NCK2(cudaMemsetAsync(n->m, 0, off * sizeof(float), n->stream));
  NCK2(cudaMemsetAsync(n->v, 0, off * sizeof(float), n->stream));
  for (int l = 0; l < layers; l++) {
    bf16 *x = nullptr;
    float *z = nullptr;
    if (l > 0) NCK2(cudaMalloc((void **)&x, P * n->layers[l].cin * sizeof(bf16)));  // layer 0 reads X0p
    n->X.push_back(x);
    NCK2(cudaMalloc((void **)&z, P * n->layers[l].cout * sizeof(float)));
    n->Z.push_back(z);
  }
  {
    int dev = 0, sms = 0;
    NCK2(cudaGetDevice(&dev));
    NCK2(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    n->nparts = std::min(1024, std::max(1, sms));
  }
  NCK2(cudaMalloc((void **)&n->wpart, (size_t)n->nparts * 64 * 9 * 64 * sizeof(float)));
  NCK2(cudaMalloc((void **)&n->dZ, P * cmax * sizeof(float)));
  NCK2(cudaMalloc((void **)&n->dZ2, P * cmax * sizeof(float)));
  NCK2(cudaMalloc((void **)&n->dZb, P * cmax * sizeof(bf16)));
  NCK2(cudaMalloc((void **)&n->dZb2, P * cmax * sizeof(bf16)));
  NCK2(cudaMalloc((void **)&n->dZb16, P * 16 * sizeof(bf16)));
  n->part_n = std::max<int64_t>(2 * 256, (P + 4095) / 4096 * (int64_t)cmax);  // loss and bias-gradient partials
  NCK2(cudaMalloc((void **)&n->part, n->part_n * sizeof(float)));
  NCK2(cudaMalloc((void **)&n->y, P * sizeof(float)));
  NCK2(cudaMalloc((void **)&n->lossv, 4 * sizeof(float)));
  NCK2(cudaMallocHost((void **)&n->lossh, 4 * sizeof(float)));
  // He-uniform weights (fan-in 9 Cin), zero biases
  for (auto &ly : n->layers) {
    float a = sqrtf(6.f / (9.f * ly.cin));
    if (&ly == &n->layers.back()) a *= 0.1f;
    k_init_uniform<<<g1((int64_t)ly.cout * 9 * ly.cin), 256, 0, n->stream>>>(n->w + ly.woff, (int64_t)ly.cout * 9 * ly.cin,
                                                                              seed + (uint64_t)ly.woff, a);
    NCK2(cudaMemsetAsync(n->w + ly.boff, 0, ly.cout * sizeof(float), n->stream));
  }
  NCK2(cudaStreamSynchronize(n->stream));
#undef NCK2
  *out = n;
  return IGA_OK;
}

extern "C" void iga_nn_destroy(iga_nn_t n) {
  if (!n) return;
  cudaStreamSynchronize(n->stream);
  nn_release(n);
  delete n;
}

extern "C" const char *iga_nn_last_error(iga_nn_t n) { return n ? n->err.c_str() : g_nn_err.c_str(); }

extern "C" iga_status iga_nn_num_params(iga_nn_t n, int64_t *count) {
  if (!n || !count) return IGA_EINVAL;
  *count = n->nparams;
  return IGA_OK;
}

extern "C" iga_status iga_nn_get_params(iga_nn_t n, float *host) {
  if (!n || !host) return IGA_EINVAL;
  NCK(cudaMemcpyAsync(host, n->w, n->nparams * sizeof(float), cudaMemcpyDeviceToHost, n->stream));
  NCK(cudaStreamSynchronize(n->stream));
  return IGA_OK;
}

extern "C" iga_status iga_nn_set_params(iga_nn_t n, const float *host) {
  if (!n || !host) return IGA_EINVAL;
  NCK(cudaMemcpyAsync(n->w, host, n->nparams * sizeof(float), cudaMemcpyHostToDevice, n->stream));
  NCK(cudaMemsetAsync(n->m, 0, n->nparams * sizeof(float), n->stream));
  NCK(cudaMemsetAsync(n->v, 0, n->nparams * sizeof(float), n->stream));
  n->adam_t = 0;
  NCK(cudaStreamSynchronize(n->stream));
  return IGA_OK;
}

#define TCK(call)                                                              \
  do {                                                                         \
    cudaError_t ce_ = (call);                                                  \
    if (ce_ != cudaSuccess) {                                                  \
      n->err = iga_format("tensor-core convolution: %s", cudaGetErrorString(ce_)); \
      return IGA_ECUDA;                                                        \
    }                                                                          \
  } while (0)

// the flag raised by a tensor-core wait that timed out (synchronises the stream)
static iga_status nn_check_tc(iga_nn_s *n) {
  NCK(cudaMemcpyAsync(n->tc_err_h, n->tc_err, sizeof(int), cudaMemcpyDeviceToHost, n->stream));
  NCK(cudaStreamSynchronize(n->stream));
  if (*n->tc_err_h) {
    n->err = "tensor-core convolution: an mbarrier wait timed out";
    cudaMemsetAsync(n->tc_err, 0, sizeof(int), n->stream);
    return IGA_ETIMEOUT;
  }
  return IGA_OK;
}

static ConvArgs conv_args(iga_nn_s *n, int B) {
  ConvArgs a{};
  a.P = B * n->H * n->W;
  a.H = n->H;
  a.W = n->W;
  a.err = n->tc_err;
  return a;
}

// forward pass for B samples: x device FP32 [B][H][W][cin]; result in n->y [B][H][W].
// train: keep the pre-activations (FP32) and the unpadded BF16 input for the backward pass.
static iga_status nn_forward(iga_nn_s *n, const float *x, int B, const float *mask, bool train) {
  const int64_t HW = (int64_t)n->H * n->W, P = (int64_t)B * HW;
  for (auto &ly : n->layers) {
    int cnt = std::max(ly.np * 9 * ly.cp, ly.cin * 9 * ly.np);
    k_prep_w<<<g1(cnt), 256, 0, n->stream>>>(n->w + ly.woff, ly.cin, ly.cout, ly.cp, ly.np, ly.wk, ly.wt);
  }
  k_pad_input<<<g1(P * 16), 256, 0, n->stream>>>(x, n->cin, P, n->X0p, nullptr);
  for (int l = 0; l < n->L; l++) {
    const NNLayer &ly = n->layers[l];
    ConvArgs a = conv_args(n, B);
    a.in = (l == 0) ? n->X0p : n->X[l];
    a.wk = ly.wk;
    a.bias = n->w + ly.boff;
    a.dil = ly.dil;
    a.sign = 1;
    if (l + 1 < n->L) {
      a.z = train ? n->Z[l] : nullptr;
      a.act = n->X[l + 1];
      TCK(launch_conv_tc(ly.cp, ly.np, CONV_EPI_FWD_SILU, a, n->stream));
    } else {
      a.z = n->Z[l];
      TCK(launch_conv_tc(ly.cp, ly.np, CONV_EPI_LAST, a, n->stream));
    }
  }
  k_output<<<g1(P), 256, 0, n->stream>>>(n->Z[n->L - 1], mask, HW, P, n->y);
  NCK(cudaGetLastError());
  return IGA_OK;
}

extern "C" iga_status iga_nn_forward(iga_nn_t n, const float *x, int B, const float *mask, float *y) {
  if (!n || !x || !y || B < 1 || B > n->maxB) {
    if (n) n->err = "bad forward arguments";
    return IGA_EINVAL;
  }
  iga_status st = nn_forward(n, x, B, mask, false);
  if (st != IGA_OK) return st;
  NCK(cudaMemcpyAsync(y, n->y, (size_t)B * n->H * n->W * sizeof(float), cudaMemcpyDeviceToDevice, n->stream));
  return nn_check_tc(n);
}

// forward + backward: masked mean-squared error against tgt [B][H][W]; gradients
// of the loss w.r.t. all parameters into the internal FP32 gradient (and into
// grads_out if non-NULL); the loss into *loss (host).
extern "C" iga_status iga_nn_loss_grad(iga_nn_t n, const float *x, const float *tgt, const float *mask, int B, float *loss,
                                       float *grads_out) {
  if (!n || !x || !tgt || B < 1 || B > n->maxB) {
    if (n) n->err = "bad loss_grad arguments";
    return IGA_EINVAL;
  }
  iga_status st = nn_forward(n, x, B, mask, true);
  if (st != IGA_OK) return st;
  const int64_t HW = (int64_t)n->H * n->W, P = (int64_t)B * HW;
  const int nbl = 256;
  k_loss_partial<<<nbl, 256, 0, n->stream>>>(n->y, tgt, mask, HW, P, n->W, n->H, n->h1, n->part);
  k_loss_final<<<1, 1, 0, n->stream>>>(n->part, nbl, n->lossv);
  k_loss_grad<<<g1(P), 256, 0, n->stream>>>(n->y, tgt, mask, HW, P, n->W, n->H, n->h1, n->lossv, n->dZ);
  // the output layer's gradient in the layouts its weight gradient and its
  // transposed convolution read
  k_pad_grad<<<g1(P * 16), 256, 0, n->stream>>>(n->dZ, P, n->dZb, n->dZb16);
  float *dz = n->dZ, *dz_next = n->dZ2;
  bf16 *dzb = n->dZb, *dzb_next = n->dZb2;
  for (int l = n->L - 1; l >= 0; l--) {
    const NNLayer &ly = n->layers[l];
    // bias gradient: column sums of dZ
    const int64_t chunk = 4096;
    const int nch = (int)((P + chunk - 1) / chunk);
    k_colsum_partial<<<nch, 256, 0, n->stream>>>(dz, P, ly.cout, chunk, n->part);
    k_sum_splits<<<g1(ly.cout), 256, 0, n->stream>>>(n->part, nch, ly.cout, n->g + ly.boff, 0);
    // weight gradient on the tensor cores: dW[co][tap][ci] = sum_p dZ[p][co] X[p + off(tap)][ci],
    // one partial per pixel range, summed in a fixed order
    {
      WgradArgs w{};
      w.x = (l == 0) ? n->X0p : n->X[l];
      w.dz = (l == n->L - 1) ? n->dZb16 : dzb;
      w.ldz = ly.np;
      w.cout = ly.cout;
      w.cin = ly.cin;
      w.part = n->wpart;
      w.dw = n->g + ly.woff;
      w.nparts = n->nparts;
      w.P = (int)P;
      w.H = n->H;
      w.W = n->W;
      w.dil = ly.dil;
      w.err = n->tc_err;
      TCK(launch_conv_wgrad_tc(ly.cp, ly.np, w, n->stream));
    }
    if (l > 0) {
      // dZ of the layer below = (transposed convolution of dZ) * SiLU'(Z below), on the tensor cores
      ConvArgs a = conv_args(n, B);
      a.in = (l == n->L - 1) ? n->dZb16 : dzb;
      a.wk = ly.wt;
      a.zprev = n->Z[l - 1];
      a.z = dz_next;
      a.act = dzb_next;
      a.dil = ly.dil;
      a.sign = -1;
      TCK(launch_conv_tc(ly.np, ly.cin, CONV_EPI_BWD_SILU, a, n->stream));
      std::swap(dz, dz_next);
      std::swap(dzb, dzb_next);
    }
  }
  NCK(cudaGetLastError());
  NCK(cudaMemcpyAsync(n->lossh, n->lossv, 2 * sizeof(float), cudaMemcpyDeviceToHost, n->stream));
  if (grads_out) NCK(cudaMemcpyAsync(grads_out, n->g, n->nparams * sizeof(float), cudaMemcpyDeviceToDevice, n->stream));
  st = nn_check_tc(n);
  if (st != IGA_OK) return st;
  if (loss) *loss = n->lossh[0];
  return IGA_OK;
}

extern "C" iga_status iga_nn_set_h1_weight(iga_nn_t n, float beta) {
  if (!n || !(beta >= 0.f) || !isfinite(beta)) return IGA_EINVAL;
  n->h1 = beta;
  return IGA_OK;
}

extern "C" iga_status iga_nn_adam_step(iga_nn_t n, float lr, float beta1, float beta2, float eps) {
  if (!n || !(lr > 0.f)) return IGA_EINVAL;
  n->adam_t++;
  float c1 = 1.f - powf(beta1, (float)n->adam_t), c2 = 1.f - powf(beta2, (float)n->adam_t);
  k_adam<<<g1(n->nparams), 256, 0, n->stream>>>(n->w, n->g, n->m, n->v, n->nparams, lr, beta1, beta2, eps, c1, c2);
  NCK(cudaGetLastError());
  return IGA_OK;
}
