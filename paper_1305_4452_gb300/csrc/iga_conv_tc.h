// Tensor-core (tcgen05) implicit-GEMM 3x3 convolution of the neural operator.
#pragma once
#include <cuda_bf16.h>
#include <cuda_runtime.h>

enum {
  CONV_EPI_FWD_SILU = 0,  // z = acc + bias (FP32, optional), act = SiLU(z) in BF16
  CONV_EPI_LAST = 1,      // z[p] = acc[p][0] + bias[0] (one output channel)
  CONV_EPI_BWD_SILU = 2   // d = acc * SiLU'(zprev): z = d (FP32), act = d (BF16)
};

struct ConvArgs {
  const __nv_bfloat16 *in;  // [P][CIN] NHWC
  const __nv_bfloat16 *wk;  // [NOUT][9][CIN]
  const float *bias;        // [NOUT] or null
  const float *zprev;       // [P][NOUT] (backward epilogue)
  float *z;                 // FP32 output (see the epilogues); may be null for CONV_EPI_FWD_SILU
  __nv_bfloat16 *act;       // BF16 output [P][NOUT]
  int P, H, W, dil, sign;   // pixels (B*H*W), grid, dilation, +1 forward / -1 transposed
  int *err;                 // set to 1 when an mbarrier wait times out
};

// Compiled shapes (hidden width H in {16, 32, 64}, inputs padded to 16 channels, the
// one-channel output padded to 16): FWD (16,H) and (H,H), LAST (H,16), BWD (H,H) and
// (16,H).  Any other (cin, nout, epi) returns cudaErrorInvalidValue.
cudaError_t launch_conv_tc(int cin, int nout, int epi, const ConvArgs &a, cudaStream_t stream);

struct WgradArgs {
  const __nv_bfloat16 *x;   // [P][CINP] layer input (channels beyond cin are zero)
  const __nv_bfloat16 *dz;  // [P][ldz] output gradient, channels < cout used
  int ldz, cout, cin;       // dz row length; real output / input channels
  float *part;              // [nparts][NOUTP][9][CINP] per-CTA partial sums (scratch)
  float *dw;                // [cout][9][cin] result (the parameter layout)
  int nparts;               // CTAs (pixel ranges), <= 1024
  int P, H, W, dil;
  int *err;
};

// dW[co][tap][ci] = sum_p dZ[p][co] X[p + dil * off(tap)][ci] on the tensor cores, with
// the input padded to CINP and the gradient channels to NOUTP (16, 32 or 64).
cudaError_t launch_conv_wgrad_tc(int cinp, int noutp, const WgradArgs &a, cudaStream_t stream);
