// FP64 exponential of the residual and reaction kernels, by the table-driven method of
// P. T. P. Tang, "Table-driven implementation of the exponential function in IEEE
// floating-point arithmetic", ACM TOMS 15(2), 1989:
//     x = (32 m + j) ln2/32 + r,   |r| <= ln2/64,   e^x = 2^m 2^(j/32) e^r,
// with k = 32 m + j the integer nearest to x 32/ln2, r = x - k L1 - k L2 (L1 + L2 = ln2/32
// to about 110 bits), e^r - 1 by its Taylor polynomial of degree 6 (truncation below
// |r|^7/7! < 4e-18) and 2^(j/32) from a 32-entry table of doubles.  The power 2^m is put
// into the exponent field with an integer addition.  On GB300 every FP64 operation runs
// on the narrow FP64 pipe (2 per clock per SM), so the 11 FP64 operations per call, one
// table load and a few integer operations matter in the kernels that evaluate e^u at
// every Gauss point.  |x| > 700 and non-finite x go to the CUDA exp().
//
// The constants are the doubles nearest to 32/ln2, ln2/32 (L1; L2 the double nearest to
// the remainder), 2^(j/32) and 1/k!, computed at 60 digits (mpmath) and written as
// hexadecimal literals.
#pragma once
#include <cuda_runtime.h>

__device__ static const double iga_exp_tab[32] = {
    0x1.0000000000000p+0, 0x1.059b0d3158574p+0, 0x1.0b5586cf9890fp+0, 0x1.11301d0125b51p+0,
    0x1.172b83c7d517bp+0, 0x1.1d4873168b9aap+0, 0x1.2387a6e756238p+0, 0x1.29e9df51fdee1p+0,
    0x1.306fe0a31b715p+0, 0x1.371a7373aa9cbp+0, 0x1.3dea64c123422p+0, 0x1.44e086061892dp+0,
    0x1.4bfdad5362a27p+0, 0x1.5342b569d4f82p+0, 0x1.5ab07dd485429p+0, 0x1.6247eb03a5585p+0,
    0x1.6a09e667f3bcdp+0, 0x1.71f75e8ec5f74p+0, 0x1.7a11473eb0187p+0, 0x1.82589994cce13p+0,
    0x1.8ace5422aa0dbp+0, 0x1.93737b0cdc5e5p+0, 0x1.9c49182a3f090p+0, 0x1.a5503b23e255dp+0,
    0x1.ae89f995ad3adp+0, 0x1.b7f76f2fb5e47p+0, 0x1.c199bdd85529cp+0, 0x1.cb720dcef9069p+0,
    0x1.d5818dcfba487p+0, 0x1.dfc97337b9b5fp+0, 0x1.ea4afa2a490dap+0, 0x1.f50765b6e4540p+0};

__device__ __forceinline__ double iga_exp(double x) {
  if (!(fabs(x) <= 700.0)) return exp(x);  // large or non-finite arguments (never on the solve path)
  const double inv_l = 0x1.71547652b82fep+5;   // 32 / ln2
  const double l1 = 0x1.62e42fefa39efp-6;      // ln2 / 32
  const double l2 = 0x1.abc9e3b39803fp-61;     // ln2 / 32 - l1
  const double shifter = 0x1.8p52;             // 1.5 * 2^52: t's low mantissa bits hold k
  const double t = fma(x, inv_l, shifter);
  const int k = __double2loint(t);
  const double kd = t - shifter;
  double r = fma(-kd, l1, x);
  r = fma(-kd, l2, r);
  // e^r - 1 = r (1 + r (1/2 + r (1/6 + r (1/24 + r (1/120 + r / 720)))))
  double q = fma(r, 0x1.6c16c16c16c17p-10, 0x1.1111111111111p-7);
  q = fma(r, q, 0x1.5555555555555p-5);
  q = fma(r, q, 0x1.5555555555555p-3);
  q = fma(r, q, 0x1.0000000000000p-1);
  q = fma(r, q, 1.0);
  const double p = r * q;
  const double s = iga_exp_tab[k & 31];
  const double y = fma(s, p, s);  // 2^(j/32) e^r, in [2^-1/64, 2^(1+1/64)]
  // times 2^m, m = floor(k / 32) (arithmetic shift), exact: |m| <= 1011 keeps y normal
  return __longlong_as_double(__double_as_longlong(y) + ((long long)(k >> 5) << 52));
}
