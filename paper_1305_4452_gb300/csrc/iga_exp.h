// FP64 exponential of the residual and reaction kernels, by the table-driven method of
// P. T. P. Tang, "Table-driven implementation of the exponential function in IEEE
// floating-point arithmetic", ACM TOMS 15(2), 1989:
//     x = (64 m + j) ln2/64 + r,   |r| <= ln2/128,   e^x = 2^m 2^(j/64) e^r,
// with k = 64 m + j the integer nearest to x 64/ln2, r = x - k L1 - k L2 (L1 + L2 = ln2/64
// to about 110 bits), e^r - 1 by its Taylor polynomial of degree 5 (truncation below
// |r|^6/6! e^|r| < 4e-17) and 2^(j/64) from a 64-entry table of doubles.  The power 2^m is
// put into the exponent field with an integer addition, and the range test is an integer
// comparison of the argument's high word.  On GB300 every FP64 operation runs on the narrow
// FP64 pipe (2 per clock per SM), so the 10 FP64 operations per call, one table load and a
// few integer operations matter in the kernels that evaluate e^u at every Gauss point.
// |x| >= 700 and non-finite x go to the CUDA exp().
//
// The constants are the doubles nearest to 64/ln2, ln2/64 (L1; L2 the double nearest to
// the remainder), 2^(j/64) and 1/k!, computed at 60 digits (mpmath) and written as
// hexadecimal literals.
#pragma once
#include <cuda_runtime.h>

__device__ static const double iga_exp_tab[64] = {
    0x1.0000000000000p+0, 0x1.02c9a3e778061p+0, 0x1.059b0d3158574p+0, 0x1.0874518759bc8p+0,
    0x1.0b5586cf9890fp+0, 0x1.0e3ec32d3d1a2p+0, 0x1.11301d0125b51p+0, 0x1.1429aaea92de0p+0,
    0x1.172b83c7d517bp+0, 0x1.1a35beb6fcb75p+0, 0x1.1d4873168b9aap+0, 0x1.2063b88628cd6p+0,
    0x1.2387a6e756238p+0, 0x1.26b4565e27cddp+0, 0x1.29e9df51fdee1p+0, 0x1.2d285a6e4030bp+0,
    0x1.306fe0a31b715p+0, 0x1.33c08b26416ffp+0, 0x1.371a7373aa9cbp+0, 0x1.3a7db34e59ff7p+0,
    0x1.3dea64c123422p+0, 0x1.4160a21f72e2ap+0, 0x1.44e086061892dp+0, 0x1.486a2b5c13cd0p+0,
    0x1.4bfdad5362a27p+0, 0x1.4f9b2769d2ca7p+0, 0x1.5342b569d4f82p+0, 0x1.56f4736b527dap+0,
    0x1.5ab07dd485429p+0, 0x1.5e76f15ad2148p+0, 0x1.6247eb03a5585p+0, 0x1.6623882552225p+0,
    0x1.6a09e667f3bcdp+0, 0x1.6dfb23c651a2fp+0, 0x1.71f75e8ec5f74p+0, 0x1.75feb564267c9p+0,
    0x1.7a11473eb0187p+0, 0x1.7e2f336cf4e62p+0, 0x1.82589994cce13p+0, 0x1.868d99b4492edp+0,
    0x1.8ace5422aa0dbp+0, 0x1.8f1ae99157736p+0, 0x1.93737b0cdc5e5p+0, 0x1.97d829fde4e50p+0,
    0x1.9c49182a3f090p+0, 0x1.a0c667b5de565p+0, 0x1.a5503b23e255dp+0, 0x1.a9e6b5579fdbfp+0,
    0x1.ae89f995ad3adp+0, 0x1.b33a2b84f15fbp+0, 0x1.b7f76f2fb5e47p+0, 0x1.bcc1e904bc1d2p+0,
    0x1.c199bdd85529cp+0, 0x1.c67f12e57d14bp+0, 0x1.cb720dcef9069p+0, 0x1.d072d4a07897cp+0,
    0x1.d5818dcfba487p+0, 0x1.da9e603db3285p+0, 0x1.dfc97337b9b5fp+0, 0x1.e502ee78b3ff6p+0,
    0x1.ea4afa2a490dap+0, 0x1.efa1bee615a27p+0, 0x1.f50765b6e4540p+0, 0x1.fa7c1819e90d8p+0};

__device__ __forceinline__ double iga_exp(double x) {
  // |x| < 700: the high word of |x| below that of 700.0 (0x4085E000); NaN and infinities fail it
  if (!(((unsigned)__double2hiint(x) & 0x7fffffffu) < 0x4085E000u)) return exp(x);
  const double inv_l = 0x1.71547652b82fep+6;   // 64 / ln2
  const double l1 = 0x1.62e42fefa39efp-7;      // ln2 / 64
  const double l2 = 0x1.abc9e3b39803fp-62;     // ln2 / 64 - l1
  const double shifter = 0x1.8p52;             // 1.5 * 2^52: t's low mantissa bits hold k
  const double t = fma(x, inv_l, shifter);
  const int k = __double2loint(t);
  const double kd = t - shifter;
  double r = fma(-kd, l1, x);
  r = fma(-kd, l2, r);
  // e^r - 1 = r (1 + r (1/2 + r (1/6 + r (1/24 + r / 120))))
  double q = fma(r, 0x1.1111111111111p-7, 0x1.5555555555555p-5);
  q = fma(r, q, 0x1.5555555555555p-3);
  q = fma(r, q, 0x1.0000000000000p-1);
  q = fma(r, q, 1.0);
  const double p = r * q;
  const double s = iga_exp_tab[k & 63];
  const double y = fma(s, p, s);  // 2^(j/64) e^r, in [2^-1/128, 2^(1+1/128)]
  // times 2^m, m = floor(k / 64) (arithmetic shift), exact: |m| <= 1010 keeps y normal
  return __longlong_as_double(__double_as_longlong(y) + ((long long)(k >> 6) << 52));
}
