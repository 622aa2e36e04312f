// isis_exp64.cuh -- FP64 exponential for the FP64 residual kernels.
//
// Table-driven method of P. T. P. Tang, "Table-driven implementation of the
// exponential function in IEEE floating-point arithmetic", ACM TOMS 15 (1989):
//   x = (256 m + j) ln2/256 + r,  |r| <= ln2/512,  0 <= j < 256
//   e^x = 2^m * 2^(j/256) * e^r,  e^r = 1 + r + r^2/2! + ... + r^5/5!
// The truncation error r^6/6! < 1e-20 is far below one ulp; the table holds
// 2^(j/256) rounded to double (filled on the host in extended precision).
// Arguments outside [-700, 700] (and NaN) take the library exp().
#pragma once
#include <cuda_runtime.h>

namespace isis {

// tab: 256 doubles, tab[j] = 2^(j/256) (see exp_table_fill)
__device__ __forceinline__ double exp_tang(double x, const double* __restrict__ tab) {
  if (!(fabs(x) <= 700.0)) return exp(x);
  const double kInvL = 369.3299304675746;            // 256 / ln 2
  const double kLhi = 0.002707604318857193;           // ln2/256 with the low 32 mantissa bits cleared
  const double kLlo = 1.855205093371747e-09;          // ln2/256 - kLhi
  const double kShift = 6755399441055744.0;           // 1.5 * 2^52: rounds to an integer
  double t = fma(x, kInvL, kShift);
  int n = __double2loint(t);
  double nd = t - kShift;
  double r = fma(-nd, kLhi, x);
  r = fma(-nd, kLlo, r);
  double p = fma(r, 1.0 / 120.0, 1.0 / 24.0);
  p = fma(p, r, 1.0 / 6.0);
  p = fma(p, r, 0.5);
  p = fma(p, r, 1.0);
  p = p * r;  // e^r - 1
  double Tj = __ldg(&tab[n & 255]);
  double y = fma(Tj, p, Tj);
  int m = n >> 8;  // arithmetic shift: floor(n / 256)
  return __hiloint2double(__double2hiint(y) + m * (1 << 20), __double2loint(y));
}

// Host: fill a 256-entry host array with 2^(j/256) rounded from long double.
void exp_table_fill(double* host256);

}  // namespace isis
