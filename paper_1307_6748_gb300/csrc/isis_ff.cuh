// isis_ff.cuh -- float-float ("double-FP32") arithmetic for the FP64-accurate
// residual of the defect-correction loop.
//
// GB300 executes FP64 at about 1/50 of its FP32 rate, so the residual kernels
// carry a value as an unevaluated sum hi + lo of two FP32 numbers (|lo| <= ulp(hi)/2,
// about 48 significant bits, relative error near 1e-14 per operation) and do all
// arithmetic with FP32 instructions:
//   - two_sum: the exact sum a + b = s + e (Knuth, TAOCP vol. 2, Sect. 4.2.2);
//   - quick_two_sum: the same when |a| >= |b| (Dekker 1971);
//   - two_prod: the exact product a * b = p + e with one fused multiply-add;
//   - add, mul: the double-length operations built from them (Dekker 1971; the
//     "accurate" addition that also adds the low parts with an exact sum).
// The exponential follows the table-driven method of P. T. P. Tang (ACM TOMS 15,
// 1989) with a 64-entry table of 2^(j/64) in float-float:
//   x = (64 m + j) L + r, L = ln2/64 split in three FP32 parts (n L1 exact), |r| <= L/2,
//   e^x = 2^m 2^(j/64) e^r, e^r - 1 = r + r^2/2 + r^3/6 + r^4/24 + r^5/120,
// where r^3 and higher terms (below 3e-8) need FP32 only; the truncation error
// r^6/720 is below 4e-17.
#pragma once
#include <cuda_runtime.h>

namespace isis {

struct ff {
  float hi, lo;
};

__device__ __forceinline__ ff ff_two_sum(float a, float b) {
  const float s = a + b;
  const float bb = s - a;
  return {s, (a - (s - bb)) + (b - bb)};
}
__device__ __forceinline__ ff ff_quick_two_sum(float a, float b) {
  const float s = a + b;
  return {s, b - (s - a)};
}
__device__ __forceinline__ ff ff_two_prod(float a, float b) {
  const float p = a * b;
  return {p, fmaf(a, b, -p)};
}
__device__ __forceinline__ ff ff_add(ff a, ff b) {
  ff s = ff_two_sum(a.hi, b.hi);
  const ff t = ff_two_sum(a.lo, b.lo);
  s.lo += t.hi;
  s = ff_quick_two_sum(s.hi, s.lo);
  s.lo += t.lo;
  return ff_quick_two_sum(s.hi, s.lo);
}
// Dekker's addition: one exact sum of the high parts, the low parts added in FP32.  Its error is about
// ulp of the low parts, 2^-48 of the larger input: absolute accuracy, which is what the stencil
// differences and their sums need (ff_add keeps relative accuracy under cancellation, at twice the cost).
__device__ __forceinline__ ff ff_add_abs(ff a, ff b) {
  ff s = ff_two_sum(a.hi, b.hi);
  s.lo += a.lo + b.lo;
  return ff_quick_two_sum(s.hi, s.lo);
}
__device__ __forceinline__ ff ff_neg(ff a) { return {-a.hi, -a.lo}; }
__device__ __forceinline__ ff ff_sub(ff a, ff b) { return ff_add(a, ff_neg(b)); }
__device__ __forceinline__ ff ff_add_f(ff a, float b) {
  ff s = ff_two_sum(a.hi, b);
  s.lo += a.lo;
  return ff_quick_two_sum(s.hi, s.lo);
}
__device__ __forceinline__ ff ff_mul(ff a, ff b) {
  ff p = ff_two_prod(a.hi, b.hi);
  p.lo = fmaf(a.hi, b.lo, fmaf(a.lo, b.hi, p.lo));
  return ff_quick_two_sum(p.hi, p.lo);
}
__device__ __forceinline__ ff ff_mul_f(ff a, float b) {
  ff p = ff_two_prod(a.hi, b);
  p.lo = fmaf(a.lo, b, p.lo);
  return ff_quick_two_sum(p.hi, p.lo);
}
// exact scaling by a power of two
__device__ __forceinline__ ff ff_ldexp(ff a, int m) { return {ldexpf(a.hi, m), ldexpf(a.lo, m)}; }
// FP64 -> float-float (one FP64 subtraction) and back
__device__ __forceinline__ ff ff_from_double(double d) {
  const float hi = __double2float_rn(d);
  return {hi, __double2float_rn(d - (double)hi)};
}
// FP64 -> float-float without the FP64 units, for the bulk conversions of the FP64 residual (GB300 runs
// FP64<->FP32 conversions on its few FP64 units): by integer operations on the bit pattern, hi = d with its
// significand cut to 24 bits and lo = the remaining 29 bits cut to 24 significant bits, so
// |d - (hi + lo)| < 2^-47 |d|, hi and lo of d's sign.  |d| < 2^-70 (zero included) gives a signed zero,
// |d| >= 2^127 gives +-Inf and NaN stays NaN (so a non-finite field still shows in the residual norm).
// No FP64 instruction, not even on a branch the compiler might predicate.
__device__ __forceinline__ ff ff_split_bits(double d) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(d);
  const unsigned h = (unsigned)(b >> 32), l = (unsigned)b;
  const unsigned sgn = h & 0x80000000u;
  const int ef = (int)((h >> 20) & 0x7FFu), e = ef - 1023;
  if (e > 126) {
    const bool nan = ef == 0x7FF && (((h & 0xFFFFFu) | l) != 0u);
    return {__uint_as_float(sgn | 0x7F800000u | (nan ? 0x400000u : 0u)), 0.0f};
  }
  if (e < -70) return {__uint_as_float(sgn), 0.0f};
  const float hi = __uint_as_float(sgn | ((unsigned)(e + 127) << 23) | ((h & 0xFFFFFu) << 3) | (l >> 29));
  const unsigned rem = l & 0x1FFFFFFFu;  // the significand bits below hi's, in units of 2^(e - 52)
  if (rem == 0u) return {hi, 0.0f};
  const int top = 31 - __clz(rem);  // position of the leading one, 0..28
  const unsigned man = top >= 23 ? (rem >> (top - 23)) : (rem << (23 - top));
  const float lo = __uint_as_float(sgn | ((unsigned)(e - 52 + top + 127) << 23) | (man & 0x7FFFFFu));
  return {hi, lo};
}
// FP32 -> FP64, exact, by integer operations (no FP64 unit): zero and subnormal floats give a signed
// zero, Inf and NaN stay Inf and NaN.
__device__ __forceinline__ double f2d_bits(float f) {
  const unsigned u = __float_as_uint(f);
  const unsigned sgn = u & 0x80000000u, ef = (u >> 23) & 0xFFu, man = u & 0x7FFFFFu;
  if (ef == 0u) return __hiloint2double((int)sgn, 0);
  const unsigned e = ef == 0xFFu ? 0x7FFu : ef - 127u + 1023u;
  return __hiloint2double((int)(sgn | (e << 20) | (man >> 3)), (int)(man << 29));
}
__device__ __forceinline__ ff ff_load(const float2& v) { return {v.x, v.y}; }
__device__ __forceinline__ float2 ff_store(ff a) { return make_float2(a.hi, a.lo); }

// Constants of exp_ff, filled on the host (ff_exp_consts).
struct FFExp {
  float invL;        // 64 / ln 2
  float L1, L2, L3;  // ln2/64 = L1 + L2 + L3, L1 with 13 significant bits (n L1 exact for |n| < 2^11)
};

// e^x for |x| < 22 (|n| < 2^11); tab: 64 float-float values 2^(j/64) (shared or global memory).
__device__ __forceinline__ ff exp_ff(ff x, const float2* tab, const FFExp& k) {
  const float nf = rintf(x.hi * k.invL);
  const int n = (int)nf;
  // r = x - n L: n L1 is exact and x.hi - n L1 is exact (Sterbenz), so one fma gives it exactly
  ff r = ff_two_sum(fmaf(-nf, k.L1, x.hi), x.lo);
  r = ff_add(r, ff_two_prod(-nf, k.L2));
  r = ff_add_f(r, -nf * k.L3);
  // e^r - 1
  ff r2 = ff_two_prod(r.hi, r.hi);
  r2.lo = fmaf(2.0f * r.hi, r.lo, r2.lo);
  const float c = r2.hi * r.hi * fmaf(r.hi, fmaf(r.hi, 1.0f / 120.0f, 1.0f / 24.0f), 1.0f / 6.0f);
  ff p = ff_add(r, ff{0.5f * r2.hi, 0.5f * r2.lo});
  p = ff_add_f(p, c);
  const ff T = ff_load(tab[n & 63]);
  return ff_ldexp(ff_add(T, ff_mul(T, p)), n >> 6);
}

// Host: the 64-entry table 2^(j/64) and the constants of exp_ff, from extended precision.
void ff_exp_table_fill(float2* host64);
FFExp ff_exp_consts();
// Host: split an FP64 value into float-float (hi = FP32 rounding, lo = FP32 rounding of the rest).
inline float2 ff_split_host(double v) {
  const float hi = (float)v;
  return make_float2(hi, (float)(v - (double)hi));
}

}  // namespace isis
