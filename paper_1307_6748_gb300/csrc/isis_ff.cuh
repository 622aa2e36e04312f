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
// A normalised float-float value hi + lo (|lo| <= ulp(hi)/2) to FP64, rounded to nearest even as one FP64
// addition of the two would round it, by integer operations (an FP64 addition runs on the narrow FP64 pipe).
// The exact sum is formed in a 64-bit integer in units of 2^(e_hi - 189): |hi| at bits 39..62, |lo| shifted by
// the exponent gap (bits shifted out only set a sticky flag), then cut to 53 bits.  hi zero, subnormal, Inf or
// NaN, and lo zero or subnormal, give f2d_bits(hi) (the flush of f2d_bits); a pair that is not normalised
// (exponent gap < 24) takes the FP64 addition.
__device__ __forceinline__ double ff_to_double_bits(float hi, float lo) {
  const unsigned uh = __float_as_uint(hi), ul = __float_as_uint(lo);
  const int eh = (int)((uh >> 23) & 0xFFu), el = (int)((ul >> 23) & 0xFFu);
  if (eh == 0 || eh == 0xFF || el == 0) return f2d_bits(hi);
  const int gap = eh - el;
  if (gap < 24) return f2d_bits(hi) + f2d_bits(lo);
  const unsigned long long H = (unsigned long long)((uh & 0x7FFFFFu) | 0x800000u);
  const unsigned long long L = (unsigned long long)((ul & 0x7FFFFFu) | 0x800000u);
  unsigned long long A = H << 39, Lp;
  bool sticky;
  const int sh = 39 - gap;  // <= 15
  if (sh >= 0) {
    Lp = L << sh;
    sticky = false;
  } else if (sh > -24) {
    Lp = L >> (-sh);
    sticky = (L & ((1ull << (-sh)) - 1ull)) != 0ull;
  } else {
    Lp = 0ull;
    sticky = true;
  }
  if ((uh ^ ul) & 0x80000000u) {
    A -= Lp;
    if (sticky) A -= 1ull;  // the exact value lies strictly between A and A + 1
  } else {
    A += Lp;
  }
  // A in [2^61, 2^63): keep 53 bits
  const int shift = (A >> 62) ? 10 : 9;
  unsigned long long M = A >> shift;
  const unsigned long long rem = A & ((1ull << shift) - 1ull), halfu = 1ull << (shift - 1);
  if (rem > halfu || (rem == halfu && (sticky || (M & 1ull)))) ++M;
  int E = eh - 127 + (shift - 10);  // unbiased exponent of the result
  if (M >> 53) {
    M >>= 1;
    ++E;
  }
  const unsigned long long bits = ((unsigned long long)(uh & 0x80000000u) << 32) |
                                  ((unsigned long long)(E + 1023) << 52) | (M & 0xFFFFFFFFFFFFFull);
  return __longlong_as_double((long long)bits);
}
__device__ __forceinline__ ff ff_load(const float2& v) { return {v.x, v.y}; }
__device__ __forceinline__ float2 ff_store(ff a) { return make_float2(a.hi, a.lo); }

// ---- two float-float values at once, in packed FP32x2 instructions (sm_100 family) ----
// ff2 holds the high parts of two values in one float2 and their low parts in another.  Each operation is
// the scalar one of the same name done lane by lane: __fadd2_rn, __fmul2_rn and __ffma2_rn round each lane
// as an FP32 add, multiply and fused multiply-add do, and a subtraction a - b is the exact fma b * (-1) + a,
// so both lanes give the scalar results bit for bit at half the instruction count.
struct ff2 {
  float2 hi, lo;
};
__device__ __forceinline__ float2 f2_add(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 f2_sub(float2 a, float2 b) { return __ffma2_rn(b, make_float2(-1.0f, -1.0f), a); }
__device__ __forceinline__ float2 f2_mul(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 f2_fma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 f2_bc(float a) { return make_float2(a, a); }

__device__ __forceinline__ ff2 ff2_two_sum(float2 a, float2 b) {
  const float2 s = f2_add(a, b);
  const float2 bb = f2_sub(s, a);
  return {s, f2_add(f2_sub(a, f2_sub(s, bb)), f2_sub(b, bb))};
}
__device__ __forceinline__ ff2 ff2_quick_two_sum(float2 a, float2 b) {
  const float2 s = f2_add(a, b);
  return {s, f2_sub(b, f2_sub(s, a))};
}
__device__ __forceinline__ ff2 ff2_two_prod(float2 a, float2 b) {
  const float2 p = f2_mul(a, b);
  return {p, f2_fma(a, b, make_float2(-p.x, -p.y))};
}
__device__ __forceinline__ ff2 ff2_add(ff2 a, ff2 b) {
  ff2 s = ff2_two_sum(a.hi, b.hi);
  const ff2 t = ff2_two_sum(a.lo, b.lo);
  s.lo = f2_add(s.lo, t.hi);
  s = ff2_quick_two_sum(s.hi, s.lo);
  s.lo = f2_add(s.lo, t.lo);
  return ff2_quick_two_sum(s.hi, s.lo);
}
__device__ __forceinline__ ff2 ff2_add_abs(ff2 a, ff2 b) {
  ff2 s = ff2_two_sum(a.hi, b.hi);
  s.lo = f2_add(s.lo, f2_add(a.lo, b.lo));
  return ff2_quick_two_sum(s.hi, s.lo);
}
__device__ __forceinline__ ff2 ff2_neg(ff2 a) {
  return {make_float2(-a.hi.x, -a.hi.y), make_float2(-a.lo.x, -a.lo.y)};
}
__device__ __forceinline__ ff2 ff2_sub(ff2 a, ff2 b) { return ff2_add(a, ff2_neg(b)); }
__device__ __forceinline__ ff2 ff2_add_f(ff2 a, float2 b) {
  ff2 s = ff2_two_sum(a.hi, b);
  s.lo = f2_add(s.lo, a.lo);
  return ff2_quick_two_sum(s.hi, s.lo);
}
__device__ __forceinline__ ff2 ff2_mul(ff2 a, ff2 b) {
  ff2 p = ff2_two_prod(a.hi, b.hi);
  p.lo = f2_fma(a.hi, b.lo, f2_fma(a.lo, b.hi, p.lo));
  return ff2_quick_two_sum(p.hi, p.lo);
}
// both lanes the same float-float constant
__device__ __forceinline__ ff2 ff2_bc(float2 v) { return {f2_bc(v.x), f2_bc(v.y)}; }
// the float-float values x (lane 0) and y (lane 1)
__device__ __forceinline__ ff2 ff2_pack(ff x, ff y) { return {make_float2(x.hi, y.hi), make_float2(x.lo, y.lo)}; }

// Constants of exp_ff2, filled on the host (ff_exp_consts).
struct FFExp {
  float invL;        // 64 / ln 2
  float L1, L2, L3;  // ln2/64 = L1 + L2 + L3, L1 with 13 significant bits (n L1 exact for |n| < 2^11)
};

// Host: the 64-entry table 2^(j/64) and the constants of exp_ff2, from extended precision.
void ff_exp_table_fill(float2* host64);
FFExp ff_exp_consts();
// Host: split an FP64 value into float-float (hi = FP32 rounding, lo = FP32 rounding of the rest).
inline float2 ff_split_host(double v) {
  const float hi = (float)v;
  return make_float2(hi, (float)(v - (double)hi));
}

// e^x of both lanes, for |x| < 22 (|n| < 2^11) per lane; a lane outside that range gives an unspecified
// value.  tab: 64 float-float values 2^(j/64) (shared or global memory).  The steps are Tang's, in packed
// arithmetic; the rounding to n, the table reads and the final scaling by 2^(n >> 6) are per lane, the
// scaling an exact multiply by a power of two built from its bits.
__device__ __forceinline__ ff2 exp_ff2(ff2 x, const float2* tab, const FFExp& k) {
  const float2 t = f2_mul(x.hi, f2_bc(k.invL));
  const float2 nf = make_float2(rintf(t.x), rintf(t.y));
  const int n0 = (int)nf.x, n1 = (int)nf.y;
  const float2 mnf = make_float2(-nf.x, -nf.y);
  ff2 r = ff2_two_sum(f2_fma(mnf, f2_bc(k.L1), x.hi), x.lo);
  r = ff2_add(r, ff2_two_prod(mnf, f2_bc(k.L2)));
  r = ff2_add_f(r, f2_mul(mnf, f2_bc(k.L3)));
  ff2 r2 = ff2_two_prod(r.hi, r.hi);
  r2.lo = f2_fma(f2_mul(f2_bc(2.0f), r.hi), r.lo, r2.lo);
  const float2 c = f2_mul(f2_mul(r2.hi, r.hi),
                          f2_fma(r.hi, f2_fma(r.hi, f2_bc(1.0f / 120.0f), f2_bc(1.0f / 24.0f)), f2_bc(1.0f / 6.0f)));
  ff2 p = ff2_add(r, ff2{f2_mul(f2_bc(0.5f), r2.hi), f2_mul(f2_bc(0.5f), r2.lo)});
  p = ff2_add_f(p, c);
  const ff2 T = ff2_pack(ff_load(tab[n0 & 63]), ff_load(tab[n1 & 63]));
  const ff2 v = ff2_add(T, ff2_mul(T, p));
  const int m0 = min(max(n0 >> 6, -126), 127), m1 = min(max(n1 >> 6, -126), 127);
  const float2 sc = make_float2(__int_as_float((m0 + 127) << 23), __int_as_float((m1 + 127) << 23));
  return {f2_mul(v.hi, sc), f2_mul(v.lo, sc)};
}

}  // namespace isis
