// isis_kernels.cu -- non-templated kernels shared by the solver instantiations.
#include <cstring>

#include "isis_solver.cuh"

namespace isis {

__global__ void __launch_bounds__(kNormThreads) reduce_final(const double* __restrict__ part, int nparts,
                                                             double* __restrict__ out) {
  // fixed assignment of partials to threads and a fixed tree: reproducible
  double v = 0.0;
  for (int t = threadIdx.x; t < nparts; t += blockDim.x) v += part[t];
  __shared__ double red[kNormThreads / 32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x < 32) {
    v = threadIdx.x < kNormThreads / 32 ? red[threadIdx.x] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if (threadIdx.x == 0) *out = v;
  }
}

__global__ void publish_scalars(const double* __restrict__ scal, int ns, const int* __restrict__ iflags, int ni,
                                double* hd, int* hi) {
  const int t = threadIdx.x;
  if (t < ns) hd[t] = scal[t];
  if (t < ni) hi[t] = iflags[t];
}

}  // namespace isis

namespace isis {

// Four cells k = 4q .. 4q+3 of a row (i, j), row-major position g0 = 4q' (a multiple of 4; N >= 8): in the
// red/black FP32 layout, (k, k+2) sit side by side at place g0/2 of the half of colour (i + j) & 1, and
// (k+1, k+3) at the same place of the other half.  pe and po receive those two places.
__device__ __forceinline__ void rb_quad(int lg, size_t g0, unsigned& pe, unsigned& po) {
  const unsigned row = (unsigned)(g0 >> lg), m = (1u << lg) - 1u;
  const unsigned half = 1u << (3 * lg - 1), base = (unsigned)(g0 >> 1);
  const bool odd = (((row >> lg) + (row & m)) & 1u) != 0u;
  pe = (odd ? half : 0u) + base;
  po = (odd ? 0u : half) + base;
}

// One thread per four cells (row-major quads): 16-byte and 8-byte accesses, every cell's bytes moved once.
__global__ void rb_to_ff(const float* __restrict__ psi, float2* __restrict__ pff, int lg, float2 shift) {
  const size_t q = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= ((size_t)1 << (3 * lg - 2))) return;
  unsigned pe, po;
  rb_quad(lg, 4 * q, pe, po);
  const float2 ve = *reinterpret_cast<const float2*>(psi + pe), vo = *reinterpret_cast<const float2*>(psi + po);
  const ff sh = ff_load(shift);
  const float2 a = ff_store(ff_add_f(sh, ve.x)), b = ff_store(ff_add_f(sh, vo.x));
  const float2 c = ff_store(ff_add_f(sh, ve.y)), d = ff_store(ff_add_f(sh, vo.y));
  float4* o = reinterpret_cast<float4*>(pff + 4 * q);
  o[0] = make_float4(a.x, a.y, b.x, b.y);
  o[1] = make_float4(c.x, c.y, d.x, d.y);
}

__global__ void update_ff(float2* __restrict__ pff, const float* __restrict__ e, int lg,
                          const float* __restrict__ emean) {
  const size_t q = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= ((size_t)1 << (3 * lg - 2))) return;
  unsigned pe, po;
  rb_quad(lg, 4 * q, pe, po);
  float2 ve = *reinterpret_cast<const float2*>(e + pe), vo = *reinterpret_cast<const float2*>(e + po);
  if (emean) {  // Poisson: the correction's mean removed (in FP32, as e is)
    const float mu = *emean;
    ve.x -= mu; ve.y -= mu; vo.x -= mu; vo.y -= mu;
  }
  float4* io = reinterpret_cast<float4*>(pff + 4 * q);
  const float4 u0 = io[0], u1 = io[1];
  const float2 a = ff_store(ff_add_f(ff{u0.x, u0.y}, ve.x)), b = ff_store(ff_add_f(ff{u0.z, u0.w}, vo.x));
  const float2 c = ff_store(ff_add_f(ff{u1.x, u1.y}, ve.y)), d = ff_store(ff_add_f(ff{u1.z, u1.w}, vo.y));
  io[0] = make_float4(a.x, a.y, b.x, b.y);
  io[1] = make_float4(c.x, c.y, d.x, d.y);
}

// Two cells per thread (n even): one 16-byte load, one 16-byte store.  The float-float value goes to FP64 by
// integer operations (ff_to_double_bits, the rounding of one FP64 addition); f(R) then adds its background in
// one FP64 addition (has_base).
__global__ void ff_to_f64(const float2* __restrict__ pff, double* __restrict__ phi, size_t n, double base,
                          int has_base) {
  const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (2 * t >= n) return;
  const float4 v = reinterpret_cast<const float4*>(pff)[t];
  double d0 = ff_to_double_bits(v.x, v.y), d1 = ff_to_double_bits(v.z, v.w);
  if (has_base) {
    d0 += base;
    d1 += base;
  }
  if ((reinterpret_cast<uintptr_t>(phi) & 15u) == 0) {  // the caller's array: 8-byte alignment is all it promises
    reinterpret_cast<double2*>(phi)[t] = make_double2(d0, d1);
  } else {
    phi[2 * t] = d0;
    phi[2 * t + 1] = d1;
  }
}

__global__ void fofr_exp_ff(const float2* __restrict__ psi, float2* __restrict__ E, size_t n,
                            const float2* __restrict__ tab, FFExp ek) {
  const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (2 * t >= n) return;
  const float4 pv = reinterpret_cast<const float4*>(psi)[t];
  const ff2 p = ff2{make_float2(pv.x, pv.z), make_float2(pv.y, pv.w)};
  // exp_ff2 covers |psi| < 22; beyond (no physical field gets there) the FP64 library exp
  ff2 e = exp_ff2(p, tab, ek);
  if (!(fabsf(p.hi.x) < 20.0f)) {
    const ff v = ff_from_double(exp((double)p.hi.x + (double)p.lo.x));
    e.hi.x = v.hi;
    e.lo.x = v.lo;
  }
  if (!(fabsf(p.hi.y) < 20.0f)) {
    const ff v = ff_from_double(exp((double)p.hi.y + (double)p.lo.y));
    e.hi.y = v.hi;
    e.lo.y = v.lo;
  }
  reinterpret_cast<float4*>(E)[t] = make_float4(e.hi.x, e.lo.x, e.hi.y, e.lo.y);
}

__global__ void mean_to_f32(const double* __restrict__ sum, double inv_n, float* __restrict__ out) {
  if (threadIdx.x == 0 && blockIdx.x == 0) *out = (float)(*sum * inv_n);
}

__global__ void __launch_bounds__(kNormThreads) moments_to_rb(const double* __restrict__ v, float* __restrict__ rb,
                                                              int lg, double* __restrict__ part2,
                                                              double* __restrict__ part1) {
  // four cells per iteration, two iterations unrolled (four 16-byte loads in flight per thread), fixed
  // assignment: reproducible
  const size_t nq = (size_t)1 << (3 * lg - 2);
  ff s1 = {0.f, 0.f};
  float s2 = 0.f;
  const bool al = (reinterpret_cast<uintptr_t>(v) & 15u) == 0;  // the caller's array: 16-byte loads if aligned
#pragma unroll 2
  for (size_t q = (size_t)blockIdx.x * blockDim.x + threadIdx.x; q < nq; q += (size_t)gridDim.x * blockDim.x) {
    double2 a, b;
    if (al) {
      a = reinterpret_cast<const double2*>(v)[2 * q];
      b = reinterpret_cast<const double2*>(v)[2 * q + 1];
    } else {
      a = make_double2(v[4 * q], v[4 * q + 1]);
      b = make_double2(v[4 * q + 2], v[4 * q + 3]);
    }
    const ff x0 = ff_split_bits(a.x), x1 = ff_split_bits(a.y), x2 = ff_split_bits(b.x), x3 = ff_split_bits(b.y);
    s1 = ff_add(s1, ff_add(ff_add(x0, x1), ff_add(x2, x3)));
    const float d0 = ff_add_f(x0, -1.0f).hi, d1 = ff_add_f(x1, -1.0f).hi;
    const float d2 = ff_add_f(x2, -1.0f).hi, d3 = ff_add_f(x3, -1.0f).hi;
    s2 = fmaf(d0, d0, fmaf(d1, d1, fmaf(d2, d2, fmaf(d3, d3, s2))));
    unsigned pe, po;
    rb_quad(lg, 4 * q, pe, po);
    *reinterpret_cast<float2*>(rb + pe) = make_float2(x0.hi, x2.hi);
    *reinterpret_cast<float2*>(rb + po) = make_float2(x1.hi, x3.hi);
  }
  block_sum_store<double>((double)s2, part2);
  __syncthreads();
  block_sum_store<double>((double)s1.hi + (double)s1.lo, part1);
}

__global__ void __launch_bounds__(kNormThreads) sum_f32_partial(const float* __restrict__ v, size_t n,
                                                                double* __restrict__ part) {
  // four values per iteration (one 16-byte load; n a multiple of 4)
  ff s = {0.f, 0.f};
  const size_t n4 = n >> 2;
#pragma unroll 2
  for (size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x; t < n4; t += (size_t)gridDim.x * blockDim.x) {
    const float4 a = reinterpret_cast<const float4*>(v)[t];
    s = ff_add(s, ff_add(ff_two_sum(a.x, a.y), ff_two_sum(a.z, a.w)));
  }
  block_sum_store<double>((double)s.hi + (double)s.lo, part);
}
}  // namespace isis

namespace isis {

// ---------------------------------------------------------------------------
// The f(R) residual in float-float (same quantity as fofr_prep64 +
// outer_residual_fofr, at FP32 instruction throughput).  With psi = u - u_bar,
// E = e^psi and C = e^{u_bar}:
//   L(u) = C h^-2 (1/2) sum_f (E + E_nb)(psi_nb - psi) - S,
//   S = K1 (eta - 1) - Kx expm1(-psi/(n+1)) + dK,  Kx = K2 e^{-u_bar/(n+1)}, dK = K3 - Kx,
// which is Sect. 4.2's operator with b = e^u and the source written without the
// cancellation of its two large terms.
// ---------------------------------------------------------------------------

void ff_exp_table_fill(float2* host64) {
  for (int j = 0; j < 64; ++j) {
    const long double v = exp2l((long double)j / 64.0L);
    const float hi = (float)v;
    host64[j] = make_float2(hi, (float)(v - (long double)hi));
  }
}

FFExp ff_exp_consts() {
  const long double L = logl(2.0L) / 64.0L;
  FFExp k;
  k.invL = (float)(1.0L / L);
  float l1 = (float)L;
  unsigned int bits;
  memcpy(&bits, &l1, sizeof(bits));
  bits &= ~0x7FFu;  // keep 13 significant bits: n * L1 is exact for |n| < 2^11
  memcpy(&l1, &bits, sizeof(l1));
  k.L1 = l1;
  const long double rest = L - (long double)l1;
  k.L2 = (float)rest;
  k.L3 = (float)(rest - (long double)k.L2);
  return k;
}

// out[t] = ff_to_double_bits(hl[2t], hl[2t+1]) (self-test of the FP64 write-back's conversion).
__global__ void selftest_ff_to_f64(const float* __restrict__ hl, double* __restrict__ out, int n) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t < n) out[t] = ff_to_double_bits(hl[2 * t], hl[2 * t + 1]);
}

// e^x of x[2t] and x[2t+1] as the two lanes of exp_ff2 (one thread per pair).
__global__ void selftest_exp_ff(const double* __restrict__ x, double* __restrict__ y, int n,
                                const float2* __restrict__ tab, FFExp ek) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (2 * t >= n) return;
  const bool two = 2 * t + 1 < n;
  const ff2 v = exp_ff2(ff2_pack(ff_from_double(x[2 * t]), ff_from_double(x[two ? 2 * t + 1 : 2 * t])), tab, ek);
  y[2 * t] = (double)v.hi.x + (double)v.lo.x;
  if (two) y[2 * t + 1] = (double)v.hi.y + (double)v.lo.y;
}

// The pair (k, k+1) of a float-float grid starting at cell q (q even): one 16-byte load.
__device__ __forceinline__ ff2 ff2_pair(const float2* __restrict__ a, size_t q) {
  const float4 v = *reinterpret_cast<const float4*>(a + q);
  return ff2{make_float2(v.x, v.z), make_float2(v.y, v.w)};
}

// Two cells per thread, (k, k+1) with k even, in packed float-float arithmetic (see outer_residual_ff).
__global__ void __launch_bounds__(kNormThreads) outer_residual_fofr_ff(int lg, FofrFF c,
                                                                       const double* __restrict__ eta,
                                                                       const float2* __restrict__ psi,
                                                                       const float2* __restrict__ E,
                                                                       const float2* __restrict__ tab,
                                                                       float* __restrict__ r32,
                                                                       float* __restrict__ B32,
                                                                       double* __restrict__ part,
                                                                       double* __restrict__ phi_out, double base) {
  __shared__ float2 stab[64];
  if (threadIdx.x < 64) stab[threadIdx.x] = tab[threadIdx.x];
  __syncthreads();
  // 32-bit positions: N <= 1024, so N^3 <= 2^30
  const unsigned np = 1u << (3 * lg - 1), half = np, m = (1u << lg) - 1u;
  const ff2 Cih2 = ff2_bc(c.Cih2), K1 = ff2_bc(c.K1), Kx = ff2_bc(c.Kx), minv = ff2_bc(c.minv);
  const float2 ub = c.ubff;
  float acc = 0.f;
  auto cid = [&](unsigned i, unsigned j, unsigned k) { return (((i << lg) | j) << lg) | k; };
  for (unsigned t = blockIdx.x * blockDim.x + threadIdx.x; t < np; t += gridDim.x * blockDim.x) {
    const unsigned q = 2 * t;
    const unsigned k = q & m, j = (q >> lg) & m, i = q >> (2 * lg);
    const unsigned pq[4] = {cid((i + 1) & m, j, k), cid((i - 1) & m, j, k), cid(i, (j + 1) & m, k),
                            cid(i, (j - 1) & m, k)};
    const unsigned qm = cid(i, j, (k - 1) & m), qp = cid(i, j, (k + 2) & m);
    const ff2 pc = ff2_pair(psi, q), ec = ff2_pair(E, q);
    // the six neighbour pairs (i+1, i-1, j+1, j-1, k+1, k-1) of psi and of e^psi
    auto nbr = [&](const float2* __restrict__ a, const ff2& own, int d) -> ff2 {
      if (d < 4) return ff2_pair(a, pq[d]);
      if (d == 4) {
        const float2 v = a[qp];
        return ff2{make_float2(own.hi.y, v.x), make_float2(own.lo.y, v.y)};
      }
      const float2 v = a[qm];
      return ff2{make_float2(v.x, own.hi.x), make_float2(v.y, own.lo.x)};
    };
    // sd = sum dp, se = sum e^psi_nb dp with dp = psi_nb - psi: every high part goes through an exact two-sum
    // (or two-product), the low parts and rounding errors are summed in FP32, and each sum is normalised once
    // at the end.  Absolute accuracy about 2^-48 of the terms, as the residual needs (its terms cancel).
    ff2 sd = {f2_bc(0.f), f2_bc(0.f)}, se = sd;
#pragma unroll
    for (int d = 0; d < 6; ++d) {
      const ff2 pn = nbr(psi, pc, d), en = nbr(E, ec, d);
      ff2 dp = ff2_two_sum(pn.hi, make_float2(-pc.hi.x, -pc.hi.y));
      dp.lo = f2_add(dp.lo, f2_sub(pn.lo, pc.lo));
      const ff2 ts = ff2_two_sum(sd.hi, dp.hi);
      sd = {ts.hi, f2_add(f2_add(sd.lo, dp.lo), ts.lo)};
      ff2 pr = ff2_two_prod(en.hi, dp.hi);
      pr.lo = f2_fma(en.hi, dp.lo, f2_fma(en.lo, dp.hi, pr.lo));
      const ff2 te = ff2_two_sum(se.hi, pr.hi);
      se = {te.hi, f2_add(f2_add(se.lo, pr.lo), te.lo)};
    }
    sd = ff2_quick_two_sum(sd.hi, sd.lo);
    se = ff2_quick_two_sum(se.hi, se.lo);
    ff2 flux = ff2_add_abs(ff2_mul(ec, sd), se);
    flux = {f2_mul(f2_bc(0.5f), flux.hi), f2_mul(f2_bc(0.5f), flux.lo)};
    ff2 em = ff2_add_f(exp_ff2(ff2_mul(pc, minv), stab, c.ek), f2_bc(-1.0f));
    if (!(fabsf(pc.hi.x) < 20.0f)) {
      const ff v = ff_from_double(expm1(-((double)pc.hi.x + (double)pc.lo.x) * c.inv_np1));
      em.hi.x = v.hi;
      em.lo.x = v.lo;
    }
    if (!(fabsf(pc.hi.y) < 20.0f)) {
      const ff v = ff_from_double(expm1(-((double)pc.hi.y + (double)pc.lo.y) * c.inv_np1));
      em.hi.y = v.hi;
      em.lo.y = v.lo;
    }
    const ff2 et = ff2_pack(ff_split_bits(eta[q]), ff_split_bits(eta[q + 1]));  // the caller's array
    // S and F = flux C - S by Dekker's addition (absolute accuracy: F is small against its terms)
    ff2 S = ff2_add_abs(ff2_mul(K1, ff2_add_f(et, f2_bc(-1.0f))), ff2_neg(ff2_mul(Kx, em)));
    S = ff2_add_f(S, f2_bc(c.dK));
    const ff2 F = ff2_add_abs(ff2_mul(flux, Cih2), ff2_neg(S));
    const float2 r = f2_add(F.hi, F.lo);
    // the base field of the correction cycles: u = psi + ub to FP32 (within an FP32 ulp of u; the cycles'
    // linearisation point, not part of the residual)
    const float2 B = f2_add(f2_add(pc.hi, f2_bc(ub.x)), f2_add(pc.lo, f2_bc(ub.y)));
    // cell k has colour (i + j + k) & 1, cell k + 1 the other; both at place q / 2 of their half
    const unsigned o0 = (((i + j) & 1u) ? half : 0u) + t, o1 = (((i + j) & 1u) ? 0u : half) + t;
    r32[o0] = -r.x;
    r32[o1] = -r.y;
    B32[o0] = B.x;
    B32[o1] = B.y;
    if (phi_out) write_f64_pair(phi_out, q, pc, base, 1);  // u = u_bar + psi
    acc = fmaf(F.hi.x, F.hi.x, acc);
    acc = fmaf(F.hi.y, F.hi.y, acc);
  }
  block_sum_store<double>((double)acc, part);
}

}  // namespace isis
