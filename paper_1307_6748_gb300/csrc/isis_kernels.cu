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

__global__ void rb_to_ff(const float* __restrict__ psi, float2* __restrict__ pff, int lg, float2 shift) {
  const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= ((size_t)1 << (3 * lg))) return;
  const int m = (1 << lg) - 1;
  const float v = psi[lidx<float>(lg, (int)(t >> (2 * lg)), (int)((t >> lg) & m), (int)(t & m))];
  pff[t] = ff_store(ff_add_f(ff_load(shift), v));
}

__global__ void update_ff(float2* __restrict__ pff, const float* __restrict__ e, int lg,
                          const float* __restrict__ emean) {
  const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= ((size_t)1 << (3 * lg))) return;
  const int m = (1 << lg) - 1;
  float v = e[lidx<float>(lg, (int)(t >> (2 * lg)), (int)((t >> lg) & m), (int)(t & m))];
  if (emean) v -= *emean;  // Poisson: the correction's mean removed (in FP32, as e is)
  pff[t] = ff_store(ff_add_f(ff_load(pff[t]), v));
}

__global__ void ff_to_f64(const float2* __restrict__ pff, double* __restrict__ phi, size_t n, double base) {
  const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n) return;
  const float2 v = pff[t];
  const double d = f2d_bits(v.x) + f2d_bits(v.y);  // the float-float value (one rounding at most)
  phi[t] = base != 0.0 ? base + d : d;
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
  const size_t n = (size_t)1 << (3 * lg);
  const int m = (1 << lg) - 1;
  ff s1 = {0.f, 0.f};
  float s2 = 0.f;
  for (size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (size_t)gridDim.x * blockDim.x) {
    const ff x = ff_split_bits(v[t]);
    s1 = ff_add(s1, x);
    const float d = ff_add_f(x, -1.0f).hi;
    s2 = fmaf(d, d, s2);
    rb[lidx<float>(lg, (int)(t >> (2 * lg)), (int)((t >> lg) & m), (int)(t & m))] = x.hi;
  }
  block_sum_store<double>((double)s2, part2);
  __syncthreads();
  block_sum_store<double>((double)s1.hi + (double)s1.lo, part1);
}

__global__ void __launch_bounds__(kNormThreads) sum_f32_partial(const float* __restrict__ v, size_t n,
                                                                double* __restrict__ part) {
  ff s = {0.f, 0.f};
  for (size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (size_t)gridDim.x * blockDim.x)
    s = ff_add_f(s, v[t]);
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
                                                                       double* __restrict__ part) {
  __shared__ float2 stab[64];
  if (threadIdx.x < 64) stab[threadIdx.x] = tab[threadIdx.x];
  __syncthreads();
  const size_t np = (size_t)1 << (3 * lg - 1), half = np;
  const int m = (1 << lg) - 1;
  const ff2 Cih2 = ff2_bc(c.Cih2), K1 = ff2_bc(c.K1), Kx = ff2_bc(c.Kx), minv = ff2_bc(c.minv);
  float acc = 0.f;
  for (size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x; t < np; t += (size_t)gridDim.x * blockDim.x) {
    const size_t q = 2 * t;
    const int k = (int)(q & m), j = (int)((q >> lg) & m), i = (int)(q >> (2 * lg));
    const size_t pq[4] = {cidx(lg, (i + 1) & m, j, k), cidx(lg, (i - 1) & m, j, k), cidx(lg, i, (j + 1) & m, k),
                          cidx(lg, i, (j - 1) & m, k)};
    const size_t qm = cidx(lg, i, j, (k - 1) & m), qp = cidx(lg, i, j, (k + 2) & m);
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
    ff2 sd = {f2_bc(0.f), f2_bc(0.f)}, se = sd;
#pragma unroll
    for (int d = 0; d < 6; ++d) {
      const ff2 dp = ff2_add_abs(nbr(psi, pc, d), ff2_neg(pc));
      sd = ff2_add_abs(sd, dp);
      se = ff2_add_abs(se, ff2_mul(nbr(E, ec, d), dp));
    }
    ff2 flux = ff2_add(ff2_mul(ec, sd), se);
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
    ff2 S = ff2_sub(ff2_mul(K1, ff2_add_f(et, f2_bc(-1.0f))), ff2_mul(Kx, em));
    S = ff2_add_f(S, f2_bc(c.dK));
    const ff2 F = ff2_sub(ff2_mul(flux, Cih2), S);
    const float2 r = f2_add(F.hi, F.lo);
    const float2 B = ff2_add(pc, ff2_bc(c.ubff)).hi;  // fp32(u), u = psi + ub
    // cell k has colour (i + j + k) & 1, cell k + 1 the other; both at place q / 2 of their half
    const size_t o0 = (((size_t)(i + j) & 1u) ? half : 0) + t, o1 = (((size_t)(i + j) & 1u) ? 0 : half) + t;
    r32[o0] = -r.x;
    r32[o1] = -r.y;
    B32[o0] = B.x;
    B32[o1] = B.y;
    acc = fmaf(F.hi.x, F.hi.x, acc);
    acc = fmaf(F.hi.y, F.hi.y, acc);
  }
  block_sum_store<double>((double)acc, part);
}

}  // namespace isis
