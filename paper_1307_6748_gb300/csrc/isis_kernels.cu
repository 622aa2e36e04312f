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
__global__ void update_phi64(double* __restrict__ phi, const float* __restrict__ e, int lg) {
  size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= ((size_t)1 << (3 * lg))) return;
  const int m = (1 << lg) - 1;
  phi[t] += (double)e[lidx<float>(lg, (int)(t >> (2 * lg)), (int)((t >> lg) & m), (int)(t & m))];
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

__global__ void selftest_exp_ff(const double* __restrict__ x, double* __restrict__ y, int n,
                                const float2* __restrict__ tab, FFExp ek) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n) return;
  const ff v = exp_ff(ff_from_double(x[t]), tab, ek);
  y[t] = (double)v.hi + (double)v.lo;
}

__global__ void fofr_prep_ff(const double* __restrict__ u, float2* __restrict__ psi, float2* __restrict__ E,
                             size_t n, float2 ubff, const float2* __restrict__ tab, FFExp ek) {
  size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n) return;
  const ff p = ff_sub(ff_split_bits(u[t]), ff_load(ubff));
  psi[t] = ff_store(p);
  // exp_ff covers |psi| < 22; beyond (no physical field gets there) the FP64 library exp
  E[t] = ff_store(fabsf(p.hi) < 20.0f ? exp_ff(p, tab, ek) : ff_from_double(exp((double)p.hi + (double)p.lo)));
}

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
  const size_t n = (size_t)1 << (3 * lg);
  const int N = 1 << lg, m = N - 1;
  const ff Cih2 = ff_load(c.Cih2), K1 = ff_load(c.K1), Kx = ff_load(c.Kx), minv = ff_load(c.minv);
  float acc = 0.f;
  for (size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (size_t)gridDim.x * blockDim.x) {
    int k = (int)(t & m), j = (int)((t >> lg) & m), i = (int)(t >> (2 * lg));
    size_t nb[6] = {cidx(lg, (i + 1) & m, j, k), cidx(lg, (i - 1) & m, j, k), cidx(lg, i, (j + 1) & m, k),
                    cidx(lg, i, (j - 1) & m, k), cidx(lg, i, j, (k + 1) & m), cidx(lg, i, j, (k - 1) & m)};
    const ff pc = ff_load(psi[t]), ec = ff_load(E[t]);
    ff sd = {0.f, 0.f}, se = {0.f, 0.f};
#pragma unroll
    for (int d = 0; d < 6; ++d) {
      const ff dp = ff_add_abs(ff_load(psi[nb[d]]), ff_neg(pc));
      sd = ff_add_abs(sd, dp);
      se = ff_add_abs(se, ff_mul(ff_load(E[nb[d]]), dp));
    }
    ff flux = ff_add(ff_mul(ec, sd), se);
    flux = {0.5f * flux.hi, 0.5f * flux.lo};
    const ff em = fabsf(pc.hi) < 20.0f
                      ? ff_add_f(exp_ff(ff_mul(pc, minv), stab, c.ek), -1.0f)
                      : ff_from_double(expm1(-((double)pc.hi + (double)pc.lo) * c.inv_np1));
    ff S = ff_sub(ff_mul(K1, ff_add_f(ff_split_bits(eta[t]), -1.0f)), ff_mul(Kx, em));
    S = ff_add_f(S, c.dK);
    const ff F = ff_sub(ff_mul(flux, Cih2), S);
    const size_t o = lidx<float>(lg, i, j, k);
    r32[o] = -(F.hi + F.lo);
    B32[o] = ff_add(pc, ff_load(c.ubff)).hi;  // fp32(u), u = psi + ub
    acc = fmaf(F.hi, F.hi, acc);
  }
  block_sum_store<double>((double)acc, part);
}

}  // namespace isis
