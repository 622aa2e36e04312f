// isis_kernels.cu -- non-templated kernels shared by the solver instantiations.
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

__global__ void fofr_prep64(const double* __restrict__ u, const double* __restrict__ eta, double* __restrict__ b,
                            double* __restrict__ S, size_t n, Coef c, const double* __restrict__ tab) {
  size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n) return;
  double v = u[t];
  b[t] = exp_tang(v, tab);
  S[t] = fma(c.K1, eta[t] - 1.0, c.K3) - c.K2 * exp_tang(-v * c.inv_np1, tab);
}

__global__ void __launch_bounds__(kNormThreads) outer_residual_fofr(int lg, double ih2, const double* __restrict__ u,
                                                                    const double* __restrict__ b,
                                                                    const double* __restrict__ S,
                                                                    float* __restrict__ r32, float* __restrict__ B32,
                                                                    double* __restrict__ part) {
  const size_t n = (size_t)1 << (3 * lg);
  const int N = 1 << lg, m = N - 1;
  double acc = 0.0;
  for (size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (size_t)gridDim.x * blockDim.x) {
    int k = (int)(t & m), j = (int)((t >> lg) & m), i = (int)(t >> (2 * lg));
    size_t nb[6] = {cidx(lg, (i + 1) & m, j, k), cidx(lg, (i - 1) & m, j, k), cidx(lg, i, (j + 1) & m, k),
                    cidx(lg, i, (j - 1) & m, k), cidx(lg, i, j, (k + 1) & m), cidx(lg, i, j, (k - 1) & m)};
    double uc = u[t], bc = b[t];
    double su = 0.0, sb = 0.0, sbu = 0.0;
#pragma unroll
    for (int d = 0; d < 6; ++d) {
      double un = u[nb[d]], bn = b[nb[d]];
      su += un;
      sb += bn;
      sbu = fma(bn, un, sbu);
    }
    double flux = 0.5 * fma(bc, fma(-6.0, uc, su), fma(-uc, sb, sbu));
    double F = fma(flux, ih2, -S[t]);
    const size_t o = lidx<float>(lg, i, j, k);
    r32[o] = (float)(-F);
    B32[o] = (float)uc;
    acc = fma(F, F, acc);
  }
  block_sum_store<double>(acc, part);
}

void exp_table_fill(double* host256) {
  for (int j = 0; j < 256; ++j) host256[j] = (double)exp2l((long double)j / 256.0L);
}

}  // namespace isis
