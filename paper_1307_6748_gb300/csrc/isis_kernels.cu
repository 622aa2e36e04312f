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
__global__ void update_phi64(double* __restrict__ phi, const float* __restrict__ e, size_t n) {
  size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t < n) phi[t] += (double)e[t];
}
}  // namespace isis
