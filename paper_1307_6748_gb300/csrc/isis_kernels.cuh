// isis_kernels.cuh -- CUDA kernels of the FAS multigrid solve on a periodic
// N^3 grid (N = 2^lg), cell (i,j,k) stored at ((i*N)+j)*N+k.
//
//   smooth_color      one colour of a red-black Newton-Gauss-Seidel sweep (Sect. 3.2)
//   resid_restrict    r = Sigma - L(x); x_H = R x, x0_H = x_H, Sigma_H = R r (Sect. 3.2)
//   coarse_sigma_add  Sigma_H += L_H(x_H)
//   prolong_correct   x_h += P(x_H - x0_H)
//   coarse_newton     dense Newton with the exact Jacobian on the coarsest grid
//   norm_partial      deterministic per-block sums of (L(x) - Sigma)^2
//
// R = mean of the 8 children; P = cell-centred trilinear interpolation
// (weights 3/4 and 1/4 per axis).  The paper leaves both unspecified.
#pragma once
#include "isis_model.cuh"

namespace isis {

constexpr int kNormBlocks = 1216;  // 8 blocks per SM on a 152-SM part; fixed for reproducible sums
constexpr int kNormThreads = 256;

template <class T>
struct LevelView {
  int N, lg;
  T ih2;           // 1/h^2
  T* x;            // unknown
  const T* eta;    // density
  const T* sig;    // FAS source, nullptr means 0
  const T* B;      // DELTA form base field
  const T* w;      // e^B (f(R) DELTA form)
};

__device__ __forceinline__ size_t cidx(int lg, int i, int j, int k) {
  return ((((size_t)i << lg) + (size_t)j) << lg) + (size_t)k;
}

// Gather one cell and its neighbours from global memory (periodic wrap).
template <Model M, Form FM, class T>
__device__ __forceinline__ Cell<T> gather(const LevelView<T>& L, int i, int j, int k) {
  const int m = L.N - 1;
  size_t c = cidx(L.lg, i, j, k);
  size_t nb[6] = {cidx(L.lg, (i + 1) & m, j, k), cidx(L.lg, (i - 1) & m, j, k), cidx(L.lg, i, (j + 1) & m, k),
                  cidx(L.lg, i, (j - 1) & m, k), cidx(L.lg, i, j, (k + 1) & m), cidx(L.lg, i, j, (k - 1) & m)};
  Cell<T> q;
  q.x = L.x[c];
#pragma unroll
  for (int d = 0; d < 6; ++d) q.xn[d] = L.x[nb[d]];
  q.sig = L.sig ? L.sig[c] : T(0);
  if constexpr (!(M == POI && FM == DELTA)) q.eta = L.eta[c]; else q.eta = T(0);
  if constexpr (FM == DELTA && M != POI) q.B = L.B[c]; else q.B = T(0);
  if constexpr (FM == DELTA && M == FOFR) {
    q.w = L.w[c];
#pragma unroll
    for (int d = 0; d < 6; ++d) { q.Bn[d] = L.B[nb[d]]; q.wn[d] = L.w[nb[d]]; }
  }
  return q;
}

// One colour (0 = red: (i+j+k) even) of a Newton-Gauss-Seidel sweep, in place.
// Thread layout: one thread per pair of cells (k = 2p, 2p+1); it updates the
// member of the pair that has the requested colour.
template <Model M, Form FM, class T>
__global__ void smooth_color(LevelView<T> L, Coef c, int color) {
  size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  size_t half = (size_t)1 << (3 * L.lg - 1);
  if (t >= half) return;
  int k2 = (int)(t & ((L.N >> 1) - 1));
  int j = (int)((t >> (L.lg - 1)) & (L.N - 1));
  int i = (int)(t >> (2 * L.lg - 1));
  int k = 2 * k2 + ((i + j + color) & 1);
  Cell<T> q = gather<M, FM, T>(L, i, j, k);
  T F, dF;
  eval_cell<M, FM, T>(c, L.ih2, q, F, dF);
  L.x[cidx(L.lg, i, j, k)] = q.x - F / dF;
}

// One thread per coarse cell: residuals of its 8 children, their means.
template <Model M, Form FM, class T>
__global__ void resid_restrict(LevelView<T> F, Coef c, T* __restrict__ xc, T* __restrict__ x0c,
                               T* __restrict__ sigc) {
  int lgc = F.lg - 1;
  size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= ((size_t)1 << (3 * lgc))) return;
  int Nc = 1 << lgc;
  int K = (int)(t & (Nc - 1)), J = (int)((t >> lgc) & (Nc - 1)), I = (int)(t >> (2 * lgc));
  T xs = 0, rs = 0;
#pragma unroll
  for (int a = 0; a < 2; ++a)
#pragma unroll
    for (int b = 0; b < 2; ++b)
#pragma unroll
      for (int d = 0; d < 2; ++d) {
        Cell<T> q = gather<M, FM, T>(F, 2 * I + a, 2 * J + b, 2 * K + d);
        T Fv, dF;
        eval_cell<M, FM, T>(c, F.ih2, q, Fv, dF);
        xs += q.x;
        rs -= Fv;  // r = Sigma - L(x)
      }
  xc[t] = xs * T(0.125);
  x0c[t] = xs * T(0.125);
  sigc[t] = rs * T(0.125);
}

// Sigma_H += L_H(x_H) (the FAS coarse source, Sect. 3.2).
template <Model M, Form FM, class T>
__global__ void coarse_sigma_add(LevelView<T> L, Coef c, T* __restrict__ sig) {
  size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= ((size_t)1 << (3 * L.lg))) return;
  int k = (int)(t & (L.N - 1)), j = (int)((t >> L.lg) & (L.N - 1)), i = (int)(t >> (2 * L.lg));
  LevelView<T> L0 = L;
  L0.sig = nullptr;
  Cell<T> q = gather<M, FM, T>(L0, i, j, k);
  T F, dF;
  eval_cell<M, FM, T>(c, L.ih2, q, F, dF);
  sig[t] += F;
}

// x_h += P(x_H - x0_H), one thread per fine cell.
template <class T>
__global__ void prolong_correct(T* __restrict__ xf, const T* __restrict__ xc, const T* __restrict__ x0c, int lgc) {
  int lgf = lgc + 1, Nc = 1 << lgc;
  size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= ((size_t)1 << (3 * lgf))) return;
  int Nf = 1 << lgf;
  int k = (int)(t & (Nf - 1)), j = (int)((t >> lgf) & (Nf - 1)), i = (int)(t >> (2 * lgf));
  int ci[2] = {i >> 1, ((i >> 1) + ((i & 1) ? 1 : -1)) & (Nc - 1)};
  int cj[2] = {j >> 1, ((j >> 1) + ((j & 1) ? 1 : -1)) & (Nc - 1)};
  int ck[2] = {k >> 1, ((k >> 1) + ((k & 1) ? 1 : -1)) & (Nc - 1)};
  const T wt[2] = {T(0.75), T(0.25)};
  T v = 0;
#pragma unroll
  for (int a = 0; a < 2; ++a)
#pragma unroll
    for (int b = 0; b < 2; ++b)
#pragma unroll
      for (int d = 0; d < 2; ++d) {
        size_t q = cidx(lgc, ci[a], cj[b], ck[d]);
        v += wt[a] * wt[b] * wt[d] * (xc[q] - x0c[q]);
      }
  xf[t] += v;
}

// coarse = mean of the 8 children of fine (plain restriction of a field).
template <class Tin, class Tout>
__global__ void restrict_mean(const Tin* __restrict__ f, Tout* __restrict__ c, int lgc) {
  size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= ((size_t)1 << (3 * lgc))) return;
  int Nc = 1 << lgc, lgf = lgc + 1;
  int K = (int)(t & (Nc - 1)), J = (int)((t >> lgc) & (Nc - 1)), I = (int)(t >> (2 * lgc));
  Tin s = 0;
#pragma unroll
  for (int a = 0; a < 2; ++a)
#pragma unroll
    for (int b = 0; b < 2; ++b)
#pragma unroll
      for (int d = 0; d < 2; ++d) s += f[cidx(lgf, 2 * I + a, 2 * J + b, 2 * K + d)];
  c[t] = (Tout)(s * Tin(0.125));
}

// Deterministic block partial sums of (L(x) - Sigma)^2 (fixed grid, fixed
// tree order); finished by reduce_final.
template <class T>
__device__ __forceinline__ void block_sum_store(double v, double* out) {
  __shared__ double red[kNormThreads / 32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x < 32) {
    v = threadIdx.x < kNormThreads / 32 ? red[threadIdx.x] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if (threadIdx.x == 0) out[blockIdx.x] = v;
  }
}

template <Model M, Form FM, class T>
__global__ void __launch_bounds__(kNormThreads) norm_partial(LevelView<T> L, Coef c, double* __restrict__ part) {
  size_t n = (size_t)1 << (3 * L.lg);
  double acc = 0.0;
  for (size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (size_t)gridDim.x * blockDim.x) {
    int k = (int)(t & (L.N - 1)), j = (int)((t >> L.lg) & (L.N - 1)), i = (int)(t >> (2 * L.lg));
    Cell<T> q = gather<M, FM, T>(L, i, j, k);
    T F, dF;
    eval_cell<M, FM, T>(c, L.ih2, q, F, dF);
    acc += (double)F * (double)F;
  }
  block_sum_store<T>(acc, part);
}

// Sum of (v - shift)^2 and of v over an array (for the reference residual
// and the Poisson mean).
template <class T>
__global__ void __launch_bounds__(kNormThreads) moments_partial(const T* __restrict__ v, size_t n, double shift,
                                                                double* __restrict__ part2,
                                                                double* __restrict__ part1) {
  double a2 = 0.0, a1 = 0.0;
  for (size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (size_t)gridDim.x * blockDim.x) {
    double d = (double)v[t] - shift;
    a2 += d * d;
    a1 += (double)v[t];
  }
  block_sum_store<T>(a2, part2);
  __syncthreads();
  block_sum_store<T>(a1, part1);
}

// One block sums nparts partials in a fixed order into *out.
__global__ void reduce_final(const double* __restrict__ part, int nparts, double* __restrict__ out);

}  // namespace isis
