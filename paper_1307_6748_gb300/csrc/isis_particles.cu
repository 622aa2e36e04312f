// isis_particles.cu -- CIC density estimate (Sect. 5.1) and the forces on
// particles (Sect. 4.1 Eq. (symmetron_geodesics_tilde_chi), Sect. 4.2).
//
// CIC convention (not fixed by the paper): positions in cell units, cell
// centres at i + 1/2; along each axis a particle at x gives weight 1 - t to
// cell floor(x - 1/2) and t to the next cell, t = (x - 1/2) - floor(x - 1/2);
// periodic wrap.  The 3-D weight is the product of the three.
#include <cmath>

#include "isis_solver.cuh"

namespace isis {

unsigned long long* get_deposit_buf(int N);

constexpr double kFix = 1099511627776.0;  // 2^40 fixed-point units per unit weight

struct Axis {
  int i0, i1;
  double w0, w1;
};

__device__ __forceinline__ Axis cic_axis(float xf, int N) {
  double xs = (double)xf - 0.5;
  double f = floor(xs);
  double t = xs - f;
  // wrap floor(x - 1/2) into [0, N) without integer overflow for far-away x
  double fw = f - (double)N * floor(f / (double)N);
  int i0 = (int)fw;
  i0 = i0 < 0 ? 0 : (i0 >= N ? N - 1 : i0);
  Axis a;
  a.i0 = i0;
  a.i1 = (i0 + 1) & (N - 1);
  a.w0 = 1.0 - t;
  a.w1 = t;
  return a;
}

__global__ void cic_scatter(const float* __restrict__ x, const float* __restrict__ y, const float* __restrict__ z,
                            long long np, int lg, unsigned long long* __restrict__ acc) {
  long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= np) return;
  const int N = 1 << lg;
  Axis ax = cic_axis(x[p], N), ay = cic_axis(y[p], N), az = cic_axis(z[p], N);
  const int ii[2] = {ax.i0, ax.i1}, jj[2] = {ay.i0, ay.i1}, kk[2] = {az.i0, az.i1};
  const double wi[2] = {ax.w0, ax.w1}, wj[2] = {ay.w0, ay.w1}, wk[2] = {az.w0, az.w1};
#pragma unroll
  for (int a = 0; a < 2; ++a)
#pragma unroll
    for (int b = 0; b < 2; ++b)
#pragma unroll
      for (int d = 0; d < 2; ++d) {
        double w = wi[a] * wj[b] * wk[d];
        unsigned long long q = (unsigned long long)llrint(w * kFix);
        if (q) atomicAdd(&acc[cidx(lg, ii[a], jj[b], kk[d])], q);
      }
}

template <class T>
__global__ void cic_finish(const unsigned long long* __restrict__ acc, T* __restrict__ eta, size_t n, double scale) {
  size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t < n) eta[t] = (T)((double)acc[t] * scale);
}

// Per-particle acceleration.  Grid force at cell c along axis d:
//   f_d(c) = a^2 D_d Phi(c) + pref(c) D_d phi(c),  D_d f(c) = (f(c+e_d) - f(c-e_d)) / (2h)
//   pref = C_s a^2 chi(c) (symmetron), e^u(c)/2 (f(R)), 0 (no scalar field)
// then g = -sum_cells W f.
template <class T, int MODEL>
__global__ void force_gather(const T* __restrict__ Phi, const T* __restrict__ phi, const float* __restrict__ x,
                             const float* __restrict__ y, const float* __restrict__ z, long long np, int lg,
                             double a2, double Cs, double inv2h, float* __restrict__ gx, float* __restrict__ gy,
                             float* __restrict__ gz) {
  long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= np) return;
  const int N = 1 << lg, m = N - 1;
  Axis ax = cic_axis(x[p], N), ay = cic_axis(y[p], N), az = cic_axis(z[p], N);
  const int ii[2] = {ax.i0, ax.i1}, jj[2] = {ay.i0, ay.i1}, kk[2] = {az.i0, az.i1};
  const double wi[2] = {ax.w0, ax.w1}, wj[2] = {ay.w0, ay.w1}, wk[2] = {az.w0, az.w1};
  double acc[3] = {0.0, 0.0, 0.0};
#pragma unroll
  for (int a = 0; a < 2; ++a)
#pragma unroll
    for (int b = 0; b < 2; ++b)
#pragma unroll
      for (int d = 0; d < 2; ++d) {
        const int i = ii[a], j = jj[b], k = kk[d];
        const double w = wi[a] * wj[b] * wk[d];
        const size_t xp = cidx(lg, (i + 1) & m, j, k), xm = cidx(lg, (i - 1) & m, j, k);
        const size_t yp = cidx(lg, i, (j + 1) & m, k), ym = cidx(lg, i, (j - 1) & m, k);
        const size_t zp = cidx(lg, i, j, (k + 1) & m), zm = cidx(lg, i, j, (k - 1) & m);
        double f0 = 0.0, f1 = 0.0, f2 = 0.0;
        if (Phi) {
          f0 = a2 * ((double)Phi[xp] - (double)Phi[xm]);
          f1 = a2 * ((double)Phi[yp] - (double)Phi[ym]);
          f2 = a2 * ((double)Phi[zp] - (double)Phi[zm]);
        }
        if (MODEL != 0) {
          double v = (double)phi[cidx(lg, i, j, k)];
          double pref = (MODEL == ISIS_SYMMETRON) ? Cs * a2 * v : 0.5 * exp(v);
          f0 += pref * ((double)phi[xp] - (double)phi[xm]);
          f1 += pref * ((double)phi[yp] - (double)phi[ym]);
          f2 += pref * ((double)phi[zp] - (double)phi[zm]);
        }
        acc[0] += w * f0;
        acc[1] += w * f1;
        acc[2] += w * f2;
      }
  gx[p] = (float)(-acc[0] * inv2h);
  gy[p] = (float)(-acc[1] * inv2h);
  gz[p] = (float)(-acc[2] * inv2h);
}

static bool grid_valid(const isis_grid* g) {
  return g && g->N >= 8 && g->N <= 1024 && (g->N & (g->N - 1)) == 0 && g->box > 0;
}

}  // namespace isis

using namespace isis;

extern "C" {

isis_status isis_cic_deposit(const isis_grid* grid, const float* x, const float* y, const float* z, int64_t npart,
                             void* eta, int eta_f64, void* stream) {
  if (!grid_valid(grid) || !x || !y || !z || !eta || npart < 1 || npart > ((int64_t)1 << 40)) return ISIS_EINVAL;
  const int N = grid->N, lg = ilog2(N);
  const size_t n = (size_t)N * N * N;
  cudaStream_t st = (cudaStream_t)stream;
  unsigned long long* acc = get_deposit_buf(N);
  if (!acc) return ISIS_ENOMEM;
  ISIS_CK(cudaMemsetAsync(acc, 0, n * sizeof(unsigned long long), st));
  ISIS_LAUNCH(KK_CIC_SCATTER, 12.0 * npart + 8.0 * n, st,
              (cic_scatter<<<nblk((size_t)npart, 256), 256, 0, st>>>(x, y, z, (long long)npart, lg, acc)));
  const double scale = (double)n / ((double)npart * kFix);
  if (eta_f64)
    ISIS_LAUNCH(KK_CIC_FINISH, 16.0 * n, st,
                (cic_finish<double><<<nblk(n, 256), 256, 0, st>>>(acc, (double*)eta, n, scale)));
  else
    ISIS_LAUNCH(KK_CIC_FINISH, 12.0 * n, st,
                (cic_finish<float><<<nblk(n, 256), 256, 0, st>>>(acc, (float*)eta, n, scale)));
  return ISIS_OK;
}

isis_status isis_fifth_force(isis_model model, const isis_params* p, const isis_grid* grid, double a,
                             const void* Phi, const void* phi, int fields_f64, const float* x, const float* y,
                             const float* z, int64_t npart, float* gx, float* gy, float* gz, void* stream) {
  if (!grid_valid(grid) || !x || !y || !z || !gx || !gy || !gz || npart < 1 || !(a > 0)) return ISIS_EINVAL;
  if (phi && (!p || (model != ISIS_SYMMETRON && model != ISIS_FOFR_HS))) return ISIS_EINVAL;
  if (phi && model == ISIS_SYMMETRON && !(p->a_ssb > 0)) return ISIS_EINVAL;
  const int lg = ilog2(grid->N);
  const double h = grid->box / grid->N;
  const double inv2h = 1.0 / (2.0 * h), a2 = a * a;
  double Cs = 0.0;
  if (phi && model == ISIS_SYMMETRON)  // Eq. (symmetron_geodesics_tilde_chi)
    Cs = 6.0 * grid->Omega_m * grid->H0 * grid->H0 * (p->beta * p->lambda0) * (p->beta * p->lambda0) /
         (p->a_ssb * p->a_ssb * p->a_ssb);
  cudaStream_t st = (cudaStream_t)stream;
  unsigned nb = nblk((size_t)npart, 256);
  int mcode = phi ? (int)model : 0;
  const double fbytes = 24.0 * npart + (double)grid->N * grid->N * grid->N * (fields_f64 ? 8 : 4) *
                                             ((Phi ? 1 : 0) + (phi ? 1 : 0));
#define ISIS_FORCE(T, MC)                                                                                    \
  ISIS_LAUNCH(KK_FORCE, fbytes, st,                                                                          \
              (force_gather<T, MC><<<nb, 256, 0, st>>>((const T*)Phi, (const T*)phi, x, y, z, (long long)npart, \
                                                       lg, a2, Cs, inv2h, gx, gy, gz)))
  if (fields_f64) {
    if (mcode == 0) ISIS_FORCE(double, 0);
    else if (mcode == ISIS_SYMMETRON) ISIS_FORCE(double, ISIS_SYMMETRON);
    else ISIS_FORCE(double, ISIS_FOFR_HS);
  } else {
    if (mcode == 0) ISIS_FORCE(float, 0);
    else if (mcode == ISIS_SYMMETRON) ISIS_FORCE(float, ISIS_SYMMETRON);
    else ISIS_FORCE(float, ISIS_FOFR_HS);
  }
#undef ISIS_FORCE
  return ISIS_OK;
}

}  // extern "C"
