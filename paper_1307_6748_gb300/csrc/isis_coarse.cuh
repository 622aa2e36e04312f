// isis_coarse.cuh -- coarsest-grid solve of the FAS hierarchy: Newton's
// method on F(x) = L(x) - Sigma with the exact (dense) Jacobian, LU with
// partial pivoting in shared memory, FP64 arithmetic whatever the storage
// type.  One CTA of 64 threads, at most 64 unknowns (4^3 grid).
//
// Stop rule: after a step dx, stop when max|dx| <= 1e-13 max(1, max|x|), at
// most 50 steps (the paper does not describe its coarsest solve).  Poisson:
// the Jacobian is made regular as J - (6/h^2) 1 1^T / n and the step is
// projected to zero mean, so the coarse solve never shifts the mean.
#pragma once
#include "isis_kernels.cuh"

namespace isis {

constexpr int kCoarseMax = 64;

// status bits written to *flags (OR-ed): 1 = singular pivot, 2 = non-finite step, 4 = no step met the stop
// rule within the 50 steps
template <Model M, Form FM, class T>
__global__ void __launch_bounds__(kCoarseMax) coarse_newton(LevelView<T> L, Coef c, int* flags, int* steps_max) {
  __shared__ double J[kCoarseMax][kCoarseMax + 1];
  __shared__ double b[kCoarseMax], xs[kCoarseMax], Bs[kCoarseMax], ws[kCoarseMax];
  __shared__ double etas[kCoarseMax], sigs[kCoarseMax];
  __shared__ double wmax[2];
  __shared__ int wpiv[2];
  __shared__ int done, bad;
  const int n = 1 << (3 * L.lg), N = L.N, lg = L.lg, r = threadIdx.x;
  const double ih2 = (double)L.ih2;
  int i = r >> (2 * lg), j = (r >> lg) & (N - 1), k = r & (N - 1);
  const size_t gr = r < n ? lidx<T>(lg, i, j, k) : 0;  // storage index of unknown r
  if (r < n) {
    xs[r] = (double)L.x[gr];
    etas[r] = uses_eta<M, FM>() ? (double)L.eta[gr] : 0.0;
    sigs[r] = L.sig ? (double)L.sig[gr] : 0.0;
    Bs[r] = (FM == DELTA && M != POI) ? (double)L.B[gr] : 0.0;
    ws[r] = (FM == DELTA && M == FOFR) ? (double)dexp<T>(L.B[gr]) : 0.0;  // e^B as the grids' kernels evaluate it
  }
  if (r == 0) { done = 0; bad = 0; }
  __syncthreads();
  int nb[6];
  if (r < n) {
    nb[0] = (((i + 1) & (N - 1)) << (2 * lg)) | (j << lg) | k;
    nb[1] = (((i - 1) & (N - 1)) << (2 * lg)) | (j << lg) | k;
    nb[2] = (i << (2 * lg)) | (((j + 1) & (N - 1)) << lg) | k;
    nb[3] = (i << (2 * lg)) | (((j - 1) & (N - 1)) << lg) | k;
    nb[4] = (i << (2 * lg)) | (j << lg) | ((k + 1) & (N - 1));
    nb[5] = (i << (2 * lg)) | (j << lg) | ((k - 1) & (N - 1));
  }
  int it = 0;
  for (; it < 50; ++it) {
    // Jacobian row r and right-hand side -F_r
    if (r < n) {
      Cell<double> q;
      q.x = xs[r]; q.eta = etas[r]; q.sig = sigs[r]; q.B = Bs[r]; q.w = ws[r];
#pragma unroll
      for (int d = 0; d < 6; ++d) { q.xn[d] = xs[nb[d]]; q.Bn[d] = Bs[nb[d]]; q.wn[d] = ws[nb[d]]; }
      q.a = aux_of<M, FM, double>(q.x, q.w);
#pragma unroll
      for (int d = 0; d < 6; ++d) q.an[d] = aux_of<M, FM, double>(q.xn[d], q.wn[d]);
      double F, dF;
      eval_cell<M, FM, double>(c, ih2, q, F, dF);
      double shift = (M == POI) ? 6.0 * ih2 / (double)n : 0.0;
      for (int cc = 0; cc < n; ++cc) J[r][cc] = -shift;
      J[r][r] += dF;
#pragma unroll
      for (int d = 0; d < 6; ++d) J[r][nb[d]] += eval_offdiag<M, FM>(c, ih2, q, d);
      b[r] = -F;
    }
    __syncthreads();
    // LU with partial pivoting; the pivot is the first largest |J[p][kk]|, p >= kk
    for (int kk = 0; kk < n; ++kk) {
      double v = (r >= kk && r < n) ? fabs(J[r][kk]) : -1.0;
      int p = r;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        double v2 = __shfl_down_sync(0xffffffffu, v, o);
        int p2 = __shfl_down_sync(0xffffffffu, p, o);
        if (v2 > v || (v2 == v && p2 < p)) { v = v2; p = p2; }
      }
      if ((r & 31) == 0) { wmax[r >> 5] = v; wpiv[r >> 5] = p; }
      __syncthreads();
      int piv = wpiv[0];
      double best = wmax[0];
      if (n > 32 && (wmax[1] > best)) { best = wmax[1]; piv = wpiv[1]; }
      if (!(best > 0.0)) {
        if (r == 0) bad |= 1;
        __syncthreads();
        break;
      }
      if (piv != kk && r < n) {
        double t = J[kk][r]; J[kk][r] = J[piv][r]; J[piv][r] = t;
        if (r == 0) { double tb = b[kk]; b[kk] = b[piv]; b[piv] = tb; }
      }
      __syncthreads();
      if (r > kk && r < n) {
        double m = J[r][kk] / J[kk][kk];
        J[r][kk] = m;
        for (int cc = kk + 1; cc < n; ++cc) J[r][cc] -= m * J[kk][cc];
        b[r] -= m * b[kk];
      }
      __syncthreads();
    }
    if (bad) break;
    if (r == 0) {
      for (int rr = n - 1; rr >= 0; --rr) {
        double s = b[rr];
        for (int cc = rr + 1; cc < n; ++cc) s -= J[rr][cc] * b[cc];
        b[rr] = s / J[rr][rr];
      }
      if (M == POI) {
        double m = 0.0;
        for (int rr = 0; rr < n; ++rr) m += b[rr];
        m /= (double)n;
        for (int rr = 0; rr < n; ++rr) b[rr] -= m;
      }
      double dmax = 0.0, xmax = 0.0;
      for (int rr = 0; rr < n; ++rr) {
        xs[rr] += b[rr];
        dmax = fmax(dmax, fabs(b[rr]));
        xmax = fmax(xmax, fabs(xs[rr]));
      }
      if (!isfinite(dmax) || !isfinite(xmax)) bad |= 2;
      else if (dmax <= 1e-13 * fmax(1.0, xmax)) done = 1;
    }
    __syncthreads();
    if (done || bad) { ++it; break; }
  }
  if (r < n) {
    L.x[gr] = (T)xs[r];
    if constexpr (M == FOFR && kExpCache<T>) L.aux[gr] = aux_of<M, FM, T>((T)xs[r], T(0));
  }
  if (r == 0) {
    const int f = bad ? bad : (done ? 0 : 4);
    if (f) atomicOr(flags, f);
    atomicMax(steps_max, it);
  }
}

}  // namespace isis
