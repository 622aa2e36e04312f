// isis_coarse.cuh -- the coarse end of the FAS hierarchy.
//
// coarse_newton: the coarsest-grid solve, Newton's method on F(x) = L(x) - Sigma with the exact (dense)
// Jacobian, LU with partial pivoting in shared memory, FP64 arithmetic whatever the storage type.  One CTA,
// at most 64 unknowns (4^3 grid).
//
// Stop rule: after a step dx, stop when max|dx| <= 1e-13 max(1, max|x|), at most 50 steps (the paper does not
// describe its coarsest solve).  Poisson: the Jacobian is made regular as J - (6/h^2) 1 1^T / n and the step
// is projected to zero mean, so the coarse solve never shifts the mean.
//
// coarse_cycle: every level of a V-cycle from a grid of at most 16^3 down to the coarsest, in one CTA with all
// of its arrays in shared memory (FP32 grids): the smoothing sweeps, residual + restriction, the FAS coarse
// source, the coarsest Newton solve and the prolongation run back to back with block barriers between them,
// where one kernel launch per step would leave the GPU waiting on launch latency.  The same operators and
// transfers as the grid kernels (Sect. 3.2, Sect. 3.3, Sect. 3.4).
#pragma once
#include "isis_kernels.cuh"

namespace isis {

constexpr int kCoarseMax = 64;

// Shared scratch of the dense Newton solve.  LU: the type of the Jacobian, the step and its factorisation; the
// iterate and the residual are FP64 whatever LU is.
template <class LU>
struct NewtonScratchT {
  LU J[kCoarseMax][kCoarseMax + 1];
  LU b[kCoarseMax];
  double xs[kCoarseMax], Bs[kCoarseMax], ws[kCoarseMax], etas[kCoarseMax], sigs[kCoarseMax];
  double as[kCoarseMax];  // f(R): the per-cell exponential of the iterate (aux_of), once per cell and step
  LU wmax[2];
  int wpiv[2];
  int done, bad;
};
using NewtonScratch = NewtonScratchT<double>;

// Dense Newton on the n = N^3 unknowns held in S.xs (with S.etas, S.sigs, S.Bs, S.ws = e^B); every thread of
// the block calls it, threads 0..n-1 own the rows (blockDim.x >= n, at most kCoarseMax rows).  Row-major
// unknown r = (i N + j) N + k.  On return S.xs holds the solution, S.bad the flags 1 (singular pivot) and
// 2 (non-finite step), S.done whether the stop rule was met; the return value is the number of steps.
// LU = float (the FP32 V-cycles): F(x) and x stay FP64, so the stop rule means the same, while the step comes
// from an FP32 factorisation of the FP32-rounded Jacobian.  That makes each step a Newton step with an
// inexact linear solve (the error contracts by about cond(J) 2^-24 per step on top of Newton's quadratic
// rate; an FP64 iterative refinement of the step, in effect) at FP32 instruction cost: FP64 instructions run
// on a narrow pipe on this part, and the FP64 factorisation took about 30 us per step of an 8-unknown
// system in one CTA.
template <Model M, Form FM, class LU = double>
__device__ int dense_newton_block(NewtonScratchT<LU>& S, int lg, double ih2, const Coef& c) {
  const int n = 1 << (3 * lg), N = 1 << lg, r = threadIdx.x;
  const int i = r >> (2 * lg), j = (r >> lg) & (N - 1), k = r & (N - 1);
  if (r == 0) { S.done = 0; S.bad = 0; }
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
    if constexpr (M == FOFR) {  // each cell's exponential once (FP64 exponentials are costly here)
      if (r < n) S.as[r] = aux_of<M, FM, double>(S.xs[r], S.ws[r]);
      __syncthreads();
    }
    // Jacobian row r and right-hand side -F_r
    if (r < n) {
      Cell<double> q;
      q.x = S.xs[r]; q.eta = S.etas[r]; q.sig = S.sigs[r]; q.B = S.Bs[r]; q.w = S.ws[r];
#pragma unroll
      for (int d = 0; d < 6; ++d) { q.xn[d] = S.xs[nb[d]]; q.Bn[d] = S.Bs[nb[d]]; q.wn[d] = S.ws[nb[d]]; }
      if constexpr (M == FOFR) {
        q.a = S.as[r];
#pragma unroll
        for (int d = 0; d < 6; ++d) q.an[d] = S.as[nb[d]];
      } else {
        q.a = 0.0;
#pragma unroll
        for (int d = 0; d < 6; ++d) q.an[d] = 0.0;
      }
      double F, dF;
      eval_cell<M, FM, double>(c, ih2, q, F, dF);
      const double shift = (M == POI) ? 6.0 * ih2 / (double)n : 0.0;
      for (int cc = 0; cc < n; ++cc) S.J[r][cc] = (LU)(-shift);
      S.J[r][r] = (LU)(dF - shift);
#pragma unroll
      for (int d = 0; d < 6; ++d) S.J[r][nb[d]] += (LU)eval_offdiag<M, FM>(c, ih2, q, d);
      S.b[r] = (LU)(-F);
    }
    __syncthreads();
    // LU with partial pivoting; the pivot is the first largest |J[p][kk]|, p >= kk (warps 0 and 1)
    for (int kk = 0; kk < n; ++kk) {
      LU v = (r >= kk && r < n) ? (LU)fabs(S.J[r][kk]) : (LU)(-1);
      int p = r;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        LU v2 = __shfl_down_sync(0xffffffffu, v, o);
        int p2 = __shfl_down_sync(0xffffffffu, p, o);
        if (v2 > v || (v2 == v && p2 < p)) { v = v2; p = p2; }
      }
      if (r < kCoarseMax && (r & 31) == 0) { S.wmax[r >> 5] = v; S.wpiv[r >> 5] = p; }
      __syncthreads();
      int piv = S.wpiv[0];
      LU best = S.wmax[0];
      if (n > 32 && (S.wmax[1] > best)) { best = S.wmax[1]; piv = S.wpiv[1]; }
      if (!(best > (LU)0)) {
        if (r == 0) S.bad |= 1;
        __syncthreads();
        break;
      }
      if (piv != kk && r < n) {
        LU t = S.J[kk][r]; S.J[kk][r] = S.J[piv][r]; S.J[piv][r] = t;
        if (r == 0) { LU tb = S.b[kk]; S.b[kk] = S.b[piv]; S.b[piv] = tb; }
      }
      __syncthreads();
      if (r > kk && r < n) {
        LU m = S.J[r][kk] / S.J[kk][kk];
        S.J[r][kk] = m;
        for (int cc = kk + 1; cc < n; ++cc) S.J[r][cc] -= m * S.J[kk][cc];
        S.b[r] -= m * S.b[kk];
      }
      __syncthreads();
    }
    if (S.bad) break;
    if (r == 0) {
      for (int rr = n - 1; rr >= 0; --rr) {
        LU s = S.b[rr];
        for (int cc = rr + 1; cc < n; ++cc) s -= S.J[rr][cc] * S.b[cc];
        S.b[rr] = s / S.J[rr][rr];
      }
      if (M == POI) {
        LU m = 0;
        for (int rr = 0; rr < n; ++rr) m += S.b[rr];
        m /= (LU)n;
        for (int rr = 0; rr < n; ++rr) S.b[rr] -= m;
      }
      double dmax = 0.0, xmax = 0.0;
      for (int rr = 0; rr < n; ++rr) {
        S.xs[rr] += (double)S.b[rr];
        dmax = fmax(dmax, fabs((double)S.b[rr]));
        xmax = fmax(xmax, fabs(S.xs[rr]));
      }
      if (!isfinite(dmax) || !isfinite(xmax)) S.bad |= 2;
      else if (dmax <= 1e-13 * fmax(1.0, xmax)) S.done = 1;
    }
    __syncthreads();
    if (S.done || S.bad) { ++it; break; }
  }
  return it;
}

// Status of a dense Newton solve in the flag bits below.
template <class LU>
__device__ __forceinline__ int newton_flags(const NewtonScratchT<LU>& S) { return S.bad ? S.bad : (S.done ? 0 : 4); }

// status bits written to *flags (OR-ed): 1 = singular pivot, 2 = non-finite step, 4 = no step met the stop
// rule within the 50 steps
template <Model M, Form FM, class T>
__global__ void __launch_bounds__(kCoarseMax) coarse_newton(LevelView<T> L, Coef c, int* flags, int* steps_max) {
  __shared__ NewtonScratch S;
  const int n = 1 << (3 * L.lg), N = L.N, lg = L.lg, r = threadIdx.x;
  const int i = r >> (2 * lg), j = (r >> lg) & (N - 1), k = r & (N - 1);
  const size_t gr = r < n ? lidx<T>(lg, i, j, k) : 0;  // storage index of unknown r
  if (r < n) {
    S.xs[r] = (double)L.x[gr];
    S.etas[r] = uses_eta<M, FM>() ? (double)L.eta[gr] : 0.0;
    S.sigs[r] = L.sig ? (double)L.sig[gr] : 0.0;
    S.Bs[r] = (FM == DELTA && M != POI) ? (double)L.B[gr] : 0.0;
    S.ws[r] = (FM == DELTA && M == FOFR) ? (double)dexp<T>(L.B[gr]) : 0.0;  // e^B as the grids' kernels evaluate it
  }
  const int it = dense_newton_block<M, FM>(S, lg, (double)L.ih2, c);
  if (r < n) {
    L.x[gr] = (T)S.xs[r];
    if constexpr (M == FOFR && kExpCache<T>) L.aux[gr] = aux_of<M, FM, T>((T)S.xs[r], T(0));
  }
  if (r == 0) {
    const int f = newton_flags(S);
    if (f) atomicOr(flags, f);
    atomicMax(steps_max, it);
  }
}

// ---------------------------------------------------------------------------
// The coarse levels of a V-cycle in one CTA (FP32 grids)
// ---------------------------------------------------------------------------

constexpr int kCVMaxN = 16;      // the finest grid a fused coarse cycle starts from
constexpr int kCVThreads = 512;
constexpr int kCVMaxLev = 4;     // 16^3, 8^3, 4^3, 2^3

// The levels of one fused cycle: L[0] is its finest grid (x read, then written back), L[nlev-1] the coarsest.
// Global arrays in the red/black FP32 layout; sig of L[0] may be null (zero).
struct CoarseCycle {
  int nlev, nu1, nu2;
  LevelView<float> L[kCVMaxLev];
};

// Floats of shared memory for the level arrays (x, x0, Sigma, eta, B of every level).
inline size_t coarse_cycle_floats(int N0, int ncoarse) {
  size_t f = 0;
  for (int n = N0; n >= ncoarse; n >>= 1) f += 5 * (size_t)n * n * n;
  return f;
}

// One level's arrays in shared memory, row-major (i N + j) N + k.
struct SmemLevel {
  int lg;
  float ih2;
  float *x, *x0, *sig, *eta, *B;
};

template <Model M, Form FM>
__device__ __forceinline__ Cell<float> cv_gather(const SmemLevel& S, int i, int j, int k) {
  const int lg = S.lg, m = (1 << lg) - 1;
  auto at = [&](int a, int b, int d) { return (((a & m) << lg) | (b & m)) << lg | (d & m); };
  const int c = at(i, j, k);
  const int nb[6] = {at(i + 1, j, k), at(i - 1, j, k), at(i, j + 1, k), at(i, j - 1, k), at(i, j, k + 1),
                     at(i, j, k - 1)};
  Cell<float> q;
  q.x = S.x[c];
#pragma unroll
  for (int d = 0; d < 6; ++d) q.xn[d] = S.x[nb[d]];
  q.sig = S.sig[c];
  q.eta = uses_eta<M, FM>() ? S.eta[c] : 0.f;
  q.B = (FM == DELTA && M != POI) ? S.B[c] : 0.f;
  if constexpr (FM == DELTA && M == FOFR) {
#pragma unroll
    for (int d = 0; d < 6; ++d) q.Bn[d] = S.B[nb[d]];
  }
  fill_exps<M, FM, float>(q);
  return q;
}

// One colour of a Newton-Gauss-Seidel sweep (the update of smooth_rb).
template <Model M, Form FM>
__device__ void cv_smooth(const SmemLevel& S, const CoefT<float>& c, int color) {
  const int lg = S.lg, half = 1 << (3 * lg - 1), m = (1 << lg) - 1;
  for (int t = threadIdx.x; t < half; t += blockDim.x) {
    const int k2 = t & ((1 << (lg - 1)) - 1), row = t >> (lg - 1), j = row & m, i = row >> lg;
    const int k = 2 * k2 + ((i + j + color) & 1);
    Cell<float> q = cv_gather<M, FM>(S, i, j, k);
    float F, dF;
    eval_cell<M, FM, float>(c, S.ih2, q, F, dF);
    S.x[(((i << lg) | j) << lg) | k] = q.x - __fdividef(F, dF);
  }
}

// c: the constants of the FP64 Newton solve; cf: the same rounded to FP32 for the FP32 levels.
template <Model M, Form FM>
__global__ void __launch_bounds__(kCVThreads, 1) coarse_cycle(CoarseCycle cc, Coef c, CoefT<float> cf, int* flags,
                                                           int* steps_max) {
  extern __shared__ float4 cv_dyn[];
  __shared__ NewtonScratchT<float> NS;
  float* sm = reinterpret_cast<float*>(cv_dyn);
  SmemLevel S[kCVMaxLev];
  for (int l = 0; l < cc.nlev; ++l) {
    const int n = 1 << (3 * cc.L[l].lg);
    S[l].lg = cc.L[l].lg;
    S[l].ih2 = cc.L[l].ih2;
    S[l].x = sm; S[l].x0 = sm + n; S[l].sig = sm + 2 * n; S[l].eta = sm + 3 * n; S[l].B = sm + 4 * n;
    sm += 5 * n;
  }
  // load: the first level's x and Sigma, every level's eta and B (the per-solve restrictions)
  for (int l = 0; l < cc.nlev; ++l) {
    const LevelView<float>& G = cc.L[l];
    const int lg = G.lg, n = 1 << (3 * lg), m = (1 << lg) - 1;
    for (int t = threadIdx.x; t < n; t += blockDim.x) {
      const int i = t >> (2 * lg), j = (t >> lg) & m, k = t & m;
      const size_t g = lidx<float>(lg, i, j, k);
      if (l == 0) {
        S[0].x[t] = G.x[g];
        S[0].sig[t] = G.sig ? G.sig[g] : 0.f;
      }
      if constexpr (uses_eta<M, FM>()) S[l].eta[t] = G.eta[g];
      if constexpr (FM == DELTA && M != POI) S[l].B[t] = G.B[g];
    }
  }
  __syncthreads();
  const int last = cc.nlev - 1;
  // down: smooth, then residual + restriction and the FAS coarse source (Sect. 3.2)
  for (int l = 0; l < last; ++l) {
    for (int s = 0; s < cc.nu1; ++s)
      for (int color = 0; color < 2; ++color) {
        cv_smooth<M, FM>(S[l], cf, color);
        __syncthreads();
      }
    const SmemLevel &F = S[l], &C = S[l + 1];
    const int lgc = C.lg, nc = 1 << (3 * lgc), mc = (1 << lgc) - 1;
    for (int t = threadIdx.x; t < nc; t += blockDim.x) {
      const int I = t >> (2 * lgc), J = (t >> lgc) & mc, K = t & mc;
      float xs = 0.f, rs = 0.f;
#pragma unroll
      for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int b = 0; b < 2; ++b)
#pragma unroll
          for (int d = 0; d < 2; ++d) {
            Cell<float> q = cv_gather<M, FM>(F, 2 * I + a, 2 * J + b, 2 * K + d);
            float Fv, dF;
            eval_cell<M, FM, float>(cf, F.ih2, q, Fv, dF);
            xs += q.x;
            rs -= Fv;  // r = Sigma - L(x)
          }
      const float xr = xs * 0.125f;
      C.x[t] = xr;
      C.x0[t] = xr;
      C.sig[t] = rs * 0.125f;
    }
    __syncthreads();
    for (int t = threadIdx.x; t < nc; t += blockDim.x) {
      const int I = t >> (2 * lgc), J = (t >> lgc) & mc, K = t & mc;
      Cell<float> q = cv_gather<M, FM>(C, I, J, K);
      q.sig = 0.f;
      float Fv, dF;
      eval_cell<M, FM, float>(cf, C.ih2, q, Fv, dF);
      C.sig[t] += Fv;  // Sigma_H = L_H(R x) + R r
    }
    __syncthreads();
  }
  // the coarsest level: dense Newton in FP64
  {
    const SmemLevel& C = S[last];
    const int n = 1 << (3 * C.lg), r = threadIdx.x;
    if (r < n) {
      NS.xs[r] = (double)C.x[r];
      NS.etas[r] = uses_eta<M, FM>() ? (double)C.eta[r] : 0.0;
      NS.sigs[r] = (double)C.sig[r];
      NS.Bs[r] = (FM == DELTA && M != POI) ? (double)C.B[r] : 0.0;
      NS.ws[r] = (FM == DELTA && M == FOFR) ? (double)dexp<float>(C.B[r]) : 0.0;
    }
    const int it = dense_newton_block<M, FM, float>(NS, C.lg, (double)C.ih2, c);
    if (r < n) C.x[r] = (float)NS.xs[r];
    if (r == 0) {
      const int f = newton_flags(NS);
      if (f) atomicOr(flags, f);
      atomicMax(steps_max, it);
    }
    __syncthreads();
  }
  // up: x_h += P(x_H - x0_H) (cell-centred trilinear, weights 3/4 and 1/4 per axis), then smooth
  for (int l = last - 1; l >= 0; --l) {
    const SmemLevel &F = S[l], &C = S[l + 1];
    const int lg = F.lg, n = 1 << (3 * lg), m = (1 << lg) - 1, lgc = C.lg, mc = (1 << lgc) - 1;
    for (int t = threadIdx.x; t < n; t += blockDim.x) {
      const int i = t >> (2 * lg), j = (t >> lg) & m, k = t & m;
      const int ci[2] = {i >> 1, ((i >> 1) + ((i & 1) ? 1 : -1)) & mc};
      const int cj[2] = {j >> 1, ((j >> 1) + ((j & 1) ? 1 : -1)) & mc};
      const int ck[2] = {k >> 1, ((k >> 1) + ((k & 1) ? 1 : -1)) & mc};
      const float w[2] = {0.75f, 0.25f};
      float v = 0.f;
#pragma unroll
      for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int b = 0; b < 2; ++b)
#pragma unroll
          for (int d = 0; d < 2; ++d) {
            const int q = (((ci[a] << lgc) | cj[b]) << lgc) | ck[d];
            v += w[a] * w[b] * w[d] * (C.x[q] - C.x0[q]);
          }
      F.x[t] += v;
    }
    __syncthreads();
    for (int s = 0; s < cc.nu2; ++s)
      for (int color = 0; color < 2; ++color) {
        cv_smooth<M, FM>(S[l], cf, color);
        __syncthreads();
      }
  }
  // store the first level's x
  {
    const LevelView<float>& G = cc.L[0];
    const int lg = G.lg, n = 1 << (3 * lg), m = (1 << lg) - 1;
    for (int t = threadIdx.x; t < n; t += blockDim.x) {
      const int i = t >> (2 * lg), j = (t >> lg) & m, k = t & m;
      G.x[lidx<float>(lg, i, j, k)] = S[0].x[t];
    }
  }
}

}  // namespace isis
