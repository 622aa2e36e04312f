// isis_solver.cuh -- host orchestration of the FAS multigrid solve
// (Sect. 3.2 of arXiv:1307.6748): level hierarchy, V-cycles, convergence
// test, and the FP64 defect-correction loop around FP32 correction cycles.
#pragma once
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <cstring>
#include <vector>

#include "../../include/isis.h"
#include "isis_coarse.cuh"
#include "isis_stream.cuh"
#include "isis_exp64.cuh"
#include "isis_prof.cuh"

namespace isis {

// ---------------------------------------------------------------------------
// Device buffers
// ---------------------------------------------------------------------------

struct DevBuf {
  void* p = nullptr;
  size_t bytes = 0;
};

// One cached allocation set per (N, element size); see isis_api.cu.
struct Workspace {
  int N = 0, esize = 0, device = -1;
  int nlev = 0;
  // per level l (0 = finest): x, x0, sig, eta, B, w (element type T)
  std::vector<void*> x, x0, sig, eta, B, w;
  std::vector<void*> xalt;    // second buffer of x for the streaming smoother (FP32, N >= kStreamMinN)
  double* part = nullptr;     // kNormBlocks partial sums
  double* part2 = nullptr;    // second set of partials
  double* scal = nullptr;     // device scalars: [0] norm^2, [1] sum, [2] aux
  int* iflags = nullptr;      // [0] coarse flags, [1] coarse steps max
  void* host = nullptr;       // pinned readback area
  double* exptab = nullptr;   // 2^(j/256), j < 256, for exp_tang
  double* b64 = nullptr;      // finest level, FP64: e^u (f(R) residual), allocated on first use
  double* s64 = nullptr;      // finest level, FP64: S(u, eta) (f(R) residual)
  std::vector<void*> owned;
};

// FP64 scratch of the f(R) residual on the finest grid (lazily allocated).
bool ensure_fofr64(Workspace* ws);

// Returns nullptr on allocation failure.  Implemented in isis_api.cu.
Workspace* get_workspace(int N, int esize, int ncoarse);

// Common arguments of one solve.
struct SolveArgs {
  int N;
  double box, a;
  Coef coef;
  const void* eta;
  void* phi;
  double tol;
  int nu1, nu2, ncoarse, max_cycles, inner;
  isis_precision prec;
  isis_init init;
  isis_solve_info* info;
  cudaStream_t st;
  // reference residual: ref = ref_scale * RMS(eta - eta_ref) (eta_ref = <eta> for Poisson)
  double ref_scale;
};

#define ISIS_CK(call)                              \
  do {                                             \
    cudaError_t e_ = (call);                       \
    if (e_ != cudaSuccess) return ISIS_ECUDA;      \
  } while (0)
#define ISIS_CKL() ISIS_CK(cudaGetLastError())

inline int ilog2(int n) {
  int l = 0;
  while ((1 << l) < n) ++l;
  return l;
}
inline unsigned nblk(size_t n, int t) { return (unsigned)((n + t - 1) / t); }

// Grids at least this large are smoothed by the temporally blocked streaming
// kernel (FP32 only); smaller ones by the one-colour kernel.
constexpr int kStreamMinN = 128;
// Sweeps fused per streaming pass (1 or 2).
constexpr int kStreamSweeps = 1;

// One streaming pass of NSW sweeps: xin -> xout.
template <Model M, Form FM, int NSW>
isis_status stream_pass(const LevelView<float>& v, float* xout, const Coef& c, cudaStream_t st, double bytes,
                        int kind) {
  constexpr int TJ = StreamCfg<M, FM, NSW>::TJ, H = 2 * NSW;
  constexpr size_t smem = stream_smem<M, FM, NSW>();
  static bool attr_done = false;
  if (!attr_done) {
    if (smem > 48 * 1024 &&
        cudaFuncSetAttribute(smooth_stream<M, FM, NSW>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
            cudaSuccess)
      return ISIS_ECUDA;
    attr_done = true;
  }
  const int N = v.N;
  const int TI = N >= 512 ? 64 : (N >= 256 ? 32 : 16);
  dim3 grid((unsigned)((N + (64 - 2 * H) - 1) / (64 - 2 * H)), (unsigned)((N + (TJ - 2 * H) - 1) / (TJ - 2 * H)),
            (unsigned)(N / TI));
  ISIS_LAUNCH(kind, bytes, st, (smooth_stream<M, FM, NSW><<<grid, 32 * TJ, smem, st>>>(v, xout, c, TI)));
  return ISIS_OK;
}

// ---------------------------------------------------------------------------
// V-cycle driver for one model / form / element type
// ---------------------------------------------------------------------------

template <Model M, Form FM, class T>
struct Cycler {
  std::vector<LevelView<T>> L;
  std::vector<T*> alt;  // second buffer of each level's x (streaming smoother), else nullptr
  Workspace* ws = nullptr;
  Coef c;
  int nu1 = 2, nu2 = 2;
  cudaStream_t st = 0;

  // Build level views; level 0 uses (x0_, eta0, sig0, B0, w0).
  void setup(Workspace* w, const SolveArgs& A, T* xfine, const T* etafine, const T* sigfine) {
    ws = w;
    c = A.coef;
    nu1 = A.nu1;
    nu2 = A.nu2;
    st = A.st;
    L.resize(ws->nlev);
    alt.assign(ws->nlev, nullptr);
    for (int l = 0; l < ws->nlev; ++l) {
      if (sizeof(T) == 4) alt[l] = (T*)ws->xalt[l];
      int N = A.N >> l;
      double h = A.box / N;
      LevelView<T> v;
      v.N = N;
      v.lg = ilog2(N);
      v.ih2 = (T)(1.0 / (h * h));
      v.x = l == 0 ? xfine : (T*)ws->x[l];
      v.eta = l == 0 ? etafine : (const T*)ws->eta[l];
      v.sig = l == 0 ? sigfine : (const T*)ws->sig[l];
      v.B = (const T*)ws->B[l];
      v.w = (const T*)ws->w[l];
      L[l] = v;
    }
  }

  // per-cell input arrays read by the operator besides x (eta, B, w, Sigma)
  static int arrays(bool has_sig) {
    int n = has_sig ? 1 : 0;
    if (!(M == POI && FM == DELTA)) n += 1;   // eta
    if (FM == DELTA && M != POI) n += 1;      // B
    if (FM == DELTA && M == FOFR) n += 1;     // w
    return n;
  }
  static double cells(const LevelView<T>& v) { return (double)v.N * v.N * v.N; }

  isis_status smooth(int l, int sweeps) {
    LevelView<T>& v = L[l];
    size_t half = ((size_t)v.N * v.N * v.N) / 2;
    // algorithmic bytes of a full sweep, and of one streaming pass of 1 or 2
    // sweeps: read x and the per-cell arrays once, write x once
    double bytes = cells(v) * sizeof(T) * (2 + arrays(v.sig != nullptr));
    int kind = l == 0 ? KK_SMOOTH_FINE : KK_SMOOTH_COARSE;
    if constexpr (sizeof(T) == 4) {
      if (v.N >= kStreamMinN && alt[l]) {
        // one sweep per pass over HBM (fusing two costs more in redundant halo
        // work than it saves in traffic); the field alternates between x and alt
        int left = sweeps;
        while (left > 0) {
          int nsw = (left >= 2 && kStreamSweeps == 2) ? 2 : 1;
          float* out = alt[l];
          isis_status r = nsw == 2 ? stream_pass<M, FM, 2>(v, out, c, st, bytes, kind)
                                   : stream_pass<M, FM, 1>(v, out, c, st, bytes, kind);
          if (r != ISIS_OK) return r;
          alt[l] = v.x;
          v.x = out;
          left -= nsw;
        }
        return ISIS_OK;
      }
    }
    for (int s = 0; s < sweeps; ++s)
      for (int color = 0; color < 2; ++color)
        ISIS_LAUNCH(kind, bytes * 0.5, st, (smooth_color<M, FM, T><<<nblk(half, 256), 256, 0, st>>>(v, c, color)));
    return ISIS_OK;
  }

  isis_status vcycle(int l) {
    const int last = (int)L.size() - 1;
    if (l == last) {
      ISIS_LAUNCH(KK_COARSE_NEWTON, 0.0, st,
                  (coarse_newton<M, FM, T><<<1, kCoarseMax, 0, st>>>(L[l], c, ws->iflags, ws->iflags + 1)));
      return ISIS_OK;
    }
    isis_status s = smooth(l, nu1);
    if (s != ISIS_OK) return s;
    LevelView<T>& C = L[l + 1];
    size_t nc = (size_t)C.N * C.N * C.N;
    double nf = cells(L[l]), ncd = (double)nc;
    ISIS_LAUNCH(l == 0 ? KK_RESTRICT_FINE : KK_RESTRICT_COARSE,
                sizeof(T) * (nf * (1 + arrays(L[l].sig != nullptr)) + 3 * ncd), st,
                (resid_restrict<M, FM, T><<<nblk(nc, 256), 256, 0, st>>>(L[l], c, C.x, (T*)ws->x0[l + 1],
                                                                        (T*)ws->sig[l + 1])));
    ISIS_LAUNCH(KK_SIGMA, sizeof(T) * ncd * (2 + arrays(true)), st,
                (coarse_sigma_add<M, FM, T><<<nblk(nc, 256), 256, 0, st>>>(C, c, (T*)ws->sig[l + 1])));
    s = vcycle(l + 1);
    if (s != ISIS_OK) return s;
    ISIS_LAUNCH(l == 0 ? KK_PROLONG_FINE : KK_PROLONG_COARSE, sizeof(T) * (2 * ncd + 2 * nf), st,
                (prolong_correct<T><<<nblk((size_t)nf, 256), 256, 0, st>>>(L[l].x, C.x, (const T*)ws->x0[l + 1],
                                                                           C.lg)));
    return smooth(l, nu2);
  }

  // RMS of L(x) - Sigma on the finest level (blocking: one stream sync).
  isis_status fine_rms(double* out) {
    ISIS_LAUNCH(KK_NORM, cells(L[0]) * sizeof(T) * (1 + arrays(L[0].sig != nullptr)), st,
                (norm_partial<M, FM, T><<<kNormBlocks, kNormThreads, 0, st>>>(L[0], c, ws->part)));
    ISIS_LAUNCH(KK_REDUCE, 0.0, st, (reduce_final<<<1, kNormThreads, 0, st>>>(ws->part, kNormBlocks, ws->scal)));
    double* h = (double*)ws->host;
    int* hi = (int*)(h + 4);
    ISIS_CK(cudaMemcpyAsync(h, ws->scal, sizeof(double), cudaMemcpyDeviceToHost, st));
    ISIS_CK(cudaMemcpyAsync(hi, ws->iflags, 2 * sizeof(int), cudaMemcpyDeviceToHost, st));
    ISIS_CK(cudaStreamSynchronize(st));
    size_t n = (size_t)L[0].N * L[0].N * L[0].N;
    *out = std::sqrt(h[0] / (double)n);
    if (hi[0] != 0) return ISIS_ENAN;
    return ISIS_OK;
  }
};

// ---------------------------------------------------------------------------
// Reductions used by the drivers
// ---------------------------------------------------------------------------

// sum((v - shift)^2) and sum(v) over n values (blocking).
template <class T>
isis_status moments(Workspace* ws, const T* v, size_t n, double shift, cudaStream_t st, double* s2, double* s1) {
  ISIS_LAUNCH(KK_REDUCE, (double)n * sizeof(T), st,
              (moments_partial<T><<<kNormBlocks, kNormThreads, 0, st>>>(v, n, shift, ws->part, ws->part2)));
  ISIS_LAUNCH(KK_REDUCE, 0.0, st, (reduce_final<<<1, kNormThreads, 0, st>>>(ws->part, kNormBlocks, ws->scal)));
  ISIS_LAUNCH(KK_REDUCE, 0.0, st,
              (reduce_final<<<1, kNormThreads, 0, st>>>(ws->part2, kNormBlocks, ws->scal + 1)));
  double* h = (double*)ws->host;
  ISIS_CK(cudaMemcpyAsync(h, ws->scal, 2 * sizeof(double), cudaMemcpyDeviceToHost, st));
  ISIS_CK(cudaStreamSynchronize(st));
  *s2 = h[0];
  *s1 = h[1];
  return ISIS_OK;
}

template <class T>
__global__ void add_scalar(T* __restrict__ v, size_t n, const double* __restrict__ sum, double inv_n) {
  size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t < n) v[t] = (T)((double)v[t] - (*sum) * inv_n);
}

// v -= mean(v), device-side (no host sync): partial sums, final sum, subtract.
template <class T>
isis_status remove_mean(Workspace* ws, T* v, size_t n, cudaStream_t st) {
  ISIS_LAUNCH(KK_REDUCE, (double)n * sizeof(T), st,
              (moments_partial<T><<<kNormBlocks, kNormThreads, 0, st>>>(v, n, 0.0, ws->part, ws->part2)));
  ISIS_LAUNCH(KK_REDUCE, 0.0, st,
              (reduce_final<<<1, kNormThreads, 0, st>>>(ws->part2, kNormBlocks, ws->scal + 1)));
  ISIS_LAUNCH(KK_REDUCE, 2.0 * n * sizeof(T), st,
              (add_scalar<T><<<nblk(n, 256), 256, 0, st>>>(v, n, ws->scal + 1, 1.0 / (double)n)));
  return ISIS_OK;
}

template <class Tin, class Tout>
__global__ void convert_k(const Tin* __restrict__ a, Tout* __restrict__ b, size_t n) {
  size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t < n) b[t] = (Tout)a[t];
}

template <class T>
__global__ void exp_k(const T* __restrict__ a, T* __restrict__ b, size_t n) {
  size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t < n) b[t] = dexp<T>(a[t]);
}

template <class T>
__global__ void fill_k(T* __restrict__ a, T v, size_t n) {
  size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t < n) a[t] = v;
}

__global__ void update_phi64(double* __restrict__ phi, const float* __restrict__ e, size_t n);

// Initial guess (isis_init): the background constant, or cell by cell the
// solution for a uniform density equal to the cell's eta (computed in FP32:
// it is only a starting point).
template <Model M, class T>
__global__ void init_guess(T* __restrict__ phi, const T* __restrict__ eta, size_t n, Coef c, int mode, double bg) {
  size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n) return;
  if (mode == ISIS_INIT_BACKGROUND || M == POI) { phi[t] = (T)bg; return; }
  float e = (float)eta[t];
  if (M == SYM) {
    float v = 1.0f - (float)c.s * e;
    phi[t] = (T)(v > 0.0f ? sqrtf(v) : 0.0f);
  } else {
    // S(u) = 0 at this eta: e^{u/(n+1)} = K2 / (K1 (eta - 1) + K3)
    float den = (float)c.K1 * (e - 1.0f) + (float)c.K3;
    phi[t] = (T)((float)c.np1 * logf((float)c.K2 / den));
  }
}

// background field of the model (the ISIS_INIT_BACKGROUND value)
template <Model M>
inline double background_value(const Coef& c) {
  if (M == SYM) return c.s < 1.0 ? std::sqrt(1.0 - c.s) : 0.0;
  if (M == FOFR) return c.np1 * std::log(c.K2 / c.K3);
  return 0.0;
}

template <Model M, class T>
isis_status apply_init(const SolveArgs& A, const Coef& c, T* phi, const T* eta, size_t n) {
  if (A.init == ISIS_INIT_INPUT) return ISIS_OK;
  cudaStream_t st = A.st;
  ISIS_LAUNCH(KK_INIT, (double)n * sizeof(T) * (A.init == ISIS_INIT_LOCAL ? 2 : 1), st,
              (init_guess<M, T><<<nblk(n, 256), 256, 0, st>>>(phi, eta, n, c, (int)A.init, background_value<M>(c))));
  return ISIS_OK;
}

// FP64 residual of the finest grid for the defect-correction loop:
// r = -L64(phi); writes r and B = phi rounded to FP32, and block partials of r^2.
// (Poisson and symmetron: the operator has no transcendental terms.)
template <Model M>
__global__ void __launch_bounds__(kNormThreads) outer_residual(LevelView<double> L, Coef c, float* __restrict__ r32,
                                                               float* __restrict__ B32, double* __restrict__ part) {
  size_t n = (size_t)1 << (3 * L.lg);
  double acc = 0.0;
  for (size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (size_t)gridDim.x * blockDim.x) {
    int k = (int)(t & (L.N - 1)), j = (int)((t >> L.lg) & (L.N - 1)), i = (int)(t >> (2 * L.lg));
    Cell<double> q = gather<M, FIELD, double>(L, i, j, k);
    double F, dF;
    eval_cell<M, FIELD, double>(c, L.ih2, q, F, dF);
    r32[t] = (float)(-F);
    B32[t] = (float)q.x;
    acc += F * F;
  }
  block_sum_store<double>(acc, part);
}

// f(R), first pass: per cell b = e^u and S(u, eta) = K1 (eta - 1) - K2 e^{-u/(n+1)} + K3,
// each exponential evaluated once per cell (Sect. 4.2).
__global__ void fofr_prep64(const double* __restrict__ u, const double* __restrict__ eta, double* __restrict__ b,
                            double* __restrict__ S, size_t n, Coef c, const double* __restrict__ tab);

// f(R), second pass: flux form of Eq. (disc_non_canonical) with face b = (b_c + b_nb)/2:
//   sum_f b_f (u_nb - u) = [ b_c (sum u_nb - 6 u) + sum b_nb u_nb - u sum b_nb ] / 2
__global__ void __launch_bounds__(kNormThreads) outer_residual_fofr(int lg, double ih2, const double* __restrict__ u,
                                                                    const double* __restrict__ b,
                                                                    const double* __restrict__ S,
                                                                    float* __restrict__ r32, float* __restrict__ B32,
                                                                    double* __restrict__ part);

// ---------------------------------------------------------------------------
// Drivers
// ---------------------------------------------------------------------------

inline void info_reset(isis_solve_info* info) {
  if (info) std::memset(info, 0, sizeof(*info));
}

// Plain solve: every level in type T, field form, in place on phi.
template <Model M, class T>
isis_status solve_field(const SolveArgs& A) {
  Workspace* ws = get_workspace(A.N, sizeof(T), A.ncoarse);
  if (!ws) return ISIS_ENOMEM;
  cudaStream_t st = A.st;
  const size_t n = (size_t)A.N * A.N * A.N;
  const T* eta = (const T*)A.eta;
  T* phi = (T*)A.phi;
  Coef c = A.coef;
  isis_solve_info loc;
  info_reset(&loc);

  double s2, s1;
  isis_status s = moments<T>(ws, eta, n, 1.0, st, &s2, &s1);
  if (s != ISIS_OK) return s;
  double eta_mean = s1 / (double)n;
  if (M == POI) {
    c.eta_mean = eta_mean;
    // sum (eta - <eta>)^2 = sum (eta - 1)^2 - n (<eta> - 1)^2
    s2 = s2 - (double)n * (eta_mean - 1.0) * (eta_mean - 1.0);
    if (s2 < 0) s2 = 0;
  }
  double ref = A.ref_scale * std::sqrt(s2 / (double)n);
  s = apply_init<M, T>(A, c, phi, eta, n);
  if (s != ISIS_OK) return s;

  // density on the coarse levels
  for (int l = 1; l < ws->nlev; ++l) {
    int lgc = ilog2(A.N >> l);
    const T* f = l == 1 ? eta : (const T*)ws->eta[l - 1];
    size_t ncl = (size_t)1 << (3 * lgc);
    ISIS_LAUNCH(KK_SETUP, 9.0 * ncl * sizeof(T), st,
                (restrict_mean<T, T><<<nblk(ncl, 256), 256, 0, st>>>(f, (T*)ws->eta[l], lgc)));
  }
  ISIS_CK(cudaMemsetAsync(ws->iflags, 0, 2 * sizeof(int), st));

  Cycler<M, FIELD, T> cy;
  SolveArgs A2 = A;
  A2.coef = c;
  cy.setup(ws, A2, phi, eta, nullptr);

  double res;
  s = cy.fine_rms(&res);
  if (s != ISIS_OK) return s;
  loc.res0 = res;
  if (!(ref > 0.0)) ref = res;
  loc.res_ref = ref;
  loc.res_final = res;
  double target = A.tol * ref;
  isis_status out = ISIS_ENOCONV;
  if (!std::isfinite(res)) out = ISIS_ENAN;
  else if (res <= target) out = ISIS_OK;
  else {
    for (int cyc = 0; cyc < A.max_cycles; ++cyc) {
      s = cy.vcycle(0);
      if (s != ISIS_OK) { out = s; break; }
      if (M == POI) {
        s = remove_mean<T>(ws, cy.L[0].x, n, st);
        if (s != ISIS_OK) { out = s; break; }
      }
      s = cy.fine_rms(&res);
      loc.cycles = cyc + 1;
      loc.hist[cyc] = res;
      loc.nhist = cyc + 1;
      loc.res_final = res;
      if (s != ISIS_OK) { out = s; break; }
      if (!std::isfinite(res)) { out = ISIS_ENAN; break; }
      if (res <= target) { out = ISIS_OK; break; }
    }
  }
  if (cy.L[0].x != phi) ISIS_CK(cudaMemcpyAsync(phi, cy.L[0].x, n * sizeof(T), cudaMemcpyDeviceToDevice, st));
  if (A.info) *A.info = loc;
  return out;
}

// Relative residual (of the reference) below which the FP32 field-form
// cycles hand over to the FP64 defect correction, and the per-cycle
// reduction above which they are taken to have reached FP32 rounding.
constexpr double kSwitchRel = 1e-4;
constexpr double kStallRatio = 0.5;

// FP32 cycles + FP64 defect correction.
//  Phase 1: FAS V-cycles on the field itself in FP32 (psi = fp32(phi)) until
//           the FP32-evaluated residual is below kSwitchRel * ref or stalls.
//  Phase 2: outer loop: r = -L64(phi) in FP64; FP32 FAS V-cycles on the
//           correction e of L(B + e) - L(B) = r, B = fp32(phi) (DELTA form);
//           phi += e in FP64; until the FP64 residual is <= tol * ref.
template <Model M>
isis_status solve_refine(const SolveArgs& A) {
  Workspace* ws = get_workspace(A.N, sizeof(float), A.ncoarse);
  if (!ws) return ISIS_ENOMEM;
  if (M == FOFR && !ensure_fofr64(ws)) return ISIS_ENOMEM;
  cudaStream_t st = A.st;
  const size_t n = (size_t)A.N * A.N * A.N;
  const double* eta64 = (const double*)A.eta;
  double* phi64 = (double*)A.phi;
  Coef c = A.coef;
  isis_solve_info loc;
  info_reset(&loc);

  // FP32 buffers of the finest level: x = e, sig = r, eta, B (= psi in phase 1), w
  float* e0 = (float*)ws->x[0];
  float* r0 = (float*)ws->sig[0];
  float* eta0 = (float*)ws->eta[0];
  float* B0 = (float*)ws->B[0];

  double s2, s1;
  isis_status s = moments<double>(ws, eta64, n, 1.0, st, &s2, &s1);
  if (s != ISIS_OK) return s;
  double eta_mean = s1 / (double)n;
  if (M == POI) {
    c.eta_mean = eta_mean;
    s2 = s2 - (double)n * (eta_mean - 1.0) * (eta_mean - 1.0);
    if (s2 < 0) s2 = 0;
  }
  double ref = A.ref_scale * std::sqrt(s2 / (double)n);
  s = apply_init<M, double>(A, c, phi64, eta64, n);
  if (s != ISIS_OK) return s;

  ISIS_LAUNCH(KK_SETUP, 12.0 * n, st, (convert_k<double, float><<<nblk(n, 256), 256, 0, st>>>(eta64, eta0, n)));
  for (int l = 1; l < ws->nlev; ++l) {
    int lgc = ilog2(A.N >> l);
    size_t ncl = (size_t)1 << (3 * lgc);
    ISIS_LAUNCH(KK_SETUP, 36.0 * ncl, st,
                (restrict_mean<float, float><<<nblk(ncl, 256), 256, 0, st>>>((const float*)ws->eta[l - 1],
                                                                            (float*)ws->eta[l], lgc)));
  }
  ISIS_CK(cudaMemsetAsync(ws->iflags, 0, 2 * sizeof(int), st));
  SolveArgs A2 = A;
  A2.coef = c;
  int nh = 0;  // history entries

  // ---- phase 1: FP32 field-form cycles ----
  ISIS_LAUNCH(KK_SETUP, 12.0 * n, st, (convert_k<double, float><<<nblk(n, 256), 256, 0, st>>>(phi64, B0, n)));
  {
    Cycler<M, FIELD, float> cy;
    cy.setup(ws, A2, B0, eta0, nullptr);
    double res;
    s = cy.fine_rms(&res);
    if (s != ISIS_OK) return s;
    loc.res0 = res;
    if (!(ref > 0.0)) ref = res;
    loc.res_ref = ref;
    double prev = res;
    double handover = std::fmax(A.tol, kSwitchRel) * ref;
    while (res > handover && loc.cycles < A.max_cycles && std::isfinite(res)) {
      s = cy.vcycle(0);
      if (s != ISIS_OK) return s;
      s = cy.fine_rms(&res);
      loc.cycles += 1;
      if (nh < 128) loc.hist[nh++] = res;
      loc.nhist = nh;
      if (s != ISIS_OK) { if (A.info) *A.info = loc; return s; }
      if (!(res <= kStallRatio * prev)) break;
      prev = res;
    }
    if (!std::isfinite(res)) {
      loc.res_final = res;
      if (A.info) *A.info = loc;
      return ISIS_ENAN;
    }
    const float* psi = cy.L[0].x;
    ISIS_LAUNCH(KK_SETUP, 12.0 * n, st, (convert_k<float, double><<<nblk(n, 256), 256, 0, st>>>(psi, phi64, n)));
    // Poisson gauge: the residual does not see the mean, so it is removed once per phase
    if (M == POI) {
      s = remove_mean<double>(ws, phi64, n, st);
      if (s != ISIS_OK) return s;
    }
  }

  // ---- phase 2: FP64 defect correction around FP32 correction cycles ----
  LevelView<double> F64;
  F64.N = A.N;
  F64.lg = ilog2(A.N);
  F64.ih2 = 1.0 / ((A.box / A.N) * (A.box / A.N));
  F64.x = phi64;
  F64.eta = eta64;
  F64.sig = nullptr;
  F64.B = nullptr;
  F64.w = nullptr;

  Cycler<M, DELTA, float> cy;
  cy.setup(ws, A2, e0, eta0, r0);

  double* h = (double*)ws->host;
  int* hi = (int*)(h + 4);
  isis_status out = ISIS_ENOCONV;
  const double target = A.tol * ref;
  for (int outer = 0;; ++outer) {
    // r = -L64(phi64), B = fp32(phi64), RMS of r
    if (M == FOFR) {
      ISIS_LAUNCH(KK_OUTER_RESID, 32.0 * n, st,
                  (fofr_prep64<<<nblk(n, 256), 256, 0, st>>>(phi64, eta64, ws->b64, ws->s64, n, c, ws->exptab)));
      ISIS_LAUNCH(KK_OUTER_RESID, 32.0 * n, st,
                  (outer_residual_fofr<<<kNormBlocks, kNormThreads, 0, st>>>(F64.lg, F64.ih2, phi64, ws->b64,
                                                                              ws->s64, r0, B0, ws->part)));
    } else {
      ISIS_LAUNCH(KK_OUTER_RESID, 24.0 * n, st,
                  (outer_residual<M><<<kNormBlocks, kNormThreads, 0, st>>>(F64, c, r0, B0, ws->part)));
    }
    ISIS_LAUNCH(KK_REDUCE, 0.0, st, (reduce_final<<<1, kNormThreads, 0, st>>>(ws->part, kNormBlocks, ws->scal)));
    ISIS_CK(cudaMemcpyAsync(h, ws->scal, sizeof(double), cudaMemcpyDeviceToHost, st));
    ISIS_CK(cudaMemcpyAsync(hi, ws->iflags, 2 * sizeof(int), cudaMemcpyDeviceToHost, st));
    ISIS_CK(cudaStreamSynchronize(st));
    double res = std::sqrt(h[0] / (double)n);
    if (outer > 0 && nh < 128) loc.hist[nh++] = res;
    loc.nhist = nh;
    loc.res_final = res;
    loc.outer = outer;
    if (hi[0] != 0) { out = ISIS_ENAN; break; }
    if (!std::isfinite(res)) { out = ISIS_ENAN; break; }
    if (res <= target) { out = ISIS_OK; break; }
    if (loc.cycles >= A.max_cycles || outer >= 127) { out = ISIS_ENOCONV; break; }

    // base field on every level (B_l = R B_{l-1}) and e^B for f(R)
    for (int l = 1; l < ws->nlev && M != POI; ++l) {
      int lgc = ilog2(A.N >> l);
      size_t ncl = (size_t)1 << (3 * lgc);
      ISIS_LAUNCH(KK_SETUP, 36.0 * ncl, st,
                  (restrict_mean<float, float><<<nblk(ncl, 256), 256, 0, st>>>((const float*)ws->B[l - 1],
                                                                              (float*)ws->B[l], lgc)));
    }
    if (M == FOFR) {
      for (int l = 0; l < ws->nlev; ++l) {
        size_t nl = (size_t)(A.N >> l) * (A.N >> l) * (A.N >> l);
        ISIS_LAUNCH(KK_SETUP, 8.0 * nl, st,
                    (exp_k<float><<<nblk(nl, 256), 256, 0, st>>>((const float*)ws->B[l], (float*)ws->w[l], nl)));
      }
    }
    ISIS_CK(cudaMemsetAsync(cy.L[0].x, 0, n * sizeof(float), st));
    int k = A.inner;
    if (loc.cycles + k > A.max_cycles) k = A.max_cycles - loc.cycles;
    for (int it = 0; it < k; ++it) {
      s = cy.vcycle(0);
      if (s != ISIS_OK) return s;
    }
    loc.cycles += k;
    const float* ecur = cy.L[0].x;
    ISIS_LAUNCH(KK_UPDATE, 20.0 * n, st, (update_phi64<<<nblk(n, 256), 256, 0, st>>>(phi64, ecur, n)));
  }
  if (M == POI) {
    s = remove_mean<double>(ws, phi64, n, st);
    if (s != ISIS_OK) return s;
  }
  if (A.info) *A.info = loc;
  return out;
}

}  // namespace isis
