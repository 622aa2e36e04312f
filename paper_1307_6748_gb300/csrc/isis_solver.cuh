// isis_solver.cuh -- host orchestration of the FAS multigrid solve
// (Sect. 3.2 of arXiv:1307.6748): level hierarchy, V-cycles, convergence
// test, and the FP64 defect-correction loop around FP32 correction cycles.
#pragma once
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <cstring>
#include <type_traits>
#include <vector>

#include "../../include/isis.h"
#include "isis_coarse.cuh"
#include "isis_ff.cuh"
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
  std::vector<void*> aux;     // f(R): cached e^x / e^B expm1(x) per level (level 0 too)
  double* part = nullptr;     // kNormBlocks partial sums
  double* part2 = nullptr;    // second set of partials
  double* scal = nullptr;     // device scalars: [0] norm^2, [1] sum, [2] aux
  int* iflags = nullptr;      // [0] coarse flags, [1] coarse steps max
  void* host = nullptr;       // mapped pinned readback area: [0..3] doubles, then ints at (int*)(host + 4)
  double* host_dev = nullptr;  // its device address
  float2* exptab_ff = nullptr;  // 2^(j/64), j < 64, float-float, for exp_ff2
  double* b64 = nullptr;      // finest level, 8 bytes per cell: psi = u - u_bar (float-float), f(R) residual
  double* s64 = nullptr;      // finest level, 8 bytes per cell: e^psi (float-float), f(R) residual
  std::vector<void*> xalt;    // FP32 levels: a scratch grid of the level's size (lazy), see get_xalt
  std::vector<void*> owned;
};

// A scratch FP32 grid of level l's size (allocated at first use; nullptr on failure).  Implemented in isis_api.cu.
float* get_xalt(Workspace* ws, int l);

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
  int fmg;  // nested-iteration start of the FP32 phase (ISIS_F32_REFINE64)
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

// Status of the solve from the coarsest Newton solve's flags: a singular pivot or a non-finite step is
// ISIS_ENAN; a solve that did not meet its stop rule in 50 steps ends the solve with ISIS_ENOCONV.
inline isis_status coarse_status(int flags) {
  if (flags & 3) return ISIS_ENAN;
  if (flags & 4) return ISIS_ENOCONV;
  return ISIS_OK;
}

// ---------------------------------------------------------------------------
// V-cycle driver for one model / form / element type
// ---------------------------------------------------------------------------

template <Model M, Form FM, class T>
struct Cycler {
  std::vector<LevelView<T>> L;
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
    for (int l = 0; l < ws->nlev; ++l) {
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
      v.aux = (T*)ws->aux[l];
      L[l] = v;
    }
  }

  // per-cell input arrays read by the operator besides x (eta, B, Sigma)
  static int arrays(bool has_sig) {
    int n = has_sig ? 1 : 0;
    if (uses_eta<M, FM>()) n += 1;        // eta
    if (FM == DELTA && M != POI) n += 1;  // B
    return n;
  }
  static double cells(const LevelView<T>& v) { return (double)v.N * v.N * v.N; }
  // kernel kind of a launch, with this instantiation's model and form
  static constexpr int tk(int kind) { return kind_tag(kind, (int)M, (int)FM); }

  isis_status smooth(int l, int sweeps) {
    LevelView<T>& v = L[l];
    size_t half = ((size_t)v.N * v.N * v.N) / 2;
    // algorithmic bytes of a full sweep: read x and the per-cell arrays once,
    // write x once (a one-colour launch moves half of that)
    double bytes = cells(v) * sizeof(T) * (2 + arrays(v.sig != nullptr));
    const int kind = tk(l == 0 ? KK_SMOOTH_FINE : KK_SMOOTH_COARSE);
    for (int s = 0; s < sweeps; ++s)
      for (int color = 0; color < 2; ++color) {
        if constexpr (sizeof(T) == 4) {
          if (v.N >= 4)
            ISIS_LAUNCH(kind, bytes * 0.5, st,
                        (smooth_rb2<M, FM><<<nblk(half / 2, 256), 256, 0, st>>>(v, c, color)));
          else
            ISIS_LAUNCH(kind, bytes * 0.5, st, (smooth_rb<M, FM><<<nblk(half, 256), 256, 0, st>>>(v, c, color)));
        }
        else
          ISIS_LAUNCH(kind, bytes * 0.5, st,
                      (smooth_color<M, FM, T><<<nblk(half, 256), 256, 0, st>>>(v, c, color)));
      }
    return ISIS_OK;
  }

  // x_l += P(x_{l+1} - x0_{l+1})
  isis_status prolong(int l) {
    LevelView<T>& C = L[l + 1];
    const size_t nc = (size_t)C.N * C.N * C.N;
    const double bytes = sizeof(T) * (2 * (double)nc + 2 * cells(L[l]));
    const int kind = tk(l == 0 ? KK_PROLONG_FINE : KK_PROLONG_COARSE);
    if constexpr (sizeof(T) == 4) {
      if (C.N >= kP2K) {
        const unsigned blocks = (unsigned)(nc / (kPTI * kPTJ * kP2K));
        ISIS_LAUNCH(kind, bytes, st,
                    (prolong_tiled2<M, FM><<<blocks, kPTI * kPTJ * kPTK, 0, st>>>(L[l], C.x, (const T*)ws->x0[l + 1],
                                                                                   C.lg)));
        return ISIS_OK;
      }
      if (C.N >= kPTK) {
        const unsigned blocks = (unsigned)(nc / (kPTI * kPTJ * kPTK));
        ISIS_LAUNCH(kind, bytes, st,
                    (prolong_tiled<M, FM><<<blocks, kPTI * kPTJ * kPTK, 0, st>>>(L[l], C.x, (const T*)ws->x0[l + 1],
                                                                                  C.lg)));
        return ISIS_OK;
      }
    }
    ISIS_LAUNCH(kind, bytes, st,
                (prolong_correct<M, FM, T><<<nblk(nc, 256), 256, 0, st>>>(L[l], C.x, (const T*)ws->x0[l + 1],
                                                                          C.lg)));
    return ISIS_OK;
  }

  // Every level from l (N <= 16) down in one CTA (FP32 grids): see coarse_cycle.
  isis_status coarse_fused(int l) {
    if constexpr (sizeof(T) == 4) {
      const int last = (int)L.size() - 1;
      CoarseCycle cc;
      cc.nlev = last - l + 1;
      cc.nu1 = nu1;
      cc.nu2 = nu2;
      double bytes = 0.0;
      for (int q = 0; q < cc.nlev; ++q) {
        cc.L[q] = L[l + q];
        bytes += cells(L[l + q]) * sizeof(float) * (arrays(false) + (q == 0 ? 3 : 0));
      }
      const size_t smem = coarse_cycle_floats(L[l].N, L[last].N) * sizeof(float);
      // the largest cycle's shared memory, allowed once per instantiation and device
      static bool attr[64] = {};
      const int dev = ws->device >= 0 && ws->device < 64 ? ws->device : 0;
      if (!attr[dev]) {
        const size_t most = coarse_cycle_floats(kCVMaxN, 2) * sizeof(float);
        ISIS_CK(cudaFuncSetAttribute(coarse_cycle<M, FM>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)most));
        attr[dev] = true;
      }
      ISIS_LAUNCH(tk(KK_COARSE_CYCLE), bytes, st,
                  (coarse_cycle<M, FM><<<1, kCVThreads, smem, st>>>(cc, c, CoefT<float>(c), ws->iflags, ws->iflags + 1)));
    }
    return ISIS_OK;
  }

  isis_status vcycle(int l) {
    const int last = (int)L.size() - 1;
    if constexpr (sizeof(T) == 4) {
      if (L[l].N <= kCVMaxN && last - l + 1 <= kCVMaxLev) return coarse_fused(l);
    }
    if (l == last) {
      ISIS_LAUNCH(tk(KK_COARSE_NEWTON), 0.0, st,
                  (coarse_newton<M, FM, T><<<1, kCoarseMax, 0, st>>>(L[l], c, ws->iflags, ws->iflags + 1)));
      return ISIS_OK;
    }
    isis_status s = smooth(l, nu1);
    if (s != ISIS_OK) return s;
    LevelView<T>& C = L[l + 1];
    size_t nc = (size_t)C.N * C.N * C.N;
    double nf = cells(L[l]), ncd = (double)nc;
    const double rbytes = sizeof(T) * (nf * (1 + arrays(L[l].sig != nullptr)) + 3 * ncd);
    bool split = false;
    if constexpr (sizeof(T) == 4 && M == FOFR && FM == DELTA) split = L[l].N >= 64;
    if (split) {
      // f(R) correction form on grids of side >= 64: the stencils of 8 children hold too many per-cell inputs
      // and exponentials for one thread, so the residual of every cell goes through a scratch grid of the level
      // (the packed pair evaluation of the smoother), then the restriction reads it (measured at 512^3: 0.7
      // against 2.9 ms per force step on the coarse grids; the field form keeps the one-pass kernel, faster for
      // it)
      if constexpr (sizeof(T) == 4) {
        float* res = l == 0 ? (float*)ws->x0[0] : get_xalt(ws, l);
        if (!res) return ISIS_ENOMEM;
        const int kind = tk(l == 0 ? KK_RESTRICT_FINE : KK_RESTRICT_COARSE);
        ISIS_LAUNCH(kind, rbytes, st, (resid_rb2<M, FM><<<nblk((size_t)nf / 2, 256), 256, 0, st>>>(L[l], c, res)));
        ISIS_LAUNCH(kind, 0.0, st,
                    (restrict_xr<M, FM><<<nblk(nc, 256), 256, 0, st>>>(L[l], res, C, (float*)ws->x0[l + 1],
                                                                        (float*)ws->sig[l + 1])));
      }
    } else {
      bool done = false;
      if constexpr (sizeof(T) == 4 && M != FOFR) {
        if (C.N >= 4) {
          ISIS_LAUNCH(tk(l == 0 ? KK_RESTRICT_FINE : KK_RESTRICT_COARSE), rbytes, st,
                      (resid_restrict2<M, FM><<<nblk(nc / 2, 256), 256, 0, st>>>(L[l], c, C, (float*)ws->x0[l + 1],
                                                                                 (float*)ws->sig[l + 1])));
          done = true;
        }
      }
      if (!done)
        ISIS_LAUNCH(tk(l == 0 ? KK_RESTRICT_FINE : KK_RESTRICT_COARSE), rbytes, st,
                    (resid_restrict<M, FM, T><<<nblk(nc, 256), 256, 0, st>>>(L[l], c, C, (T*)ws->x0[l + 1],
                                                                            (T*)ws->sig[l + 1])));
    }
    bool paired = false;  // FP32 levels of side 4 or more: the paired gather
    if constexpr (sizeof(T) == 4) {
      if (C.N >= 4) {
        ISIS_LAUNCH(tk(KK_SIGMA), sizeof(T) * ncd * (2 + arrays(true)), st,
                    (sigma_rb2<M, FM><<<nblk(nc / 2, 256), 256, 0, st>>>(C, c, (float*)ws->sig[l + 1])));
        paired = true;
      }
    }
    if (!paired) {
      ISIS_LAUNCH(tk(KK_SIGMA), sizeof(T) * ncd * (2 + arrays(true)), st,
                  (coarse_sigma_add<M, FM, T><<<nblk(nc, 256), 256, 0, st>>>(C, c, (T*)ws->sig[l + 1])));
    }
    s = vcycle(l + 1);
    if (s != ISIS_OK) return s;
    s = prolong(l);
    if (s != ISIS_OK) return s;
    return smooth(l, nu2);
  }

  // Nested iteration (full multigrid start): the guess on level 0 is restricted to every level (R, the
  // full-approximation restriction); the coarsest level's own problem (Sigma = 0) is solved; then on each
  // finer level the coarse correction P(x_{l+1} - R x_l) is added to the restricted guess and one V-cycle
  // is run on that level's own problem.  Level 0 must be the finest level with no Sigma.
  isis_status fmg() {
    const int last = (int)L.size() - 1;
    for (int l = 1; l <= last; ++l) {
      LevelView<T>& C = L[l];
      size_t nc = (size_t)C.N * C.N * C.N;
      ISIS_LAUNCH(KK_SETUP, 9.0 * nc * sizeof(T), st,
                  (restrict_mean<T, T><<<nblk(nc, 256), 256, 0, st>>>(L[l - 1].x, C.x, C.lg)));
      ISIS_CK(cudaMemcpyAsync(ws->x0[l], C.x, nc * sizeof(T), cudaMemcpyDeviceToDevice, st));
      ISIS_CK(cudaMemsetAsync(ws->sig[l], 0, nc * sizeof(T), st));
    }
    isis_status s = vcycle(last);
    if (s != ISIS_OK) return s;
    for (int l = last - 1; l >= 0; --l) {
      LevelView<T>& C = L[l + 1];
      size_t nc = (size_t)C.N * C.N * C.N;
      (void)nc;
      s = prolong(l);
      if (s != ISIS_OK) return s;
      s = vcycle(l);
      if (s != ISIS_OK) return s;
    }
    return ISIS_OK;
  }

  // RMS of L(x) - Sigma on the finest level (blocking: one stream sync).
  isis_status fine_rms(double* out) {
    if constexpr (std::is_same<T, float>::value) {
      if (L[0].lg >= 3) {
        ISIS_LAUNCH(tk(KK_NORM), cells(L[0]) * sizeof(T) * (1 + arrays(L[0].sig != nullptr)), st,
                    (norm_rb2<M, FM><<<kNormBlocks, kNormThreads, 0, st>>>(L[0], c, ws->part)));
      } else {
        ISIS_LAUNCH(tk(KK_NORM), cells(L[0]) * sizeof(T) * (1 + arrays(L[0].sig != nullptr)), st,
                    (norm_partial<M, FM, T><<<kNormBlocks, kNormThreads, 0, st>>>(L[0], c, ws->part)));
      }
    } else {
      ISIS_LAUNCH(tk(KK_NORM), cells(L[0]) * sizeof(T) * (1 + arrays(L[0].sig != nullptr)), st,
                  (norm_partial<M, FM, T><<<kNormBlocks, kNormThreads, 0, st>>>(L[0], c, ws->part)));
    }
    ISIS_LAUNCH(KK_REDUCE, 0.0, st, (reduce_final<<<1, kNormThreads, 0, st>>>(ws->part, kNormBlocks, ws->scal)));
    double* h = (double*)ws->host;
    int* hi = (int*)(h + 4);
    ISIS_LAUNCH(KK_REDUCE, 0.0, st,
                (publish_scalars<<<1, 32, 0, st>>>(ws->scal, 1, ws->iflags, 2, ws->host_dev, (int*)(ws->host_dev + 4))));
    ISIS_CK(cudaStreamSynchronize(st));
    size_t n = (size_t)L[0].N * L[0].N * L[0].N;
    *out = std::sqrt(h[0] / (double)n);
    return coarse_status(hi[0]);
  }
};

// ---------------------------------------------------------------------------
// Reductions used by the drivers
// ---------------------------------------------------------------------------

// sum((v - shift)^2) and sum(v) over n values (blocking).
template <class T, bool kFast = false>
isis_status moments(Workspace* ws, const T* v, size_t n, double shift, cudaStream_t st, double* s2, double* s1) {
  ISIS_LAUNCH(KK_REDUCE, (double)n * sizeof(T), st,
              (moments_partial<T, kFast><<<kNormBlocks, kNormThreads, 0, st>>>(v, n, shift, ws->part, ws->part2)));
  ISIS_LAUNCH(KK_REDUCE, 0.0, st, (reduce_final<<<1, kNormThreads, 0, st>>>(ws->part, kNormBlocks, ws->scal)));
  ISIS_LAUNCH(KK_REDUCE, 0.0, st,
              (reduce_final<<<1, kNormThreads, 0, st>>>(ws->part2, kNormBlocks, ws->scal + 1)));
  double* h = (double*)ws->host;
  ISIS_LAUNCH(KK_REDUCE, 0.0, st,
              (publish_scalars<<<1, 32, 0, st>>>(ws->scal, 2, ws->iflags, 0, ws->host_dev, (int*)(ws->host_dev + 4))));
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
template <class T, bool kFast = false>
isis_status remove_mean(Workspace* ws, T* v, size_t n, cudaStream_t st) {
  ISIS_LAUNCH(KK_REDUCE, (double)n * sizeof(T), st,
              (moments_partial<T, kFast><<<kNormBlocks, kNormThreads, 0, st>>>(v, n, 0.0, ws->part, ws->part2)));
  ISIS_LAUNCH(KK_REDUCE, 0.0, st,
              (reduce_final<<<1, kNormThreads, 0, st>>>(ws->part2, kNormBlocks, ws->scal + 1)));
  ISIS_LAUNCH(KK_REDUCE, 2.0 * n * sizeof(T), st,
              (add_scalar<T><<<nblk(n, 256), 256, 0, st>>>(v, n, ws->scal + 1, 1.0 / (double)n)));
  return ISIS_OK;
}


// Row-major (caller, FP64 or FP32) <-> red/black split FP32 workspace.
template <class Tin>
__global__ void to_rb(const Tin* __restrict__ a, float* __restrict__ b, int lg) {
  size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= ((size_t)1 << (3 * lg))) return;
  const int m = (1 << lg) - 1;
  float v;
  if constexpr (sizeof(Tin) == 8) v = ff_split_bits((double)a[t]).hi;  // no FP64 unit (truncated to 24 bits)
  else v = (float)a[t];
  b[lidx<float>(lg, (int)(t >> (2 * lg)), (int)((t >> lg) & m), (int)(t & m))] = v;
}
template <class Tout>
__global__ void from_rb(const float* __restrict__ b, Tout* __restrict__ a, int lg) {
  size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= ((size_t)1 << (3 * lg))) return;
  const int m = (1 << lg) - 1;
  const float v = b[lidx<float>(lg, (int)(t >> (2 * lg)), (int)((t >> lg) & m), (int)(t & m))];
  if constexpr (sizeof(Tout) == 8) a[t] = f2d_bits(v);
  else a[t] = (Tout)v;
}

// b (red/black FP32) = a - shift, a row-major FP64, shift float-float (FP32 arithmetic only)
static __global__ void to_rb_shift(const double* __restrict__ a, float* __restrict__ b, int lg, float2 shift) {
  size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= ((size_t)1 << (3 * lg))) return;
  const int m = (1 << lg) - 1;
  b[lidx<float>(lg, (int)(t >> (2 * lg)), (int)((t >> lg) & m), (int)(t & m))] =
      ff_add(ff_split_bits(a[t]), ff_neg(ff_load(shift))).hi;
}
// a (row-major FP64) = shift + b, b red/black FP32 (one FP64 addition only when shift != 0)
static __global__ void from_rb_shift(const float* __restrict__ b, double* __restrict__ a, int lg, double shift) {
  size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= ((size_t)1 << (3 * lg))) return;
  const int m = (1 << lg) - 1;
  const double v = f2d_bits(b[lidx<float>(lg, (int)(t >> (2 * lg)), (int)((t >> lg) & m), (int)(t & m))]);
  a[t] = shift != 0.0 ? shift + v : v;
}
template <class T>
__global__ void exp_k(const T* __restrict__ a, T* __restrict__ b, size_t n) {
  size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t < n) b[t] = dexp<T>(a[t]);
}


// The FP32 value to_rb writes for an FP64 value (the significand cut to 24 bits, as ff_split_bits' high part;
// normal values).
inline float f32_cut(double d) {
  unsigned long long b;
  std::memcpy(&b, &d, sizeof b);
  b &= ~((1ull << 29) - 1ull);
  double t;
  std::memcpy(&t, &b, sizeof t);
  return (float)t;  // exact: 24 significant bits
}

__global__ void fill_f32(float* __restrict__ a, size_t n, float v);

// The field of the defect-correction loop, carried in float-float (row-major, 8 bytes per cell):
//   rb_to_ff   pff = shift + psi, psi the FP32 red/black field of the first phase (one exact float-float add);
//   update_ff  pff += e (minus its mean *emean for Poisson), FP32 instructions only;
//   ff_to_f64  phi = base + (hi + lo), the FP64 field returned to the caller.
// rb_to_ff and update_ff take one thread per four cells of a row (N^3/4 threads), ff_to_f64 one per two.
__global__ void rb_to_ff(const float* __restrict__ psi, float2* __restrict__ pff, int lg, float2 shift);
__global__ void update_ff(float2* __restrict__ pff, const float* __restrict__ e, int lg,
                          const float* __restrict__ emean);
__global__ void ff_to_f64(const float2* __restrict__ pff, double* __restrict__ phi, size_t n, double base,
                          int has_base);
// f(R): e^psi (float-float) of the carried psi = u - u_bar, two cells per thread (n even)
__global__ void fofr_exp_ff(const float2* __restrict__ psi, float2* __restrict__ E, size_t n,
                            const float2* __restrict__ tab, FFExp ek);
// *out = (float)(*sum * inv_n), one thread: the FP32 mean for the update (its threads then run no FP64
// arithmetic for it).
__global__ void mean_to_f32(const double* __restrict__ sum, double inv_n, float* __restrict__ out);

// Sum of an FP32 array on the device, left in ws->scal[1] (no host sync).
isis_status sum_f32(Workspace* ws, const float* v, size_t n, cudaStream_t st);

// Initial guess (isis_init): the background constant, or cell by cell the
// solution for a uniform density equal to the cell's eta (computed in FP32:
// it is only a starting point).
template <Model M, class T>
__global__ void init_guess(T* __restrict__ phi, const T* __restrict__ eta, size_t n, CoefT<float> c, int mode,
                           double bg) {
  size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n) return;
  if (mode == ISIS_INIT_BACKGROUND || M == POI) { phi[t] = (T)bg; return; }
  float e = (float)eta[t];
  if (M == SYM) {
    float v = 1.0f - c.s * e;
    phi[t] = (T)(v > 0.0f ? sqrtf(v) : 0.0f);
  } else {
    // S(u) = 0 at this eta: e^{u/(n+1)} = K2 / (K1 (eta - 1) + K3)
    float den = c.K1 * (e - 1.0f) + c.K3;
    phi[t] = (T)(c.np1 * logf(c.K2 / den));
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

// FP64-accurate residual of the finest grid for the defect-correction loop, in
// float-float (FP32 instruction throughput): r = -L(phi), written FP32 in the
// red/black layout with B = fp32(phi) and block partials of r^2.  Poisson and the
// symmetron here (the operator of Sect. 3.1, and of Eq. (symmetron_dimensionles)).
struct ResFF {
  float2 ih2;          // 1/h^2
  float2 K;            // Poisson: 1.5 Omega_m H0^2 / a; symmetron: A = a^2 / (2 lambda0^2)
  float2 s, eta_mean;  // symmetron: (a_SSB/a)^3; Poisson: mean density (float-float)
};
// r = -L(phi) in float-float from phi's float-float copy pff; B = the copy's high part (fp32 phi).
// Two cells per thread, (k, k+1) with k even, as the lanes of packed FP32x2 float-float arithmetic (ff2):
// the pair's own values and its i and j neighbours are 16-byte loads, the k neighbours outside the pair two
// 8-byte loads.  In the red/black output the pair's two cells sit at the same place of the two halves.
// phi_out (nullptr: none): the carried field written to FP64 as ff_to_f64 writes it, in the same pass.
__device__ __forceinline__ void write_f64_pair(double* __restrict__ phi, unsigned q, const ff2& v, double base,
                                               int has_base) {
  double d0 = ff_to_double_bits(v.hi.x, v.lo.x), d1 = ff_to_double_bits(v.hi.y, v.lo.y);
  if (has_base) {
    d0 += base;
    d1 += base;
  }
  if ((reinterpret_cast<uintptr_t>(phi) & 15u) == 0) {  // the caller's array: 8-byte alignment is all it promises
    reinterpret_cast<double2*>(phi)[q >> 1] = make_double2(d0, d1);
  } else {
    phi[q] = d0;
    phi[q + 1] = d1;
  }
}

template <Model M>
__global__ void __launch_bounds__(kNormThreads) outer_residual_ff(int lg, ResFF c, const double* __restrict__ eta,
                                                                  const float2* __restrict__ pff,
                                                                  float* __restrict__ r32, float* __restrict__ B32,
                                                                  double* __restrict__ part,
                                                                  double* __restrict__ phi_out) {
  // 32-bit positions: N <= 1024, so N^3 <= 2^30
  const unsigned np = 1u << (3 * lg - 1), half = np, m = (1u << lg) - 1u;
  const ff2 ih2 = ff2_bc(c.ih2), K = ff2_bc(c.K);
  float acc = 0.f;
  auto cid = [&](unsigned i, unsigned j, unsigned k) { return (((i << lg) | j) << lg) | k; };
  for (unsigned t = blockIdx.x * blockDim.x + threadIdx.x; t < np; t += gridDim.x * blockDim.x) {
    const unsigned q = 2 * t;
    const unsigned k = q & m, j = (q >> lg) & m, i = q >> (2 * lg);
    auto pair = [&](unsigned at) {
      const float4 v = *reinterpret_cast<const float4*>(pff + at);
      return ff2{make_float2(v.x, v.z), make_float2(v.y, v.w)};
    };
    const ff2 pc = pair(q);
    const float2 km = pff[cid(i, j, (k - 1) & m)], kp = pff[cid(i, j, (k + 2) & m)];
    const ff2 nb[6] = {pair(cid((i + 1) & m, j, k)), pair(cid((i - 1) & m, j, k)),
                       pair(cid(i, (j + 1) & m, k)), pair(cid(i, (j - 1) & m, k)),
                       ff2{make_float2(pc.hi.y, kp.x), make_float2(pc.lo.y, kp.y)},   // k + 1
                       ff2{make_float2(km.x, pc.hi.x), make_float2(km.y, pc.lo.x)}};  // k - 1
    // sd = sum (phi_nb - phi): each difference's high parts by an exact two-sum, the sum's high parts by
    // two-sums, low parts and rounding errors summed in FP32, normalised once (absolute accuracy about 2^-48
    // of the differences)
    ff2 sd = {f2_bc(0.f), f2_bc(0.f)};
    const float2 mh = make_float2(-pc.hi.x, -pc.hi.y);
#pragma unroll
    for (int d = 0; d < 6; ++d) {
      ff2 dp = ff2_two_sum(nb[d].hi, mh);
      dp.lo = f2_add(dp.lo, f2_sub(nb[d].lo, pc.lo));
      const ff2 ts = ff2_two_sum(sd.hi, dp.hi);
      sd = {ts.hi, f2_add(f2_add(sd.lo, dp.lo), ts.lo)};
    }
    sd = ff2_quick_two_sum(sd.hi, sd.lo);
    const ff2 lap = ff2_mul(sd, ih2);
    const ff2 et = ff2_pack(ff_split_bits(eta[q]), ff_split_bits(eta[q + 1]));  // the caller's array: 8-byte loads
    // F by Dekker's addition: absolute accuracy, F being small against its terms
    ff2 F;
    if constexpr (M == POI) {
      F = ff2_add_abs(lap, ff2_neg(ff2_mul(K, ff2_add_abs(et, ff2_neg(ff2_bc(c.eta_mean))))));
    } else {  // symmetron: L = lap - A [(s eta - 1) chi + chi^3]
      const ff2 qv = ff2_add_f(ff2_mul(ff2_bc(c.s), et), f2_bc(-1.0f));
      const ff2 x2 = ff2_mul(pc, pc);
      F = ff2_add_abs(lap, ff2_neg(ff2_mul(K, ff2_mul(ff2_add_abs(qv, x2), pc))));
    }
    const float2 r = f2_add(F.hi, F.lo);
    // cell k has colour (i + j + k) & 1, cell k + 1 the other; both at place q / 2 of their half
    const unsigned o0 = (((i + j) & 1u) ? half : 0u) + t, o1 = (((i + j) & 1u) ? 0u : half) + t;
    r32[o0] = -r.x;
    r32[o1] = -r.y;
    B32[o0] = pc.hi.x;
    B32[o1] = pc.hi.y;
    if (phi_out) write_f64_pair(phi_out, q, pc, 0.0, 0);
    acc = fmaf(F.hi.x, F.hi.x, acc);
    acc = fmaf(F.hi.y, F.hi.y, acc);
  }
  block_sum_store<double>((double)acc, part);
}

// f(R) residual in float-float (FP32 instruction throughput), two passes.
// Constants: psi = u - ub, C = e^ub, S = K1 (eta - 1) - Kx expm1(-psi/(n+1)) + dK.
struct FofrFF {
  double ub, inv_np1;
  float2 Cih2, K1, Kx, minv;  // C / h^2, K1, Kx = K2 e^{-ub/(n+1)}, -1/(n+1) (float-float)
  float2 ubff;                // ub (float-float)
  float dK;                   // K3 - Kx (zero up to rounding)
  FFExp ek;
};
__global__ void selftest_exp_ff(const double* __restrict__ x, double* __restrict__ y, int n,
                                const float2* __restrict__ tab, FFExp ek);
__global__ void selftest_ff_to_f64(const float* __restrict__ hl, double* __restrict__ out, int n);
// second pass: r = -L(u) (written FP32, red/black), B = fp32(u), block partials of r^2
__global__ void __launch_bounds__(kNormThreads) outer_residual_fofr_ff(int lg, FofrFF c,
                                                                       const double* __restrict__ eta,
                                                                       const float2* __restrict__ psi,
                                                                       const float2* __restrict__ E,
                                                                       const float2* __restrict__ tab,
                                                                       float* __restrict__ r32,
                                                                       float* __restrict__ B32,
                                                                       double* __restrict__ part,
                                                                       double* __restrict__ phi_out, double base);

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

  // FP32 grids work in the red/black layout of the workspace; FP64 in place
  const int lg = ilog2(A.N);
  T* xw = phi;
  const T* etaw = eta;
  if constexpr (sizeof(T) == 4) {
    xw = (T*)ws->x[0];
    etaw = (const T*)ws->eta[0];
    ISIS_LAUNCH(KK_SETUP, 8.0 * n, st, (to_rb<T><<<nblk(n, 256), 256, 0, st>>>(eta, (float*)ws->eta[0], lg)));
    ISIS_LAUNCH(KK_SETUP, 8.0 * n, st, (to_rb<T><<<nblk(n, 256), 256, 0, st>>>(phi, (float*)xw, lg)));
  }

  // density on the coarse levels
  for (int l = 1; l < ws->nlev; ++l) {
    int lgc = ilog2(A.N >> l);
    const T* f = l == 1 ? etaw : (const T*)ws->eta[l - 1];
    size_t ncl = (size_t)1 << (3 * lgc);
    ISIS_LAUNCH(KK_SETUP, 9.0 * ncl * sizeof(T), st,
                (restrict_mean<T, T><<<nblk(ncl, 256), 256, 0, st>>>(f, (T*)ws->eta[l], lgc)));
  }
  ISIS_CK(cudaMemsetAsync(ws->iflags, 0, 2 * sizeof(int), st));

  if (M == FOFR && kExpCache<T>)  // cached e^u of the finest level (FP64 grids)
    ISIS_LAUNCH(KK_SETUP, 2.0 * n * sizeof(T), st,
                (exp_k<T><<<nblk(n, 256), 256, 0, st>>>(xw, (T*)ws->aux[0], n)));

  Cycler<M, FIELD, T> cy;
  SolveArgs A2 = A;
  A2.coef = c;
  cy.setup(ws, A2, xw, etaw, nullptr);

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
  if constexpr (sizeof(T) == 4)
    ISIS_LAUNCH(KK_SETUP, 8.0 * n, st, (from_rb<T><<<nblk(n, 256), 256, 0, st>>>((const float*)xw, phi, lg)));
  if (A.info) *A.info = loc;
  return out;
}

// Relative residual (of the reference) below which the FP32 field-form
// cycles hand over to the FP64 defect correction, and the per-cycle
// reduction above which they are taken to have reached FP32 rounding.
constexpr double kSwitchRel = 2e-4;
constexpr double kStallRatio = 0.5;

// FP32 cycles + FP64 defect correction.
//  Phase 1: FAS V-cycles on the field in FP32 (psi = fp32(phi), for f(R)
//           psi = fp32(u - u_bar)) until the FP32-evaluated residual is below
//           kSwitchRel * ref or stalls.
//  Phase 2: outer loop: r = -L64(phi) in FP64; FP32 FAS V-cycles on the
//           correction e of L(B + e) - L(B) = r, B = fp32(phi) (DELTA form);
//           phi += e in FP64; until the FP64 residual is <= tol * ref.
template <Model M>
isis_status solve_refine(const SolveArgs& A) {
  Workspace* ws = get_workspace(A.N, sizeof(float), A.ncoarse);
  if (!ws) return ISIS_ENOMEM;
  if (!ensure_fofr64(ws)) return ISIS_ENOMEM;  // float-float scratch of the FP64-accurate residual
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

  const int lg = ilog2(A.N);
  double s2, s1;
  // the density's moments and its FP32 red/black copy in one pass
  {
    ISIS_LAUNCH(KK_SETUP, 12.0 * n, st,
                (moments_to_rb<<<kNormBlocks, kNormThreads, 0, st>>>(eta64, eta0, lg, ws->part, ws->part2)));
    ISIS_LAUNCH(KK_REDUCE, 0.0, st, (reduce_final<<<1, kNormThreads, 0, st>>>(ws->part, kNormBlocks, ws->scal)));
    ISIS_LAUNCH(KK_REDUCE, 0.0, st,
                (reduce_final<<<1, kNormThreads, 0, st>>>(ws->part2, kNormBlocks, ws->scal + 1)));
    ISIS_LAUNCH(KK_REDUCE, 0.0, st,
                (publish_scalars<<<1, 32, 0, st>>>(ws->scal, 2, ws->iflags, 0, ws->host_dev,
                                                   (int*)(ws->host_dev + 4))));
    ISIS_CK(cudaStreamSynchronize(st));
    s2 = ((double*)ws->host)[0];
    s1 = ((double*)ws->host)[1];
  }
  isis_status s = ISIS_OK;
  double eta_mean = s1 / (double)n;
  if (M == POI) {
    c.eta_mean = eta_mean;
    s2 = s2 - (double)n * (eta_mean - 1.0) * (eta_mean - 1.0);
    if (s2 < 0) s2 = 0;
  }
  double ref = A.ref_scale * std::sqrt(s2 / (double)n);
  // a background start is written straight into the FP32 field of phase 1 (phi64 is written when the solve
  // ends)
  const bool bg_start = A.init == ISIS_INIT_BACKGROUND;
  if (!bg_start) {
    s = apply_init<M, double>(A, c, phi64, eta64, n);
    if (s != ISIS_OK) return s;
  }
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
  // f(R) runs in the shifted variable psi = u - u_bar (u_bar the background, S(u_bar) = 0 at
  // eta = 1): the source S = K1 (eta - 1) - K3 expm1(-psi/(n+1)) no longer cancels two large
  // terms and psi is small, so FP32 rounding stalls the cycles far later than in u itself.
  const double u0 = (M == FOFR) ? background_value<FOFR>(c) : 0.0;
  SolveArgs A1 = A2;
  if (M == FOFR) {
    A1.coef.fscale = std::exp(u0);
    A1.coef.fKx = c.K2 * std::exp(-u0 * c.inv_np1);
    A1.coef.fK3x = c.K3 - A1.coef.fKx;
  }
  // the FP32 field of phase 1 from the caller's FP64 field (phi64 is not written until the solve ends)
  auto start_field = [&]() -> isis_status {
    if (bg_start) {
      // f(R) and Poisson start at psi = 0 (u = u_bar, Phi = 0); the symmetron at fp32(chi_bg)
      const float v = M == SYM ? f32_cut(background_value<SYM>(c)) : 0.0f;
      ISIS_LAUNCH(KK_INIT, 4.0 * n, st, (fill_f32<<<nblk(n / 4, 256), 256, 0, st>>>(B0, n, v)));
      return ISIS_OK;
    }
    if (M == FOFR)
      ISIS_LAUNCH(KK_SETUP, 12.0 * n, st,
                  (to_rb_shift<<<nblk(n, 256), 256, 0, st>>>(phi64, B0, lg, ff_split_host(u0))));
    else
      ISIS_LAUNCH(KK_SETUP, 12.0 * n, st, (to_rb<double><<<nblk(n, 256), 256, 0, st>>>(phi64, B0, lg)));
    return ISIS_OK;
  };
  s = start_field();
  if (s != ISIS_OK) return s;
  {
    Cycler<M, FIELD, float> cy;
    cy.setup(ws, A1, B0, eta0, nullptr);
    double res;
    if (bg_start && ref > 0.0) {
      // The background field's residual is the reference itself, in closed form: -ref_scale (eta - <eta>) for
      // Poisson at Phi = 0, -A s chi_bg (eta - 1) for the symmetron at chi_bg (chi_bg^2 = 1 - s), -K1 (eta - 1)
      // for f(R) and the chameleon at their background (S vanishes there at eta = 1).  No norm pass.
      res = ref;
    } else {
      s = cy.fine_rms(&res);
      if (s != ISIS_OK) return s;
    }
    loc.res0 = res;
    if (!(ref > 0.0)) ref = res;
    loc.res_ref = ref;
    double prev = res;
    double handover = std::fmax(A.tol, kSwitchRel) * ref;
    bool nested = A.fmg != 0, after_nested = false;
    while (res > handover && loc.cycles < A.max_cycles && std::isfinite(res)) {
      if (nested) {
        // the nested-iteration start leaves the residual near 1e-2 of the reference, far above the handover:
        // the next V-cycle follows without a norm in between
        nested = false;
        after_nested = true;
        s = cy.fmg();
        if (s != ISIS_OK) return s;
        loc.cycles += 1;
        if (loc.cycles >= A.max_cycles) break;
        if (handover < 1e-3 * ref) {
          // and a V(2,1) cycle contracts it by about 0.1: a second V-cycle follows without a norm as well (the
          // check of the start below then comes one cycle later)
          s = cy.vcycle(0);
          if (s != ISIS_OK) return s;
          loc.cycles += 1;
          if (loc.cycles >= A.max_cycles) break;
        }
      }
      s = cy.vcycle(0);
      if (s != ISIS_OK) return s;
      s = cy.fine_rms(&res);
      loc.cycles += 1;
      if (nh < 128) loc.hist[nh++] = res;
      loc.nhist = nh;
      if (after_nested) {
        after_nested = false;
        if (s != ISIS_OK || !std::isfinite(res) || res > loc.res0) {
          // The nested start solves each coarse grid's own problem from the restricted density.  Where a coarse
          // cell is wide against the field's range (6/h^2 below the source's slope), its Newton-Gauss-Seidel
          // denominator can change sign and the start diverges (the symmetron near symmetry breaking on
          // strongly clustered densities).  It is only an acceleration: the phase restarts from the caller's
          // field with plain V-cycles, and the fixed point is unchanged.
          ISIS_CK(cudaMemsetAsync(ws->iflags, 0, 2 * sizeof(int), st));
          s = start_field();
          if (s != ISIS_OK) return s;
          res = prev = loc.res0;
          continue;
        }
      }
      if (s != ISIS_OK) {
        // the last iterate to the caller (from the FP32 field of this phase)
        ISIS_LAUNCH(KK_SETUP, 12.0 * n, st,
                    (from_rb_shift<<<nblk(n, 256), 256, 0, st>>>(cy.L[0].x, phi64, lg, u0)));
        if (A.info) *A.info = loc;
        return s;
      }
      if (!(res <= kStallRatio * prev)) break;
      prev = res;
    }
    if (!std::isfinite(res)) {
      loc.res_final = res;
      if (A.info) *A.info = loc;
      return ISIS_ENAN;
    }
    const float* psi = cy.L[0].x;
    // The field of phase 2 is carried in float-float (ws->b64): phi for Poisson and the symmetron, psi = u - u_bar
    // for f(R).  Poisson gauge: the residual does not see the mean, so it is removed once per phase; here from
    // the FP32 field's mean, in the conversion.
    float2 shift = make_float2(0.f, 0.f);
    if (M == POI) {
      s = sum_f32(ws, psi, n, st);
      if (s != ISIS_OK) return s;
      // read through the mapped readback area, as the norms are (no copy engine)
      ISIS_LAUNCH(KK_REDUCE, 0.0, st,
                  (publish_scalars<<<1, 32, 0, st>>>(ws->scal, 2, ws->iflags, 0, ws->host_dev,
                                                     (int*)(ws->host_dev + 4))));
      ISIS_CK(cudaStreamSynchronize(st));
      shift = ff_split_host(-((double*)ws->host)[1] / (double)n);
    }
    ISIS_LAUNCH(KK_SETUP, 12.0 * n, st,
                (rb_to_ff<<<nblk(n / 4, 256), 256, 0, st>>>(psi, reinterpret_cast<float2*>(ws->b64), lg, shift)));
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
  F64.aux = nullptr;

  Cycler<M, DELTA, float> cy;
  cy.setup(ws, A2, e0, eta0, r0);
  ResFF rff{};
  rff.ih2 = ff_split_host(F64.ih2);
  rff.K = ff_split_host(M == POI ? c.KP : c.A);
  rff.s = ff_split_host(c.s);
  rff.eta_mean = ff_split_host(c.eta_mean);
  FofrFF ffc{};
  if (M == FOFR) {
    const double ub = background_value<FOFR>(c), Kx = c.K2 * std::exp(-ub * c.inv_np1);
    ffc.ub = ub;
    ffc.inv_np1 = c.inv_np1;
    ffc.Cih2 = ff_split_host(std::exp(ub) * F64.ih2);
    ffc.K1 = ff_split_host(c.K1);
    ffc.Kx = ff_split_host(Kx);
    ffc.minv = ff_split_host(-c.inv_np1);
    ffc.ubff = ff_split_host(ub);
    ffc.dK = (float)(c.K3 - Kx);
    ffc.ek = ff_exp_consts();
  }

  double* h = (double*)ws->host;
  int* hi = (int*)(h + 4);
  isis_status out = ISIS_ENOCONV;
  const double target = A.tol * ref;
  double prev_res = 0.0;
  int prev_k = 0;
  bool written = false;  // the caller's FP64 field holds the carried field
  for (int outer = 0;; ++outer) {
    // r = -L(phi) to FP64 accuracy from the carried float-float field, B = its FP32 value, RMS of r.  After a
    // correction the pass also writes the field to the caller's FP64 array: it is the answer whenever this
    // residual ends the loop (a residual that does not only costs the write).
    float2* carry = reinterpret_cast<float2*>(ws->b64);
    double* wout = outer > 0 ? phi64 : nullptr;
    if (M == FOFR) {
      float2* E_ff = reinterpret_cast<float2*>(ws->s64);
      ISIS_LAUNCH(kind_tag(KK_OUTER_RESID, (int)M, (int)FIELD), 16.0 * n, st,
                  (fofr_exp_ff<<<nblk(n / 2, 256), 256, 0, st>>>(carry, E_ff, n, ws->exptab_ff, ffc.ek)));
      ISIS_LAUNCH(kind_tag(KK_OUTER_RESID, (int)M, (int)FIELD), (wout ? 40.0 : 32.0) * n, st,
                  (outer_residual_fofr_ff<<<kNormBlocks, kNormThreads, 0, st>>>(F64.lg, ffc, eta64, carry, E_ff,
                                                                                 ws->exptab_ff, r0, B0, ws->part,
                                                                                 wout, u0)));
    } else {
      // phi_ff and eta read, r and B written: 24 bytes per cell (and the FP64 field, 8 more)
      ISIS_LAUNCH(kind_tag(KK_OUTER_RESID, (int)M, (int)FIELD), (wout ? 32.0 : 24.0) * n, st,
                  (outer_residual_ff<M><<<kNormBlocks, kNormThreads, 0, st>>>(F64.lg, rff, eta64, carry, r0, B0,
                                                                              ws->part, wout)));
    }
    ISIS_LAUNCH(KK_REDUCE, 0.0, st, (reduce_final<<<1, kNormThreads, 0, st>>>(ws->part, kNormBlocks, ws->scal)));
    ISIS_LAUNCH(KK_REDUCE, 0.0, st,
                (publish_scalars<<<1, 32, 0, st>>>(ws->scal, 1, ws->iflags, 2, ws->host_dev, (int*)(ws->host_dev + 4))));
    ISIS_CK(cudaStreamSynchronize(st));
    written = wout != nullptr;
    double res = std::sqrt(h[0] / (double)n);
    if (outer > 0 && nh < 128) loc.hist[nh++] = res;
    loc.nhist = nh;
    loc.res_final = res;
    loc.outer = outer;
    if (hi[0] != 0) { out = coarse_status(hi[0]); break; }
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
    ISIS_CK(cudaMemsetAsync(cy.L[0].x, 0, n * sizeof(float), st));
    // inner_cycles FP32 cycles; after the first outer iteration, only as many
    // as the measured contraction per cycle says reach half the target
    int k = A.inner;
    if (prev_res > 0.0 && prev_k > 0 && res < prev_res) {
      const double rho = std::pow(res / prev_res, 1.0 / prev_k);
      if (rho > 0.0 && rho < 1.0) {
        const double need = std::ceil(std::log(0.5 * target / res) / std::log(rho));
        if (need >= 1.0 && need < (double)k) k = (int)need;
      }
    }
    if (loc.cycles + k > A.max_cycles) k = A.max_cycles - loc.cycles;
    prev_res = res;
    prev_k = k;
    for (int it = 0; it < k; ++it) {
      s = cy.vcycle(0);
      if (s != ISIS_OK) return s;
    }
    loc.cycles += k;
    const float* ecur = cy.L[0].x;
    const float* emean = nullptr;
    if (M == POI) {  // the gauge: each correction enters with its mean removed
      s = sum_f32(ws, ecur, n, st);
      if (s != ISIS_OK) return s;
      float* mf = reinterpret_cast<float*>(ws->scal + 2);
      ISIS_LAUNCH(KK_REDUCE, 0.0, st, (mean_to_f32<<<1, 32, 0, st>>>(ws->scal + 1, 1.0 / (double)n, mf)));
      emean = mf;
    }
    ISIS_LAUNCH(KK_UPDATE, 20.0 * n, st, (update_ff<<<nblk(n / 4, 256), 256, 0, st>>>(carry, ecur, lg, emean)));
  }
  // the carried field to the caller: phi = hi + lo (f(R): u = u_bar + psi), in FP64, unless the last residual
  // pass wrote it
  if (!written) {
    ISIS_LAUNCH(KK_UPDATE, 16.0 * n, st,
                (ff_to_f64<<<nblk(n / 2, 256), 256, 0, st>>>(reinterpret_cast<const float2*>(ws->b64), phi64, n,
                                                             M == FOFR ? u0 : 0.0, M == FOFR ? 1 : 0)));
  }
  if (A.info) *A.info = loc;
  return out;
}

}  // namespace isis
