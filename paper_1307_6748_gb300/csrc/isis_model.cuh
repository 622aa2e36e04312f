// isis_model.cuh -- per-cell operator L, its diagonal derivative and the
// Newton-Gauss-Seidel update for the three equations of the ISIS solver
// (Llinares, Mota & Winther 2013, arXiv:1307.6748).
//
//   Poisson   L(Phi) = lap Phi - KP (eta - <eta>)        Sect. 3.1, Eq. (disc_lap)
//   symmetron L(chi) = lap chi - A[(s eta - 1) chi + chi^3]
//                                                         Sect. 4.1, Eq. (symmetron_dimensionles)
//   f(R)      L(u)   = h^-2 sum_f b_f (u_nb - u) - S(u),  b_f = (e^u + e^u_nb)/2
//             S(u)   = K1 (eta - 1) - K2 e^{-u/(n+1)} + K3
//                                                         Sect. 3.4 Eq. (disc_non_canonical), Sect. 4.2
//   update    x <- x - (L - Sigma) / (dL/dx)              Sect. 3.2
//   dL/dx     canonical: -6/h^2 - dS/dx                    Sect. 3.3
//             f(R): h^-2 sum_f [-b_f + (e^u/2)(u_nb - u)] - dS/du
//                   (Eq. (dbeq) with the exact factor 1/2 of the face average)
//
// Two forms of every operator:
//   FIELD  the unknown x is the field itself (phi, chi or u).
//   DELTA  the unknown x = e is a correction about a fixed base field B:
//          N_B(e) = L(B + e) - L(B), written so that no large terms cancel
//          (used by the FP32 inner cycles of the FP64 defect-correction loop).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace isis {

enum Model : int { POI = 0, SYM = 1, FOFR = 2 };
enum Form : int { FIELD = 0, DELTA = 1 };

// Constants of the source terms; host code fills them from the physical
// parameters (see isis_api.cu).
struct Coef {
  double A, s;          // symmetron: A = a^2/(2 lambda0^2), s = (a_SSB/a)^3
  double K1, K2, K3;    // f(R) source constants (Sect. 4.2)
  // f(R) field form in a shifted variable x = u - u0 (u0 = 0: x = u):
  //   b = fscale e^x with fscale = e^{u0};
  //   S = K1 (eta - 1) - fKx expm1(-x/(n+1)) + fK3x with fKx = K2 e^{-u0/(n+1)}, fK3x = K3 - fKx.
  // With u0 the background (fK3x = 0) the two large source terms no longer cancel.
  double fscale, fKx, fK3x;
  double np1, inv_np1;  // n + 1 and its inverse
  double KP, eta_mean;  // Poisson: KP = 1.5 Om H0^2 / a, mean density
};

// The same constants in a kernel's own precision.  The FP32 kernels receive them rounded to FP32 once on the host
// (the launch converts a Coef argument): converted per thread, each would be an FP64-to-FP32 conversion on the
// narrow FP64 pipe of this part.  CoefT<double> holds the values unchanged.
template <class T>
struct CoefT {
  T A, s, K1, K2, K3, fscale, fKx, fK3x, np1, inv_np1, KP, eta_mean;
  CoefT() = default;
  __host__ __device__ CoefT(const Coef& c)
      : A((T)c.A), s((T)c.s), K1((T)c.K1), K2((T)c.K2), K3((T)c.K3), fscale((T)c.fscale), fKx((T)c.fKx),
        fK3x((T)c.fK3x), np1((T)c.np1), inv_np1((T)c.inv_np1), KP((T)c.KP), eta_mean((T)c.eta_mean) {}
};

// Values of one cell and its six neighbours, in the order
// (i+1, i-1, j+1, j-1, k+1, k-1).
template <class T>
struct Cell {
  T x, xn[6];      // unknown
  T eta, sig;      // density and FAS source
  T B, Bn[6];      // base field (DELTA form)
  T w, wn[6];      // e^B (f(R) DELTA form)
  T a, an[6];      // f(R): cached b = e^x (FIELD) or m = e^B expm1(e) (DELTA)
};

template <class T> __device__ __forceinline__ T dexp(T v);
template <> __device__ __forceinline__ double dexp<double>(double v) { return exp(v); }
template <> __device__ __forceinline__ float dexp<float>(float v) { return __expf(v); }
template <class T> __device__ __forceinline__ T dexpm1(T v);
template <> __device__ __forceinline__ double dexpm1<double>(double v) { return expm1(v); }
// FP32 e^v - 1: Taylor series to degree 3 for |v| <= 2^-7 (truncation below 2.0e-8
// relative, a third of an FP32 ulp: the corrections of the refinement loop live there), to
// degree 8 for |v| <= 1/2 (below 1.4e-8 relative), else expf(v) - 1 (no cancellation beyond
// a factor 3).
template <> __device__ __forceinline__ float dexpm1<float>(float v) {
  if (fabsf(v) <= 0.0078125f) {
    float p = fmaf(v, 1.0f / 6.0f, 0.5f);
    p = fmaf(p, v, 1.0f);
    return p * v;
  }
  if (fabsf(v) <= 0.5f) {
    float p = fmaf(v, 1.0f / 40320.0f, 1.0f / 5040.0f);
    p = fmaf(p, v, 1.0f / 720.0f);
    p = fmaf(p, v, 1.0f / 120.0f);
    p = fmaf(p, v, 1.0f / 24.0f);
    p = fmaf(p, v, 1.0f / 6.0f);
    p = fmaf(p, v, 0.5f);
    p = fmaf(p, v, 1.0f);
    return p * v;
  }
  return expf(v) - 1.0f;
}

// f(R) in the field form with b = e^x of the cell and its neighbours given:
//   F  = h^-2 sum_f b_f (x_nb - x) - S(x) - Sigma,   b_f = (b + b_nb)/2
//   dF = h^-2 sum_f [ (b/2)(x_nb - x) - b_f ] - dS/dx
// with x the shifted variable and b = fscale e^x (ex, exn: the cached e^x of the cell and its neighbours).
template <class T, class CT>
__device__ __forceinline__ void fofr_field_eval(const CT& c, T ih2, T x, T ex, const T* xn, const T* exn, T eta,
                                                T sig, T& F, T& dF) {
  // sums with e^x and e^x_nb, scaled by fscale once
  T flux = 0, dsum = 0;
#pragma unroll
  for (int d = 0; d < 6; ++d) {
    T du = xn[d] - x;
    T ef = T(0.5) * (ex + exn[d]);
    flux += ef * du;
    dsum += T(0.5) * ex * du - ef;
  }
  const T bs = T(c.fscale);
  flux *= bs;
  dsum *= bs;
  T Kx = T(c.fKx), inp1 = T(c.inv_np1);
  T em = dexpm1<T>(-x * inp1);
  T S = T(c.K1) * (eta - T(1)) - Kx * em + T(c.fK3x);
  F = flux * ih2 - S - sig;
  dF = dsum * ih2 - Kx * inp1 * (em + T(1));
}

// f(R) in the correction form about the base B, with m = e^B expm1(e) and
// bt = e^{B+e} = e^B + m of the cell and its neighbours given:
//   N_B(e) = h^-2 sum_f { (m + m_nb)/2 (B_nb - B) + (bt + bt_nb)/2 (e_nb - e) }
//            + K2 e^{-B/(n+1)} expm1(-e/(n+1))
template <class T, class CT>
__device__ __forceinline__ void fofr_delta_eval(const CT& c, T ih2, T e, T B, T m, T bt, const T* en, const T* Bn,
                                                const T* mn, const T* btn, T sig, T& F, T& dF) {
  T flux = 0, dsum = 0;
#pragma unroll
  for (int d = 0; d < 6; ++d) {
    T dB = Bn[d] - B, de = en[d] - e;
    T bf = T(0.5) * (bt + btn[d]);
    flux += T(0.5) * (m + mn[d]) * dB + bf * de;
    dsum += T(0.5) * bt * (dB + de) - bf;
  }
  T K2 = T(c.K2), inp1 = T(c.inv_np1);
  T exB = dexp<T>(-B * inp1), em = dexpm1<T>(-e * inp1);
  F = flux * ih2 + K2 * exB * em - sig;
  dF = dsum * ih2 - K2 * inp1 * exB * (em + T(1));
}

// F = L(x) - Sigma and dF = dL/dx at one cell (c: Coef or CoefT).
template <Model M, Form FM, class T, class CT>
__device__ __forceinline__ void eval_cell(const CT& c, T ih2, const Cell<T>& q, T& F, T& dF) {
  if constexpr (M == POI) {
    T lap = (((q.xn[0] + q.xn[1]) + (q.xn[2] + q.xn[3])) + (q.xn[4] + q.xn[5]) - T(6) * q.x) * ih2;
    if constexpr (FM == FIELD) F = lap - T(c.KP) * (q.eta - T(c.eta_mean)) - q.sig;
    else F = lap - q.sig;  // linear: N(e) = lap e
    dF = T(-6) * ih2;
  } else if constexpr (M == SYM) {
    T lap = (((q.xn[0] + q.xn[1]) + (q.xn[2] + q.xn[3])) + (q.xn[4] + q.xn[5]) - T(6) * q.x) * ih2;
    T A = T(c.A), sm1 = T(c.s) * q.eta - T(1);
    if constexpr (FM == FIELD) {
      T x2 = q.x * q.x;
      F = lap - A * (sm1 + x2) * q.x - q.sig;
      dF = T(-6) * ih2 - A * (sm1 + T(3) * x2);
    } else {
      // (B+e)^3 - B^3 = e (3B^2 + 3Be + e^2)
      T e = q.x, B = q.B;
      T cub = e * (T(3) * B * B + e * (T(3) * B + e));
      F = lap - A * (sm1 * e + cub) - q.sig;
      T u = B + e;
      dF = T(-6) * ih2 - A * (sm1 + T(3) * u * u);
    }
  } else {  // FOFR: the per-cell exponentials come from the cached q.a, q.an
    if constexpr (FM == FIELD) {
      fofr_field_eval<T>(c, ih2, q.x, q.a, q.xn, q.an, q.eta, q.sig, F, dF);
    } else {
      T btn[6];
#pragma unroll
      for (int d = 0; d < 6; ++d) btn[d] = q.wn[d] + q.an[d];
      fofr_delta_eval<T>(c, ih2, q.x, q.B, q.a, q.w + q.a, q.xn, q.Bn, q.an, btn, q.sig, F, dF);
    }
  }
}

// Whether the operator reads the density: not in the correction forms of Poisson
// (linear) and f(R) (eta enters only its right-hand side).
template <Model M, Form FM>
__host__ __device__ constexpr bool uses_eta() { return !(FM == DELTA && M != SYM); }

// The per-cell exponential of f(R) for a cell holding x (and e^B = w).
template <Model M, Form FM, class T>
__device__ __forceinline__ T aux_of(T x, T w) {
  if constexpr (M == FOFR && FM == FIELD) return dexp<T>(x);
  if constexpr (M == FOFR && FM == DELTA) return w * dexpm1<T>(x);
  (void)x;
  (void)w;
  return T(0);
}

// Off-diagonal Jacobian entry dF_c/dx_nb for neighbour direction d (used by
// the dense coarsest-level Newton solve).  f(R): b = e^u of the cell and of its
// neighbour from the cell's cached exponentials (q.a, q.an: e^x in the field
// form, with b = fscale e^x; e^B expm1(e) in the correction form, with
// b = e^B + e^B expm1(e) = e^{B+e}), which the caller has filled.
template <Model M, Form FM>
__device__ __forceinline__ double eval_offdiag(const Coef& c, double ih2, const Cell<double>& q, int d) {
  (void)c;
  if constexpr (M == FOFR) {
    double u = (FM == FIELD) ? q.x : q.B + q.x;
    double un = (FM == FIELD) ? q.xn[d] : q.Bn[d] + q.xn[d];
    const double bu = (FM == FIELD) ? c.fscale * q.a : q.w + q.a;
    const double bn = (FM == FIELD) ? c.fscale * q.an[d] : q.wn[d] + q.an[d];
    return (0.5 * (bu + bn) + 0.5 * bn * (un - u)) * ih2;
  } else {
    return ih2;
  }
}

}  // namespace isis
