// isis_particles.cu -- CIC density estimate (Sect. 5.1) and the forces on
// particles (Sect. 4.1 Eq. (symmetron_geodesics_tilde_chi), Sect. 4.2).
//
// CIC convention (not fixed by the paper): positions in cell units, cell
// centres at i + 1/2; along each axis a particle at x gives weight 1 - t to
// cell floor(x - 1/2) and t to the next cell, t = (x - 1/2) - floor(x - 1/2);
// periodic wrap.  The 3-D weight is the product of the three.
#include <cmath>
#include <mutex>

#include "isis_solver.cuh"

namespace isis {

unsigned long long* get_deposit_buf(int N);
float* get_force_buf(int N);

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

// Exact per-axis CIC weights in units of 2^-23 for 1 <= x < N (every float
// there is a multiple of 2^-23, so floor, the offset t and 1 - t are exact).
// Returns false outside that range (those particles take the FP64 path).
__device__ __forceinline__ bool cic_axis_fix(float x, int N, int& i0, unsigned& w0, unsigned& w1) {
  if (!(x >= 1.0f && x < (float)N)) return false;
  const float xi = floorf(x), fx = x - xi;
  float t;
  if (fx >= 0.5f) { i0 = (int)xi; t = fx - 0.5f; }
  else { i0 = (int)xi - 1; t = fx + 0.5f; }
  w1 = (unsigned)(t * 8388608.0f);  // exact: t is a multiple of 2^-23
  w0 = 8388608u - w1;
  return true;
}

// (a b c) 2^-69 in units of 2^-40, truncated; a, b, c <= 2^23.
__device__ __forceinline__ unsigned long long fix3(unsigned a, unsigned b, unsigned c) {
  const unsigned long long ab = (unsigned long long)a * b;  // <= 2^46, exact
  const unsigned long long lo = ab * c, hi = __umul64hi(ab, (unsigned long long)c);
  return (hi << 35) | (lo >> 29);
}

__global__ void cic_scatter(const float* __restrict__ x, const float* __restrict__ y, const float* __restrict__ z,
                            long long np, int lg, unsigned long long* __restrict__ acc) {
  long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= np) return;
  const int N = 1 << lg, m = N - 1;
  const float px = x[p], py = y[p], pz = z[p];
  int ii, jj, kk;
  unsigned wi[2], wj[2], wk[2];
  if (cic_axis_fix(px, N, ii, wi[0], wi[1]) && cic_axis_fix(py, N, jj, wj[0], wj[1]) &&
      cic_axis_fix(pz, N, kk, wk[0], wk[1])) {
    // all-integer path: exact weights, exact products, truncation to 2^-40
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
      for (int b = 0; b < 2; ++b)
#pragma unroll
        for (int d = 0; d < 2; ++d) {
          const unsigned long long q = fix3(wi[a], wj[b], wk[d]);
          if (q) atomicAdd(&acc[cidx(lg, (ii + a) & m, (jj + b) & m, (kk + d) & m)], q);
        }
    return;
  }
  // positions in [0, 1) or outside [0, N): FP64 weights, truncated to 2^-40
  Axis ax = cic_axis(px, N), ay = cic_axis(py, N), az = cic_axis(pz, N);
  const int is[2] = {ax.i0, ax.i1}, js[2] = {ay.i0, ay.i1}, ks[2] = {az.i0, az.i1};
  const double wx[2] = {ax.w0, ax.w1}, wy[2] = {ay.w0, ay.w1}, wz[2] = {az.w0, az.w1};
#pragma unroll
  for (int a = 0; a < 2; ++a)
#pragma unroll
    for (int b = 0; b < 2; ++b)
#pragma unroll
      for (int d = 0; d < 2; ++d) {
        const unsigned long long q = (unsigned long long)(wx[a] * wy[b] * wz[d] * kFix);
        if (q) atomicAdd(&acc[cidx(lg, is[a], js[b], ks[d])], q);
      }
}

// u 2^e2 rounded to FP64 as (double)u * 2^e2 rounds it (to nearest even, the power-of-two product exact), by
// integer operations: the conversion and the multiply would run on the narrow FP64 pipe.  Normal results only
// (e2 > -960 for the densities here).
__device__ __forceinline__ double u64_scaled_to_double(unsigned long long u, int e2) {
  if (u == 0ull) return 0.0;
  const int top = 63 - __clzll((long long)u);  // position of the leading one
  unsigned long long M;
  int E = top + e2;
  if (top <= 52) {
    M = u << (52 - top);
  } else {
    const int sh = top - 52;
    M = u >> sh;
    const unsigned long long rem = u & ((1ull << sh) - 1ull), half = 1ull << (sh - 1);
    if (rem > half || (rem == half && (M & 1ull))) ++M;
    if (M >> 53) {
      M >>= 1;
      ++E;
    }
  }
  return __longlong_as_double((long long)(((unsigned long long)(E + 1023) << 52) | (M & 0xFFFFFFFFFFFFFull)));
}

// eta = acc * scale.  pow2 != 0: scale = 2^e2 exactly (the particle count is the cell count times a power of
// two, the usual PM set-up), converted by integer operations, bit for bit the FP64 result.
template <class T>
__global__ void cic_finish(const unsigned long long* __restrict__ acc, T* __restrict__ eta, size_t n, double scale,
                           int pow2, int e2) {
  size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n) return;
  if (sizeof(T) == 8 && pow2) eta[t] = (T)u64_scaled_to_double(acc[t], e2);
  else eta[t] = (T)((double)acc[t] * scale);
}

// Whether scale is an exact power of two 2^e2 (host).
inline bool exact_pow2(double scale, int* e2) {
  int e = 0;
  const double mant = std::frexp(scale, &e);  // scale = mant 2^e, mant in [1/2, 1)
  if (mant != 0.5) return false;
  *e2 = e - 1;
  return *e2 > -960 && *e2 < 960;
}

// Grid force at every cell (one pass):
//   f_d(c) = [a^2 (Phi(c+e_d) - Phi(c-e_d)) + pref(c) (phi(c+e_d) - phi(c-e_d))] / (2h)
//   pref = C_s a^2 chi(c) (symmetron, Eq. (symmetron_geodesics_tilde_chi) with chi~ = a chi),
//          C_s e^u(c) (the b = e^u models: C_s = 1/2 for f(R), Sect. 4.2; a^2 beta phi_0 / M_pl for
//          the chameleon), 0 without a scalar field.
// The differences keep the field's digits (FP64 fields through their float-float
// splits, see fdiff), the products are FP32 (the output is FP32).
// a - b rounded to FP32.  FP64 fields: from the float-float splits of a and b by integer operations, so no
// FP64 instruction runs (GB300 has few FP64 units); (a.hi - b.hi) + (a.lo - b.lo) carries the difference to
// FP32 accuracy.
template <class T>
__device__ __forceinline__ float fdiff(T a, T b) {
  if constexpr (sizeof(T) == 8) {
    const ff A = ff_split_bits((double)a), B = ff_split_bits((double)b);
    return (A.hi - B.hi) + (A.lo - B.lo);
  } else {
    return (float)(a - b);
  }
}
template <class T>
__device__ __forceinline__ float to_f32(T a) {
  if constexpr (sizeof(T) == 8) return ff_split_bits((double)a).hi;
  else return (float)a;
}

// The grid force is stored interleaved, one float4 (f_x, f_y, f_z, 0) per cell: the gather then reads each of a
// particle's eight cells with one 16-byte load instead of three scattered 4-byte ones.
template <class T, int MODEL>
__global__ void force_grid(const T* __restrict__ Phi, const T* __restrict__ phi, int lg, float a2, float Cs,
                           float inv2h, float4* __restrict__ f) {
  size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  const size_t n = (size_t)1 << (3 * lg);
  if (t >= n) return;
  const int m = (1 << lg) - 1;
  int k = (int)(t & m), j = (int)((t >> lg) & m), i = (int)(t >> (2 * lg));
  const size_t xp = cidx(lg, (i + 1) & m, j, k), xm = cidx(lg, (i - 1) & m, j, k);
  const size_t yp = cidx(lg, i, (j + 1) & m, k), ym = cidx(lg, i, (j - 1) & m, k);
  const size_t zp = cidx(lg, i, j, (k + 1) & m), zm = cidx(lg, i, j, (k - 1) & m);
  float g0 = 0.f, g1 = 0.f, g2 = 0.f;
  if (Phi) {
    g0 = a2 * fdiff<T>(Phi[xp], Phi[xm]);
    g1 = a2 * fdiff<T>(Phi[yp], Phi[ym]);
    g2 = a2 * fdiff<T>(Phi[zp], Phi[zm]);
  }
  if (MODEL != 0) {
    float v = to_f32<T>(phi[t]);
    float pref = (MODEL == ISIS_SYMMETRON) ? Cs * a2 * v : Cs * expf(v);
    g0 = fmaf(pref, fdiff<T>(phi[xp], phi[xm]), g0);
    g1 = fmaf(pref, fdiff<T>(phi[yp], phi[ym]), g1);
    g2 = fmaf(pref, fdiff<T>(phi[zp], phi[zm]), g2);
  }
  f[t] = make_float4(g0 * inv2h, g1 * inv2h, g2 * inv2h, 0.f);
}

// The same grid force, streamed: a block takes a tile of 8 x 32 cells in (j, k) through 32 planes in i and keeps
// three planes of both fields (tile plus a one-cell halo) in shared memory as float-float pairs, so each FP64
// value is split once per block instead of once per stencil that reads it (seven times); the next plane's
// values are loaded into registers while the current one is differenced.  Same arithmetic as force_grid.
// N >= 32.
constexpr int kFGTJ = 8, kFGTK = 32, kFGCh = 32;
constexpr int kFGHalo = (kFGTJ + 2) * (kFGTK + 2);

template <class T>
__device__ __forceinline__ float2 split_pair(T a) {
  if constexpr (sizeof(T) == 8) {
    const ff v = ff_split_bits((double)a);
    return make_float2(v.hi, v.lo);
  } else {
    return make_float2((float)a, 0.0f);
  }
}

template <class T, int MODEL>
__global__ void __launch_bounds__(kFGTJ * kFGTK) force_grid_st(const T* __restrict__ Phi, const T* __restrict__ phi,
                                                               int lg, float a2, float Cs, float inv2h,
                                                               float4* __restrict__ f) {
  __shared__ float2 sP[3][kFGHalo], sF[3][kFGHalo];
  const int N = 1 << lg, m = N - 1, ntk = N / kFGTK, ntj = N / kFGTJ;
  int b = blockIdx.x;
  const int k0 = (b % ntk) * kFGTK;
  b /= ntk;
  const int j0 = (b % ntj) * kFGTJ;
  const int i0 = (b / ntj) * kFGCh;
  const bool hasP = Phi != nullptr;
  constexpr int kU = (kFGHalo + kFGTJ * kFGTK - 1) / (kFGTJ * kFGTK);
  T rP[kU], rF[kU];
  auto load = [&](int p) {
#pragma unroll
    for (int u = 0; u < kU; ++u) {
      const int e = threadIdx.x + u * kFGTJ * kFGTK;
      if (e < kFGHalo) {
        const int r = e / (kFGTK + 2), col = e - r * (kFGTK + 2);
        const size_t g = cidx(lg, p & m, (j0 + r - 1) & m, (k0 + col - 1) & m);
        if (hasP) rP[u] = Phi[g];
        if (MODEL != 0) rF[u] = phi[g];
      }
    }
  };
  auto store = [&](int s) {
#pragma unroll
    for (int u = 0; u < kU; ++u) {
      const int e = threadIdx.x + u * kFGTJ * kFGTK;
      if (e < kFGHalo) {
        if (hasP) sP[s][e] = split_pair<T>(rP[u]);
        if (MODEL != 0) sF[s][e] = split_pair<T>(rF[u]);
      }
    }
  };
  auto diff = [](float2 a, float2 b) { return (a.x - b.x) + (a.y - b.y); };
  const int tj = threadIdx.x / kFGTK, tk = threadIdx.x - tj * kFGTK;
  const int c = (tj + 1) * (kFGTK + 2) + tk + 1;  // this thread's cell in the halo tile
  constexpr int kRow = kFGTK + 2;
  load(i0 - 1);
  store(0);
  load(i0);
  store(1);
  load(i0 + 1);
  for (int q = 1; q <= kFGCh; ++q) {
    const int i = i0 + q - 1;
    store((q + 1) % 3);  // plane i + 1
    if (q < kFGCh) load(i + 2);
    __syncthreads();
    const int sm = (q + 2) % 3, sc = q % 3, sp = (q + 1) % 3;
    float g0 = 0.f, g1 = 0.f, g2 = 0.f;
    if (hasP) {
      g0 = a2 * diff(sP[sp][c], sP[sm][c]);
      g1 = a2 * diff(sP[sc][c + kRow], sP[sc][c - kRow]);
      g2 = a2 * diff(sP[sc][c + 1], sP[sc][c - 1]);
    }
    if (MODEL != 0) {
      const float v = sF[sc][c].x;
      const float pref = (MODEL == ISIS_SYMMETRON) ? Cs * a2 * v : Cs * expf(v);
      g0 = fmaf(pref, diff(sF[sp][c], sF[sm][c]), g0);
      g1 = fmaf(pref, diff(sF[sc][c + kRow], sF[sc][c - kRow]), g1);
      g2 = fmaf(pref, diff(sF[sc][c + 1], sF[sc][c - 1]), g2);
    }
    const size_t o = cidx(lg, i, j0 + tj, k0 + tk);
    f[o] = make_float4(g0 * inv2h, g1 * inv2h, g2 * inv2h, 0.f);
    __syncthreads();
  }
}

// FP32 CIC weights of one axis (exact for 1 <= x < N; to FP32 rounding elsewhere).
__device__ __forceinline__ void cic_axis_f(float x, int N, int& i0, int& i1, float& w0, float& w1) {
  float xs = x - 0.5f;
  float f = floorf(xs);
  float t = xs - f;
  float fw = f - (float)N * floorf(f / (float)N);
  int i = (int)fw;
  i = i < 0 ? 0 : (i >= N ? N - 1 : i);
  i0 = i;
  i1 = (i + 1) & (N - 1);
  w0 = 1.0f - t;
  w1 = t;
}

// Per-particle acceleration g = -sum over the 8 CIC cells of W f (FP32).
__global__ void force_gather(const float4* __restrict__ f, const float* __restrict__ x, const float* __restrict__ y,
                             const float* __restrict__ z, long long np, int lg, float* __restrict__ gx,
                             float* __restrict__ gy, float* __restrict__ gz) {
  long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= np) return;
  const int N = 1 << lg;
  int ii[2], jj[2], kk[2];
  float wi[2], wj[2], wk[2];
  cic_axis_f(x[p], N, ii[0], ii[1], wi[0], wi[1]);
  cic_axis_f(y[p], N, jj[0], jj[1], wj[0], wj[1]);
  cic_axis_f(z[p], N, kk[0], kk[1], wk[0], wk[1]);
  float a0 = 0.f, a1 = 0.f, a2 = 0.f;
#pragma unroll
  for (int a = 0; a < 2; ++a)
#pragma unroll
    for (int b = 0; b < 2; ++b) {
      const float wab = wi[a] * wj[b];
#pragma unroll
      for (int d = 0; d < 2; ++d) {
        const size_t c = cidx(lg, ii[a], jj[b], kk[d]);
        const float w = wab * wk[d];
        const float4 v = __ldg(&f[c]);
        a0 = fmaf(w, v.x, a0);
        a1 = fmaf(w, v.y, a1);
        a2 = fmaf(w, v.z, a2);
      }
    }
  gx[p] = -a0;
  gy[p] = -a1;
  gz[p] = -a2;
}

// ---------------------------------------------------------------------------
// Deposit without device allocation (isis_cic_deposit_noalloc)
// ---------------------------------------------------------------------------

// Largest grid the allocation-free deposit accepts: 64^3 cells, 2 MiB of
// 64-bit accumulators held for the life of the process on every GPU that
// loads this library.
constexpr int kNoAllocMaxN = 64;
static __device__ __align__(256) unsigned long long g_noalloc_acc[(size_t)kNoAllocMaxN * kNoAllocMaxN * kNoAllocMaxN];

// Device address of g_noalloc_acc, looked up once per device.  In host code
// the name g_noalloc_acc is only a host-side stand-in for the array, so its
// address must come from cudaGetSymbolAddress with the device current.
// The table is filled under a mutex, so host threads that make their first calls at once are safe.  The
// cached address outlives nothing but the device's context: a device reset between calls is not supported.
constexpr int kMaxDevices = 64;
static unsigned long long* g_noalloc_ptr[kMaxDevices] = {nullptr};
static std::mutex g_noalloc_mu;
// Fewer particles than this cannot wrap a 64-bit accumulator of 2^-40 units in any cell.
constexpr int64_t kNoAllocMaxParticles = (int64_t)1 << 24;

static isis_status noalloc_scratch(unsigned long long** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return ISIS_ECUDA;
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (!g_noalloc_ptr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_acc) != cudaSuccess || !p) {
      cudaGetLastError();
      return ISIS_ECUDA;
    }
    g_noalloc_ptr[dev] = (unsigned long long*)p;
  }
  *out = g_noalloc_ptr[dev];
  return ISIS_OK;
}

__global__ void zero_u64(unsigned long long* __restrict__ a, size_t n) {
  size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t < n) a[t] = 0ull;
}

static bool grid_valid(const isis_grid* g) {
  return g && g->N >= 8 && g->N <= 1024 && (g->N & (g->N - 1)) == 0 && g->box > 0;
}

}  // namespace isis

using namespace isis;

// Leapfrog in super-comoving time tau (Eqs. (leap_frog_1)-(leap_frog_3)): one fused
// kick and drift per particle, positions and velocities in cell units:
//   v += kick g / h;  x += drift v;  x wrapped into [0, N).
// kick = (dtau_{n-1} + dtau_n)/2 merges the second half-kick of step n-1 with the
// first of step n (the paper's reuse of the second velocity evaluation), drift = dtau_n.
__global__ void kick_drift(float* __restrict__ x, float* __restrict__ y, float* __restrict__ z,
                           float* __restrict__ vx, float* __restrict__ vy, float* __restrict__ vz,
                           const float* __restrict__ gx, const float* __restrict__ gy, const float* __restrict__ gz,
                           long long np, float kick_h, float drift, float N) {
  const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= np) return;
  auto wrap = [N](float v) {
    v -= N * floorf(v / N);
    return v >= N ? v - N : v;  // floorf rounding can leave v == N
  };
  const float ux = fmaf(kick_h, gx[p], vx[p]), uy = fmaf(kick_h, gy[p], vy[p]), uz = fmaf(kick_h, gz[p], vz[p]);
  vx[p] = ux;
  vy[p] = uy;
  vz[p] = uz;
  x[p] = wrap(fmaf(drift, ux, x[p]));
  y[p] = wrap(fmaf(drift, uy, y[p]));
  z[p] = wrap(fmaf(drift, uz, z[p]));
}

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
  int e2 = 0;
  const int pow2 = exact_pow2(scale, &e2) ? 1 : 0;
  if (eta_f64)
    ISIS_LAUNCH(KK_CIC_FINISH, 16.0 * n, st,
                (cic_finish<double><<<nblk(n, 256), 256, 0, st>>>(acc, (double*)eta, n, scale, pow2, e2)));
  else
    ISIS_LAUNCH(KK_CIC_FINISH, 12.0 * n, st,
                (cic_finish<float><<<nblk(n, 256), 256, 0, st>>>(acc, (float*)eta, n, scale, pow2, e2)));
  return ISIS_OK;
}

isis_status isis_cic_deposit_noalloc(const isis_grid* grid, const float* x, const float* y, const float* z,
                                     int64_t npart, void* eta, int eta_f64, void* stream) {
  if (!grid_valid(grid) || !x || !y || !z || !eta || npart < 1 || npart > ((int64_t)1 << 40)) return ISIS_EINVAL;
  if (grid->N > kNoAllocMaxN || npart >= kNoAllocMaxParticles) return ISIS_EINVAL;  // use isis_cic_deposit
  unsigned long long* acc = nullptr;
  isis_status s = noalloc_scratch(&acc);
  if (s != ISIS_OK) return s;
  const int N = grid->N, lg = ilog2(N);
  const size_t n = (size_t)N * N * N;
  cudaStream_t st = (cudaStream_t)stream;
  // the array keeps the previous call's sums: clear the part this grid uses
  ISIS_LAUNCH(KK_SETUP, 8.0 * n, st, (zero_u64<<<nblk(n, 256), 256, 0, st>>>(acc, n)));
  ISIS_LAUNCH(KK_CIC_SCATTER, 12.0 * npart + 8.0 * n, st,
              (cic_scatter<<<nblk((size_t)npart, 256), 256, 0, st>>>(x, y, z, (long long)npart, lg, acc)));
  const double scale = (double)n / ((double)npart * kFix);
  int e2 = 0;
  const int pow2 = exact_pow2(scale, &e2) ? 1 : 0;
  if (eta_f64)
    ISIS_LAUNCH(KK_CIC_FINISH, 16.0 * n, st,
                (cic_finish<double><<<nblk(n, 256), 256, 0, st>>>(acc, (double*)eta, n, scale, pow2, e2)));
  else
    ISIS_LAUNCH(KK_CIC_FINISH, 12.0 * n, st,
                (cic_finish<float><<<nblk(n, 256), 256, 0, st>>>(acc, (float*)eta, n, scale, pow2, e2)));
  return ISIS_OK;
}

isis_status isis_fifth_force(isis_model model, const isis_params* p, const isis_grid* grid, double a,
                             const void* Phi, const void* phi, int fields_f64, const float* x, const float* y,
                             const float* z, int64_t npart, float* gx, float* gy, float* gz, void* stream) {
  if (!grid_valid(grid) || !x || !y || !z || !gx || !gy || !gz || npart < 1 || !(a > 0)) return ISIS_EINVAL;
  if (phi && (!p || (model != ISIS_SYMMETRON && model != ISIS_FOFR_HS && model != ISIS_CHAMELEON)))
    return ISIS_EINVAL;
  if (phi && model == ISIS_SYMMETRON && !(p->a_ssb > 0)) return ISIS_EINVAL;
  if (phi && model == ISIS_CHAMELEON && !(p->cham_n > -1.0)) return ISIS_EINVAL;
  const int lg = ilog2(grid->N);
  const double h = grid->box / grid->N;
  const double inv2h = 1.0 / (2.0 * h), a2 = a * a;
  double Cs = 0.0;
  if (phi && model == ISIS_SYMMETRON)  // Eq. (symmetron_geodesics_tilde_chi)
    Cs = 6.0 * grid->Omega_m * grid->H0 * grid->H0 * (p->beta * p->lambda0) * (p->beta * p->lambda0) /
         (p->a_ssb * p->a_ssb * p->a_ssb);
  if (phi && model == ISIS_FOFR_HS) Cs = 0.5;  // Sect. 4.2: (1/2) e^u grad u
  if (phi && model == ISIS_CHAMELEON)  // a^2 grad ln A, ln A = beta phi / M_pl = (beta phi_0 / M_pl) e^u
    Cs = a2 * 3.0 * (1.0 + p->cham_n) * p->beta * p->beta * grid->Omega_m * grid->H0 * grid->H0 * p->lambda0 *
         p->lambda0;
  cudaStream_t st = (cudaStream_t)stream;
  const size_t n = (size_t)grid->N * grid->N * grid->N;
  float* fg = get_force_buf(grid->N);
  if (!fg) return ISIS_ENOMEM;
  float4* f4 = reinterpret_cast<float4*>(fg);
  int mcode = phi ? (int)model : 0;
  const double gbytes = (double)n * ((fields_f64 ? 8 : 4) * ((Phi ? 1 : 0) + (phi ? 1 : 0)) + 12);
  const int Ng = grid->N;
  const unsigned st_blocks = (unsigned)((Ng / kFGTK) * (Ng / kFGTJ) * (Ng / kFGCh));
#define ISIS_FGRID(T, MC)                                                                                      \
  if (Ng >= 32)                                                                                                \
    ISIS_LAUNCH(KK_FORCE_GRID, gbytes, st,                                                                     \
                (force_grid_st<T, MC><<<st_blocks, kFGTJ * kFGTK, 0, st>>>((const T*)Phi, (const T*)phi, lg,    \
                                                                          (float)a2, (float)Cs, (float)inv2h,   \
                                                                          f4)));                                \
  else                                                                                                         \
    ISIS_LAUNCH(KK_FORCE_GRID, gbytes, st,                                                                     \
                (force_grid<T, MC><<<nblk(n, 256), 256, 0, st>>>((const T*)Phi, (const T*)phi, lg, (float)a2,  \
                                                                 (float)Cs, (float)inv2h, f4)))
  if (fields_f64) {
    if (mcode == 0) ISIS_FGRID(double, 0);
    else if (mcode == ISIS_SYMMETRON) ISIS_FGRID(double, ISIS_SYMMETRON);
    else ISIS_FGRID(double, ISIS_FOFR_HS);
  } else {
    if (mcode == 0) ISIS_FGRID(float, 0);
    else if (mcode == ISIS_SYMMETRON) ISIS_FGRID(float, ISIS_SYMMETRON);
    else ISIS_FGRID(float, ISIS_FOFR_HS);
  }
#undef ISIS_FGRID
  ISIS_LAUNCH(KK_FORCE, 24.0 * npart + 12.0 * n, st,
              (force_gather<<<nblk((size_t)npart, 256), 256, 0, st>>>(f4, x, y, z, (long long)npart, lg, gx, gy,
                                                                      gz)));
  return ISIS_OK;
}


isis_status isis_kick_drift(const isis_grid* grid, float* x, float* y, float* z, float* vx, float* vy, float* vz,
                            const float* gx, const float* gy, const float* gz, int64_t npart, double kick,
                            double drift, void* stream) {
  if (!grid_valid(grid) || !x || !y || !z || !vx || !vy || !vz || !gx || !gy || !gz || npart < 1 ||
      !std::isfinite(kick) || !std::isfinite(drift))
    return ISIS_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  const double h = grid->box / grid->N;
  ISIS_LAUNCH(KK_FORCE, 36.0 * npart, st,
              (kick_drift<<<nblk((size_t)npart, 256), 256, 0, st>>>(x, y, z, vx, vy, vz, gx, gy, gz, (long long)npart,
                                                                     (float)(kick / h), (float)drift,
                                                                     (float)grid->N)));
  return ISIS_OK;
}

}  // extern "C"
