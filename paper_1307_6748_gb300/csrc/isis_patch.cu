// isis_patch.cu -- FAS solve on a refinement patch (Sect. 3.3.1, Sect. 3.4.1)
// for the three models: FP64 throughout, or FP32 correction cycles inside an
// FP64 defect correction (ISIS_F32_REFINE64).  The readings are listed in
// isis_patch.cuh.
//
// Every level of the patch is a dense box in row-major order (k fastest);
// kernels run one thread per cell.  The host loop synchronises once per cycle
// (FP64) or once per outer iteration (mixed) to read the residual norm.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "isis_patch.cuh"
#include "isis_prof.cuh"

namespace isis {

namespace {

constexpr int kPT = 256;          // threads per block of the cell kernels
constexpr int kPNormBlocks = 256;  // blocks of the norm kernels
constexpr int kCoarseSweeps = 16;  // red/black sweeps on the coarsest patch level
constexpr int kCoarseThreads = 256;
constexpr size_t kCoarseSmem = 220 * 1024;  // the coarsest level in shared memory up to this many bytes

template <class T>
struct PL {  // one level of the patch
  int n0, n1, n2;
  T ih2;
  const T* m;
  const T* eta;  // nullptr where the form does not read the density
  T* u;          // the unknown: the field (FIELD) or the correction e about B (DELTA)
  const T* pre;
  const T* sig;  // nullptr: Sigma = 0 (the FP64 finest level)
  const T* B;    // DELTA: the base field, else nullptr
};

__device__ __forceinline__ size_t pidx(int n1, int n2, int i, int j, int k) {
  return ((size_t)i * n1 + j) * n2 + k;
}

__device__ __forceinline__ void pdecode(size_t t, int n1, int n2, int& i, int& j, int& k) {
  k = (int)(t % n2);
  size_t r = t / n2;
  j = (int)(r % n1);
  i = (int)(r / n1);
}

// An unknown: m > 0 and off the outer layer (whose stencil would leave the box).
template <class T>
__device__ __forceinline__ bool unknown(const PL<T>& L, size_t t, int i, int j, int k) {
  return L.m[t] > T(0) && i > 0 && j > 0 && k > 0 && i < L.n0 - 1 && j < L.n1 - 1 && k < L.n2 - 1;
}

// L(u) - Sigma and dL/du at the unknown (i,j,k).  with_pre: ghosts follow Eq. (ueq) with the stored u^Pre;
// otherwise u^Pre = u and a ghost is the neighbour's value.
// DELTA form (the FP32 cycles of the defect correction): u = B + e, and the operator is L(B + e) - L(B).  The
// ghost of a masked neighbour is B_nb + e_nb + (m_nb/m_c)(e_c - e_c^Pre): B_c cancels from u_c - u_c^Pre, so the
// correction enters the ghost as the field does in Eq. (ueq).
template <Model M, Form FM, class T>
__device__ __forceinline__ void pt_eval(const CoefT<T>& c, const PL<T>& L, int i, int j, int k, bool with_pre, T& F,
                                        T& dF) {
  const size_t q = pidx(L.n1, L.n2, i, j, k);
  const T mc = L.m[q], u = L.u[q];
  const T dpre = with_pre ? u - L.pre[q] : T(0);
  Cell<T> cell;
  cell.x = u;
  cell.eta = uses_eta<M, FM>() ? L.eta[q] : T(0);
  cell.sig = L.sig ? L.sig[q] : T(0);
  T mu[6];
  const size_t s0 = (size_t)L.n1 * L.n2, s1 = (size_t)L.n2;
  const size_t qn[6] = {q + s0, q - s0, q + s1, q - s1, q + 1, q - 1};
#pragma unroll
  for (int d = 0; d < 6; ++d) {
    const T mn = L.m[qn[d]];
    T un = L.u[qn[d]];
    mu[d] = T(0);
    if (!(mn > T(0))) {
      mu[d] = mn / mc;
      un += mu[d] * dpre;
    }
    cell.xn[d] = un;
  }
  if constexpr (FM == DELTA) {
    cell.B = L.B[q];
#pragma unroll
    for (int d = 0; d < 6; ++d) cell.Bn[d] = L.B[qn[d]];
  }
  if constexpr (M == FOFR) {
    if constexpr (FM == FIELD) {
      cell.a = dexp<T>(u);
#pragma unroll
      for (int d = 0; d < 6; ++d) cell.an[d] = dexp<T>(cell.xn[d]);
    } else {
      cell.w = dexp<T>(cell.B);
      cell.a = cell.w * dexpm1<T>(u);
#pragma unroll
      for (int d = 0; d < 6; ++d) {
        cell.wn[d] = dexp<T>(cell.Bn[d]);
        cell.an[d] = cell.wn[d] * dexpm1<T>(cell.xn[d]);
      }
    }
  }
  eval_cell<M, FM, T>(c, L.ih2, cell, F, dF);
  // the derivative through the ghost values of the masked neighbours
  T extra = T(0);
#pragma unroll
  for (int d = 0; d < 6; ++d) {
    if constexpr (M == FOFR && FM == FIELD) {
      extra += mu[d] * (T(0.5) * cell.an[d] * (cell.xn[d] - u) + T(0.5) * (cell.a + cell.an[d]));
    } else if constexpr (M == FOFR) {
      // e^u of the cell and of the ghost, u_nb - u_c = (B_nb - B_c) + (e_nb - e_c)
      const T bt = cell.w + cell.a, btn = cell.wn[d] + cell.an[d];
      extra += mu[d] * (T(0.5) * btn * ((cell.Bn[d] - cell.B) + (cell.xn[d] - u)) + T(0.5) * (bt + btn));
    } else {
      extra += mu[d];
    }
  }
  dF += extra * L.ih2;
}

__global__ void pt_mask0(const uint8_t* __restrict__ flags, int b1, int b2, double* __restrict__ m, int n0, int n1,
                         int n2) {
  const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (size_t)n0 * n1 * n2) return;
  int i, j, k;
  pdecode(t, n1, n2, i, j, k);
  m[t] = flags[pidx(b1, b2, i >> 1, j >> 1, k >> 1)] ? 1.0 : -1.0;
}

// coarse = mean of the 8 children (fine dims = 2 x coarse dims); edge != 0: the outer layer gets -1 (masks);
// c0 != nullptr: a second copy (the u_H^0 that the prolongation subtracts)
template <class T>
__global__ void pt_restrict(const T* __restrict__ f, T* __restrict__ c, int n0, int n1, int n2, int edge = 0,
                            T* __restrict__ c0 = nullptr) {
  const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (size_t)n0 * n1 * n2) return;
  int I, J, K;
  pdecode(t, n1, n2, I, J, K);
  const int f1 = 2 * n1, f2 = 2 * n2;
  T s = T(0);
#pragma unroll
  for (int a = 0; a < 2; ++a)
#pragma unroll
    for (int b = 0; b < 2; ++b) {
      const size_t r = pidx(f1, f2, 2 * I + a, 2 * J + b, 2 * K);
      s += f[r] + f[r + 1];
    }
  const T v = (edge && (I == 0 || J == 0 || K == 0 || I == n0 - 1 || J == n1 - 1 || K == n2 - 1)) ? T(-1)
                                                                                                 : T(0.125) * s;
  c[t] = v;
  if (c0) c0[t] = v;
}

// Cell-centred trilinear interpolation of the parent at the finest patch cells: written where m <= 0,
// or everywhere when all != 0.
__global__ void pt_interp(const double* __restrict__ parent, int p0, int p1, int p2, int o0, int o1, int o2,
                          int periodic, const double* __restrict__ m, double* __restrict__ u, int n0, int n1, int n2,
                          int all) {
  const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (size_t)n0 * n1 * n2) return;
  if (!all && m[t] > 0.0) return;
  int f[3];
  pdecode(t, n1, n2, f[0], f[1], f[2]);
  const int pd[3] = {p0, p1, p2}, od[3] = {o0, o1, o2};
  int c[3][2];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    c[a][0] = od[a] + (f[a] >> 1);
    c[a][1] = c[a][0] + ((f[a] & 1) ? 1 : -1);
    if (periodic) {
      c[a][0] = (c[a][0] % pd[a] + pd[a]) % pd[a];
      c[a][1] = (c[a][1] % pd[a] + pd[a]) % pd[a];
    }
  }
  const double w[2] = {0.75, 0.25};
  double v = 0.0;
#pragma unroll
  for (int a = 0; a < 2; ++a)
#pragma unroll
    for (int b = 0; b < 2; ++b)
#pragma unroll
      for (int d = 0; d < 2; ++d) v += w[a] * w[b] * w[d] * parent[pidx(p1, p2, c[0][a], c[1][b], c[2][d])];
  u[t] = v;
}

// res = Sigma - L(u) at the unknowns, 0 elsewhere.
template <Model M, Form FM, class T>
__global__ void __launch_bounds__(kPT) pt_resid(PL<T> L, CoefT<T> c, T* __restrict__ res) {
  const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (size_t)L.n0 * L.n1 * L.n2) return;
  T r = T(0);
  int i, j, k;
  pdecode(t, L.n1, L.n2, i, j, k);
  if (unknown(L, t, i, j, k)) {
    T F, dF;
    pt_eval<M, FM, T>(c, L, i, j, k, false, F, dF);
    r = -F;
  }
  res[t] = r;
}

// Sigma_H = L_H(u_H) + R(res) at the coarse unknowns (the coarse level has sig == nullptr in L: its own
// source is written to sig).
template <Model M, Form FM, class T>
__global__ void __launch_bounds__(kPT) pt_sigma(PL<T> C, CoefT<T> c, const T* __restrict__ rf, T* __restrict__ sig) {
  const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (size_t)C.n0 * C.n1 * C.n2) return;
  int I, J, K;
  pdecode(t, C.n1, C.n2, I, J, K);
  T s = T(0);
  if (unknown(C, t, I, J, K)) {
    T F, dF;
    pt_eval<M, FM, T>(c, C, I, J, K, false, F, dF);  // C.sig == nullptr: F = L_H(u_H)
    const int f1 = 2 * C.n1, f2 = 2 * C.n2;
    T r = T(0);
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
      for (int b = 0; b < 2; ++b) {
        const size_t q = pidx(f1, f2, 2 * I + a, 2 * J + b, 2 * K);
        r += rf[q] + rf[q + 1];
      }
    s = F + T(0.125) * r;
  }
  sig[t] = s;
}

// u += P(uc - uc0) at the fine unknowns; coarse cells outside the box contribute nothing.
template <class T>
__global__ void __launch_bounds__(kPT) pt_prolong(PL<T> L, const T* __restrict__ uc, const T* __restrict__ uc0,
                                                  int c0, int c1, int c2) {
  const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (size_t)L.n0 * L.n1 * L.n2) return;
  int f[3];
  pdecode(t, L.n1, L.n2, f[0], f[1], f[2]);
  if (!unknown(L, t, f[0], f[1], f[2])) return;
  const int cd[3] = {c0, c1, c2};
  int ci[3][2];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    ci[a][0] = f[a] >> 1;
    ci[a][1] = ci[a][0] + ((f[a] & 1) ? 1 : -1);
  }
  const T w[2] = {T(0.75), T(0.25)};
  T v = T(0);
#pragma unroll
  for (int a = 0; a < 2; ++a)
#pragma unroll
    for (int b = 0; b < 2; ++b)
#pragma unroll
      for (int d = 0; d < 2; ++d) {
        const int x = ci[0][a], y = ci[1][b], z = ci[2][d];
        if (x < 0 || x >= cd[0] || y < 0 || y >= cd[1] || z < 0 || z >= cd[2]) continue;
        const size_t q = pidx(c1, c2, x, y, z);
        v += w[a] * w[b] * w[d] * (uc[q] - uc0[q]);
      }
  L.u[t] += v;
}

// Shared memory of the coarsest level per cell: u, u^Pre, m, eta, Sigma (and B in the DELTA form), one list entry.
template <Form FM, class T>
constexpr size_t coarse_bytes_per_cell() {
  return (FM == DELTA ? 6 : 5) * sizeof(T) + sizeof(int);
}

// The coarsest patch level held in shared memory (u, u^Pre, m, eta, Sigma, and B in the DELTA form, of every
// cell, and the unknowns of each colour as lists): u^Pre = u, then kCoarseSweeps red/black sweeps, in one
// block; u written back.  One block pays each half-sweep's latency (in FP64 on GB300's few FP64 units):
// shared memory and the lists keep that short.
template <Model M, Form FM, class T>
__global__ void __launch_bounds__(kCoarseThreads) pt_coarsest_smem(PL<T> L, CoefT<T> c) {
  extern __shared__ __align__(16) unsigned char pt_smem[];
  __shared__ int cnt[2];
  const int n = L.n0 * L.n1 * L.n2;
  constexpr int nA = FM == DELTA ? 6 : 5;
  T* sh = reinterpret_cast<T*>(pt_smem);
  T *su = sh, *spre = sh + n, *sm = sh + 2 * n, *seta = sh + 3 * n, *ssig = sh + 4 * n;
  T* sB = FM == DELTA ? sh + 5 * n : nullptr;
  int* lst = reinterpret_cast<int*>(sh + nA * n);  // red unknowns from the front, black from the back
  if (threadIdx.x < 2) cnt[threadIdx.x] = 0;
  for (int t = threadIdx.x; t < n; t += blockDim.x) {
    su[t] = L.u[t];
    spre[t] = su[t];
    sm[t] = L.m[t];
    seta[t] = uses_eta<M, FM>() ? L.eta[t] : T(0);
    ssig[t] = L.sig ? L.sig[t] : T(0);
    if constexpr (FM == DELTA) sB[t] = L.B[t];
  }
  __syncthreads();
  PL<T> S{L.n0, L.n1, L.n2, L.ih2, sm, seta, su, spre, ssig, sB};
  for (int t = threadIdx.x; t < n; t += blockDim.x) {
    const int k = t % S.n2, j = (t / S.n2) % S.n1, i = t / (S.n1 * S.n2);
    if (!unknown(S, t, i, j, k)) continue;
    const int color = (i + j + k) & 1;
    const int pos = atomicAdd(&cnt[color], 1);
    lst[color ? n - 1 - pos : pos] = t;
  }
  __syncthreads();
  for (int s = 0; s < kCoarseSweeps; ++s) {
    for (int color = 0; color < 2; ++color) {
      for (int q = threadIdx.x; q < cnt[color]; q += blockDim.x) {
        const int t = lst[color ? n - 1 - q : q];
        const int k = t % S.n2, j = (t / S.n2) % S.n1, i = t / (S.n1 * S.n2);
        T F, dF;
        pt_eval<M, FM, T>(c, S, i, j, k, true, F, dF);
        su[t] -= F / dF;
      }
      __syncthreads();
    }
  }
  for (int t = threadIdx.x; t < n; t += blockDim.x) L.u[t] = su[t];
}

// One colour of a sweep over a list of that colour's unknowns.  save_pre (the phase's first sweep of this
// colour): u^Pre = u is stored first, for this colour's unknowns, the only cells whose u^Pre a ghost reads; the
// other colour's sweeps have not moved them since the phase began.  Then u - u^Pre = 0 in this sweep.
template <Model M, Form FM, class T>
__global__ void __launch_bounds__(kPT) pt_smooth_list(PL<T> L, CoefT<T> c, const int* __restrict__ list, int count,
                                                      T* __restrict__ pre_out) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= count) return;
  const size_t t = (size_t)list[q];
  int i, j, k;
  pdecode(t, L.n1, L.n2, i, j, k);
  if (!unknown(L, t, i, j, k)) return;
  if (pre_out) pre_out[t] = L.u[t];
  T F, dF;
  pt_eval<M, FM, T>(c, L, i, j, k, pre_out == nullptr, F, dF);
  L.u[t] -= F / dF;
}

// The unknowns of each colour, as lists of cell indices (in any order: cells of one colour do not read one
// another, so the order does not change a sweep's result).
__global__ void __launch_bounds__(kPT) pt_compact(PL<double> L, int* __restrict__ red, int* __restrict__ black,
                                                  int* __restrict__ counts) {
  const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (size_t)L.n0 * L.n1 * L.n2) return;
  int i, j, k;
  pdecode(t, L.n1, L.n2, i, j, k);
  if (!unknown(L, t, i, j, k)) return;
  const int color = (i + j + k) & 1;
  const int pos = atomicAdd(&counts[color], 1);
  (color ? black : red)[pos] = (int)t;
}

// The coarsest patch level: u^Pre = u, then kCoarseSweeps red/black sweeps, in one block.
template <Model M, Form FM, class T>
__global__ void __launch_bounds__(1024) pt_coarsest(PL<T> L, CoefT<T> c, T* pre) {
  const size_t n = (size_t)L.n0 * L.n1 * L.n2;
  for (size_t t = threadIdx.x; t < n; t += blockDim.x) pre[t] = L.u[t];
  __syncthreads();
  for (int s = 0; s < kCoarseSweeps; ++s) {
    for (int color = 0; color < 2; ++color) {
      for (size_t t = threadIdx.x; t < n; t += blockDim.x) {
        int i, j, k;
        pdecode(t, L.n1, L.n2, i, j, k);
        if (((i + j + k) & 1) != color || !unknown(L, t, i, j, k)) continue;
        T F, dF;
        pt_eval<M, FM, T>(c, L, i, j, k, true, F, dF);
        L.u[t] -= F / dF;
      }
      __syncthreads();
    }
  }
}

__device__ __forceinline__ void pt_block_sum(double v, double* out) {
  __shared__ double red[kPT / 32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x < 32) {
    v = threadIdx.x < kPT / 32 ? red[threadIdx.x] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if (threadIdx.x == 0) out[blockIdx.x] = v;
  }
}

// Block partial sums of (L(u) - Sigma)^2 over the unknowns (u^Pre = u).
template <Model M>
__global__ void __launch_bounds__(kPT) pt_norm(PL<double> L, CoefT<double> c, double* __restrict__ part) {
  const size_t n = (size_t)L.n0 * L.n1 * L.n2;
  double acc = 0.0;
  for (size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (size_t)gridDim.x * blockDim.x) {
    int i, j, k;
    pdecode(t, L.n1, L.n2, i, j, k);
    if (!unknown(L, t, i, j, k)) continue;
    double F, dF;
    pt_eval<M, FIELD, double>(c, L, i, j, k, false, F, dF);
    acc += F * F;
  }
  pt_block_sum(acc, part);
}

// Block partial sums of res^2 (res from pt_resid: zero off the unknowns).
__global__ void __launch_bounds__(kPT) pt_sumsq(const double* __restrict__ res, size_t n, double* __restrict__ part) {
  double acc = 0.0;
  for (size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (size_t)gridDim.x * blockDim.x)
    acc += res[t] * res[t];
  pt_block_sum(acc, part);
}

// Block partial sums of (eta - eref)^2 over the unknowns.
__global__ void __launch_bounds__(kPT) pt_ref(const double* __restrict__ m, const double* __restrict__ eta, size_t n,
                                              double eref, double* __restrict__ part) {
  double acc = 0.0;
  for (size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (size_t)gridDim.x * blockDim.x)
    if (m[t] > 0.0) acc += (eta[t] - eref) * (eta[t] - eref);
  pt_block_sum(acc, part);
}

__global__ void __launch_bounds__(kPT) pt_to_f32(const double* __restrict__ src, float* __restrict__ dst, size_t n) {
  const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t < n) dst[t] = (float)src[t];
}

// The FP32 problem of one outer iteration on the finest level: base B = u rounded to FP32, correction e = 0,
// source Sigma = the FP64 residual (rounded).
__global__ void __launch_bounds__(kPT) pt_prep32(const double* __restrict__ u, const double* __restrict__ res,
                                                 float* __restrict__ B, float* __restrict__ e,
                                                 float* __restrict__ sig, size_t n) {
  const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n) return;
  B[t] = (float)u[t];
  e[t] = 0.f;
  sig[t] = (float)res[t];
}

// u += e (e is zero off the unknowns).
__global__ void __launch_bounds__(kPT) pt_add_correction(double* __restrict__ u, const float* __restrict__ e,
                                                         size_t n) {
  const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t < n) u[t] += (double)e[t];
}

inline unsigned nblk(size_t n) { return (unsigned)((n + kPT - 1) / kPT); }

struct PLevel {
  int n[3];
  double h;
  double *m, *eta, *u, *u0, *sig, *res, *pre;
  int* list[2];  // unknowns of each colour
  int count[2];
  // FP32 correction form (ISIS_F32_REFINE64): masks, density (symmetron), correction e and its coarse copy,
  // Sigma, residual, e^Pre, base B
  float *m32 = nullptr, *eta32 = nullptr, *e = nullptr, *e0 = nullptr, *sig32 = nullptr, *res32 = nullptr,
        *pre32 = nullptr, *B = nullptr;
  size_t cells() const { return (size_t)n[0] * n[1] * n[2]; }
  PL<double> view(bool with_sig) const {
    return PL<double>{n[0], n[1], n[2], 1.0 / (h * h), m, eta, u, pre, with_sig ? sig : nullptr, nullptr};
  }
  PL<float> view32(bool with_sig) const {
    return PL<float>{n[0], n[1], n[2], (float)(1.0 / (h * h)), m32, eta32, e, pre32, with_sig ? sig32 : nullptr, B};
  }
};

template <Model M>
struct PatchSolver {
  const PatchArgs& A;
  std::vector<PLevel> lev;
  double* part = nullptr;
  double* host = nullptr;
  int* counts = nullptr;
  cudaStream_t strm;  // the caller's stream; a private one while a V-cycle is captured into a graph
  // one V-cycle (vcycle or vcycle32 from the finest level) as a CUDA graph: the same launches, captured once
  // per solve and replayed for every cycle, which takes the host's launch overhead off these small grids
  cudaStream_t cap = nullptr;
  cudaGraphExec_t graph = nullptr;
  long long graph_launches = 0;
  bool try_graph = true;

  explicit PatchSolver(const PatchArgs& a) : A(a), strm(a.st) {}
  ~PatchSolver() {
    if (graph) {
      cudaStreamSynchronize(A.st);
      cudaGraphExecDestroy(graph);
    }
    if (cap) cudaStreamDestroy(cap);
  }

  // One V-cycle from the finest level: through the graph, captured at the first call on a private stream (the
  // caller's stream may be the legacy default stream, which cannot be captured) and launched on the caller's;
  // launch by launch while per-launch events are on or if the capture fails.
  template <class Cycle>
  isis_status cycle_graphed(Cycle cycle) {
    if (!graph && try_graph && !prof_enabled()) {
      try_graph = false;
      if (cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking) == cudaSuccess &&
          cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
        const long long before = prof_launches();
        strm = cap;
        const isis_status s = cycle();
        strm = A.st;
        cudaGraph_t g = nullptr;
        const cudaError_t e = cudaStreamEndCapture(cap, &g);
        graph_launches = prof_launches() - before;
        prof_add_launches(-graph_launches);  // recorded, not run
        if (s != ISIS_OK || e != cudaSuccess || !g || cudaGraphInstantiate(&graph, g, 0) != cudaSuccess)
          graph = nullptr;
        if (g) cudaGraphDestroy(g);
      }
      cudaGetLastError();  // a capture that failed leaves no error behind: the cycle then runs launch by launch
    }
    if (graph) {
      if (cudaGraphLaunch(graph, A.st) != cudaSuccess) return ISIS_ECUDA;
      prof_add_launches(graph_launches);
      return ISIS_OK;
    }
    return cycle();
  }

  // bytes a level-sweep kernel reads and writes once (u, m, eta, pre, sig; u written)
  static double sweep_bytes(const PLevel& L) { return 48.0 * L.cells(); }

  isis_status sum_parts(double* out) {
    if (cudaMemcpyAsync(host, part, kPNormBlocks * sizeof(double), cudaMemcpyDeviceToHost, strm) != cudaSuccess)
      return ISIS_ECUDA;
    if (cudaStreamSynchronize(strm) != cudaSuccess) return ISIS_ECUDA;
    double s = 0.0;
    for (int b = 0; b < kPNormBlocks; ++b) s += host[b];
    *out = s;
    return ISIS_OK;
  }

  isis_status norm(double* rms) {
    const PLevel& F = lev[0];
    ISIS_LAUNCH(KK_PATCH_OTHER, sweep_bytes(F), strm,
                (pt_norm<M><<<kPNormBlocks, kPT, 0, strm>>>(F.view(false), A.coef, part)));
    double s = 0.0;
    isis_status st = sum_parts(&s);
    if (st != ISIS_OK) return st;
    *rms = A.unknowns > 0 ? std::sqrt(s / (double)A.unknowns) : 0.0;
    return ISIS_OK;
  }

  isis_status phase(size_t l, int nsweep) {
    const PLevel& L = lev[l];
    for (int s = 0; s < nsweep; ++s)
      for (int color = 0; color < 2; ++color) {
        if (L.count[color] == 0) continue;
        ISIS_LAUNCH(KK_PATCH_SMOOTH, 48.0 * L.count[color], strm,
                    (pt_smooth_list<M, FIELD, double><<<nblk(L.count[color]), kPT, 0, strm>>>(
                        L.view(l > 0), A.coef, L.list[color], L.count[color], s == 0 ? L.pre : nullptr)));
      }
    return ISIS_OK;
  }

  isis_status vcycle(size_t l) {
    const PLevel& L = lev[l];
    if (l + 1 == lev.size()) {
      const size_t smem = coarse_bytes_per_cell<FIELD, double>() * L.cells();
      if (smem <= kCoarseSmem) {
        ISIS_LAUNCH(KK_PATCH_COARSEST, 40.0 * L.cells(), strm,
                    (pt_coarsest_smem<M, FIELD, double><<<1, kCoarseThreads, smem, strm>>>(L.view(l > 0), A.coef)));
      } else {
        ISIS_LAUNCH(KK_PATCH_COARSEST, kCoarseSweeps * sweep_bytes(L), strm,
                    (pt_coarsest<M, FIELD, double><<<1, 1024, 0, strm>>>(L.view(l > 0), A.coef, L.pre)));
      }
      return ISIS_OK;
    }
    const PLevel& C = lev[l + 1];
    isis_status st = phase(l, A.nu1);
    if (st != ISIS_OK) return st;
    ISIS_LAUNCH(KK_PATCH_OTHER, 48.0 * L.cells(), strm,
                (pt_resid<M, FIELD, double><<<nblk(L.cells()), kPT, 0, strm>>>(L.view(l > 0), A.coef, L.res)));
    ISIS_LAUNCH(KK_PATCH_OTHER, 10.0 * C.cells() * 8.0, strm,
                (pt_restrict<double><<<nblk(C.cells()), kPT, 0, strm>>>(L.u, C.u, C.n[0], C.n[1], C.n[2], 0, C.u0)));
    ISIS_LAUNCH(KK_PATCH_OTHER, 48.0 * C.cells() + 64.0 * C.cells(), strm,
                (pt_sigma<M, FIELD, double><<<nblk(C.cells()), kPT, 0, strm>>>(C.view(false), A.coef, L.res, C.sig)));
    st = vcycle(l + 1);
    if (st != ISIS_OK) return st;
    ISIS_LAUNCH(KK_PATCH_OTHER, 24.0 * L.cells() + 16.0 * C.cells(), strm,
                (pt_prolong<double><<<nblk(L.cells()), kPT, 0, strm>>>(L.view(l > 0), C.u, C.u0, C.n[0], C.n[1],
                                                                       C.n[2])));
    return phase(l, A.nu2);
  }

  // ---- the FP32 correction cycles of ISIS_F32_REFINE64 (every level in the DELTA form, Sigma on all) ----
  isis_status phase32(size_t l, int nsweep) {
    const PLevel& L = lev[l];
    for (int s = 0; s < nsweep; ++s)
      for (int color = 0; color < 2; ++color) {
        if (L.count[color] == 0) continue;
        ISIS_LAUNCH(KK_PATCH_SMOOTH, 28.0 * L.count[color], strm,
                    (pt_smooth_list<M, DELTA, float><<<nblk(L.count[color]), kPT, 0, strm>>>(
                        L.view32(true), A.coef, L.list[color], L.count[color], s == 0 ? L.pre32 : nullptr)));
      }
    return ISIS_OK;
  }

  isis_status vcycle32(size_t l) {
    const PLevel& L = lev[l];
    if (l + 1 == lev.size()) {
      const size_t smem = coarse_bytes_per_cell<DELTA, float>() * L.cells();
      if (smem <= kCoarseSmem) {
        ISIS_LAUNCH(KK_PATCH_COARSEST, 24.0 * L.cells(), strm,
                    (pt_coarsest_smem<M, DELTA, float><<<1, kCoarseThreads, smem, strm>>>(L.view32(true), A.coef)));
      } else {
        ISIS_LAUNCH(KK_PATCH_COARSEST, kCoarseSweeps * 28.0 * L.cells(), strm,
                    (pt_coarsest<M, DELTA, float><<<1, 1024, 0, strm>>>(L.view32(true), A.coef, L.pre32)));
      }
      return ISIS_OK;
    }
    const PLevel& C = lev[l + 1];
    isis_status st = phase32(l, A.nu1);
    if (st != ISIS_OK) return st;
    ISIS_LAUNCH(KK_PATCH_OTHER, 28.0 * L.cells(), strm,
                (pt_resid<M, DELTA, float><<<nblk(L.cells()), kPT, 0, strm>>>(L.view32(true), A.coef, L.res32)));
    ISIS_LAUNCH(KK_PATCH_OTHER, 5.0 * C.cells() * 8.0, strm,
                (pt_restrict<float><<<nblk(C.cells()), kPT, 0, strm>>>(L.e, C.e, C.n[0], C.n[1], C.n[2], 0, C.e0)));
    ISIS_LAUNCH(KK_PATCH_OTHER, 24.0 * C.cells() + 32.0 * C.cells(), strm,
                (pt_sigma<M, DELTA, float><<<nblk(C.cells()), kPT, 0, strm>>>(C.view32(false), A.coef, L.res32,
                                                                             C.sig32)));
    st = vcycle32(l + 1);
    if (st != ISIS_OK) return st;
    ISIS_LAUNCH(KK_PATCH_OTHER, 12.0 * L.cells() + 8.0 * C.cells(), strm,
                (pt_prolong<float><<<nblk(L.cells()), kPT, 0, strm>>>(L.view32(true), C.e, C.e0, C.n[0], C.n[1],
                                                                      C.n[2])));
    return phase32(l, A.nu2);
  }

  isis_status setup() {
    const PLevel& F = lev[0];
    ISIS_LAUNCH(KK_PATCH_OTHER, 9.0 * F.cells(), strm,
                (pt_mask0<<<nblk(F.cells()), kPT, 0, strm>>>(A.flags, A.n[1], A.n[2], F.m, F.n[0], F.n[1], F.n[2])));
    for (size_t l = 1; l < lev.size(); ++l) {
      const PLevel& C = lev[l];
      const PLevel& L = lev[l - 1];
      ISIS_LAUNCH(KK_PATCH_OTHER, 9.0 * C.cells() * 8.0, strm,
                  (pt_restrict<double><<<nblk(C.cells()), kPT, 0, strm>>>(L.m, C.m, C.n[0], C.n[1], C.n[2], 1)));
      ISIS_LAUNCH(KK_PATCH_OTHER, 9.0 * C.cells() * 8.0, strm,
                  (pt_restrict<double><<<nblk(C.cells()), kPT, 0, strm>>>(L.eta, C.eta, C.n[0], C.n[1], C.n[2])));
    }
    ISIS_LAUNCH(KK_PATCH_OTHER, 16.0 * F.cells(), strm,
                (pt_interp<<<nblk(F.cells()), kPT, 0, strm>>>(A.parent, A.pn[0], A.pn[1], A.pn[2], A.origin[0],
                                                              A.origin[1], A.origin[2], A.periodic, F.m, F.u,
                                                              F.n[0], F.n[1], F.n[2], A.init_parent)));
    // the unknowns of each level and colour
    if (cudaMemsetAsync(counts, 0, 2 * lev.size() * sizeof(int), strm) != cudaSuccess) return ISIS_ECUDA;
    for (size_t l = 0; l < lev.size(); ++l) {
      const PLevel& L = lev[l];
      ISIS_LAUNCH(KK_PATCH_OTHER, 8.0 * L.cells(), strm,
                  (pt_compact<<<nblk(L.cells()), kPT, 0, strm>>>(L.view(false), L.list[0], L.list[1],
                                                                 counts + 2 * l)));
    }
    // FP32 copies of the masks (exact: means of +-1 over 8^l cells) and of the symmetron's density
    if (A.prec == ISIS_F32_REFINE64) {
      for (size_t l = 0; l < lev.size(); ++l) {
        const PLevel& L = lev[l];
        ISIS_LAUNCH(KK_PATCH_OTHER, 12.0 * L.cells(), strm,
                    (pt_to_f32<<<nblk(L.cells()), kPT, 0, strm>>>(L.m, L.m32, L.cells())));
        if (L.eta32)
          ISIS_LAUNCH(KK_PATCH_OTHER, 12.0 * L.cells(), strm,
                      (pt_to_f32<<<nblk(L.cells()), kPT, 0, strm>>>(L.eta, L.eta32, L.cells())));
      }
    }
    std::vector<int> hc(2 * lev.size());
    if (cudaMemcpyAsync(hc.data(), counts, hc.size() * sizeof(int), cudaMemcpyDeviceToHost, strm) != cudaSuccess ||
        cudaStreamSynchronize(strm) != cudaSuccess)
      return ISIS_ECUDA;
    for (size_t l = 0; l < lev.size(); ++l) {
      lev[l].count[0] = hc[2 * l];
      lev[l].count[1] = hc[2 * l + 1];
    }
    return ISIS_OK;
  }

  isis_status reference(isis_solve_info& info) {
    const PLevel& F = lev[0];
    ISIS_LAUNCH(KK_PATCH_OTHER, 17.0 * F.cells(), strm,
                (pt_ref<<<kPNormBlocks, kPT, 0, strm>>>(F.m, F.eta, F.cells(), A.eref, part)));
    double s = 0.0;
    isis_status st = sum_parts(&s);
    if (st != ISIS_OK) return st;
    info.res_ref = A.unknowns > 0 ? A.ref_scale * std::sqrt(s / (double)A.unknowns) : 0.0;
    return ISIS_OK;
  }

  isis_status run() {
    isis_solve_info info;
    std::memset(&info, 0, sizeof(info));
    isis_status st = setup();
    if (st != ISIS_OK) return st;
    st = reference(info);
    if (st != ISIS_OK) return st;
    if (A.prec == ISIS_F32_REFINE64) {
      st = run_refine(info);
      if (A.info) *A.info = info;
      return st;
    }
    double res = 0.0;
    st = norm(&res);
    if (st != ISIS_OK) return st;
    info.res0 = res;
    if (!(info.res_ref > 0.0)) info.res_ref = res;
    info.res_final = res;
    if (A.unknowns == 0 || res <= A.tol * info.res_ref) {
      st = ISIS_OK;
    } else if (!std::isfinite(res)) {
      st = ISIS_ENAN;
    } else {
      st = ISIS_ENOCONV;
      for (int cyc = 0; cyc < A.max_cycles; ++cyc) {
        isis_status vs = cycle_graphed([&] { return vcycle(0); });
        if (vs != ISIS_OK) return vs;
        vs = norm(&res);
        if (vs != ISIS_OK) return vs;
        if (cyc < 128) info.hist[cyc] = res;
        info.nhist = cyc + 1 < 128 ? cyc + 1 : 128;
        info.cycles = cyc + 1;
        info.res_final = res;
        if (!std::isfinite(res)) { st = ISIS_ENAN; break; }
        if (res <= A.tol * info.res_ref) { st = ISIS_OK; break; }
      }
    }
    if (A.info) *A.info = info;
    return st;
  }

  // Defect correction: the FP64 residual r = -L(u) at the unknowns, then FP32 V-cycles of the
  // correction problem L(B + e) - L(B) = r about B = fp32(u) (the same patch FAS in the DELTA form), then
  // u += e; until the FP64 residual meets the tolerance.  One synchronisation per outer iteration.
  isis_status run_refine(isis_solve_info& info) {
    const PLevel& F = lev[0];
    const size_t n = F.cells();
    isis_status st = ISIS_ENOCONV;
    double prev_res = 0.0;
    int prev_k = 0;
    for (int outer = 0;; ++outer) {
      ISIS_LAUNCH(KK_PATCH_OTHER, 48.0 * n, strm,
                  (pt_resid<M, FIELD, double><<<nblk(n), kPT, 0, strm>>>(F.view(false), A.coef, F.res)));
      ISIS_LAUNCH(KK_PATCH_OTHER, 8.0 * n, strm, (pt_sumsq<<<kPNormBlocks, kPT, 0, strm>>>(F.res, n, part)));
      double s = 0.0;
      st = sum_parts(&s);
      if (st != ISIS_OK) return st;
      const double res = A.unknowns > 0 ? std::sqrt(s / (double)A.unknowns) : 0.0;
      if (outer == 0) {
        info.res0 = res;
        if (!(info.res_ref > 0.0)) info.res_ref = res;
      } else if (outer <= 128) {
        info.hist[outer - 1] = res;
        info.nhist = outer;
      }
      info.res_final = res;
      if (A.unknowns == 0 || res <= A.tol * info.res_ref) { st = ISIS_OK; break; }
      if (!std::isfinite(res)) { st = ISIS_ENAN; break; }
      if (info.cycles >= A.max_cycles) { st = ISIS_ENOCONV; break; }
      ISIS_LAUNCH(KK_PATCH_OTHER, 28.0 * n, strm,
                  (pt_prep32<<<nblk(n), kPT, 0, strm>>>(F.u, F.res, F.B, F.e, F.sig32, n)));
      for (size_t l = 1; l < lev.size(); ++l) {
        const PLevel& C = lev[l];
        ISIS_LAUNCH(KK_PATCH_OTHER, 4.5 * C.cells() * 8.0, strm,
                    (pt_restrict<float><<<nblk(C.cells()), kPT, 0, strm>>>(lev[l - 1].B, C.B, C.n[0], C.n[1],
                                                                          C.n[2])));
      }
      // inner cycles; after the first outer iteration, only as many as the measured contraction per cycle
      // says reach half the target
      int k = A.inner;
      if (prev_res > 0.0 && prev_k > 0 && res < prev_res) {
        const double rho = std::pow(res / prev_res, 1.0 / prev_k);
        if (rho > 0.0 && rho < 1.0) {
          const double need = std::ceil(std::log(0.5 * A.tol * info.res_ref / res) / std::log(rho));
          if (need >= 1.0 && need < (double)k) k = (int)need;
        }
      }
      k = std::min(k, A.max_cycles - info.cycles);
      prev_res = res;
      prev_k = k;
      for (int c = 0; c < k; ++c) {
        st = cycle_graphed([&] { return vcycle32(0); });
        if (st != ISIS_OK) return st;
      }
      ISIS_LAUNCH(KK_PATCH_OTHER, 20.0 * n, strm, (pt_add_correction<<<nblk(n), kPT, 0, strm>>>(F.u, F.e, n)));
      info.cycles += k;
      info.outer = outer + 1;
    }
    return st;
  }
};

template <Model M>
isis_status patch_solve(const PatchArgs& A) {
  PatchSolver<M> S(A);
  const bool mixed = A.prec == ISIS_F32_REFINE64;
  // level dimensions
  int n[3] = {2 * A.n[0], 2 * A.n[1], 2 * A.n[2]};
  double h = A.h;
  size_t total = 0, floats = 0;
  for (int l = 0;; ++l) {
    PLevel L;
    std::memcpy(L.n, n, sizeof(n));
    L.h = h;
    S.lev.push_back(L);
    total += L.cells() * (l == 0 ? 4 : 7);
    if (mixed) floats += L.cells() * ((l == 0 ? 6 : 7) + (M == SYM ? 1 : 0));
    const int mn = std::min(n[0], std::min(n[1], n[2]));
    if ((n[0] & 1) || (n[1] & 1) || (n[2] & 1) || mn < 8 || l == 15) break;
    n[0] /= 2;
    n[1] /= 2;
    n[2] /= 2;
    h *= 2.0;
  }
  total += kPNormBlocks;
  size_t ints = 2 * S.lev.size();  // counts
  for (const PLevel& L : S.lev) ints += 2 * (L.cells() / 2 + 1);
  total += (ints + 1) / 2;
  total += (floats + 1) / 2;
  double* mem = nullptr;
  if (cudaMallocAsync((void**)&mem, total * sizeof(double), A.st) != cudaSuccess) {
    cudaGetLastError();
    return ISIS_ENOMEM;
  }
  double* p = mem;
  for (size_t l = 0; l < S.lev.size(); ++l) {
    PLevel& L = S.lev[l];
    const size_t c = L.cells();
    L.m = p; p += c;
    L.u0 = p; p += c;
    L.res = p; p += c;
    L.pre = p; p += c;
    if (l == 0) {
      L.eta = const_cast<double*>(A.eta);
      L.u = A.phi;
      L.sig = nullptr;  // the finest level's Sigma is 0
    } else {
      L.eta = p; p += c;
      L.u = p; p += c;
      L.sig = p; p += c;
    }
  }
  S.part = p;
  p += kPNormBlocks;
  int* ip = reinterpret_cast<int*>(p);
  S.counts = ip;
  ip += 2 * S.lev.size();
  for (PLevel& L : S.lev) {
    L.list[0] = ip;
    ip += L.cells() / 2 + 1;
    L.list[1] = ip;
    ip += L.cells() / 2 + 1;
  }
  p += (ints + 1) / 2;
  if (mixed) {
    float* fp = reinterpret_cast<float*>(p);
    for (size_t l = 0; l < S.lev.size(); ++l) {
      PLevel& L = S.lev[l];
      const size_t c = L.cells();
      L.m32 = fp; fp += c;
      L.e = fp; fp += c;
      L.sig32 = fp; fp += c;
      L.res32 = fp; fp += c;
      L.pre32 = fp; fp += c;
      L.B = fp; fp += c;
      if (l > 0) { L.e0 = fp; fp += c; }
      if (M == SYM) { L.eta32 = fp; fp += c; }
    }
  }
  isis_status st = ISIS_OK;
  const void* smem_kernel = mixed ? (const void*)pt_coarsest_smem<M, DELTA, float>
                                  : (const void*)pt_coarsest_smem<M, FIELD, double>;
  if (cudaFuncSetAttribute(smem_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kCoarseSmem) !=
      cudaSuccess) {
    cudaGetLastError();
    st = ISIS_ECUDA;
  }
  if (st == ISIS_OK && cudaMallocHost((void**)&S.host, kPNormBlocks * sizeof(double)) != cudaSuccess) {
    cudaGetLastError();
    st = ISIS_ENOMEM;
  }
  if (st == ISIS_OK) st = S.run();
  cudaFreeAsync(mem, A.st);
  if (S.host) {
    cudaStreamSynchronize(A.st);
    cudaFreeHost(S.host);
  }
  if (st == ISIS_ECUDA) cudaGetLastError();
  return st;
}

}  // namespace

isis_status run_patch_poi(const PatchArgs& A) { return patch_solve<POI>(A); }
isis_status run_patch_sym(const PatchArgs& A) { return patch_solve<SYM>(A); }
isis_status run_patch_fofr(const PatchArgs& A) { return patch_solve<FOFR>(A); }

}  // namespace isis
