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
//
// Memory layout.  FP64 grids (the caller's arrays, the FP64 solver) are
// row-major.  FP32 grids (the workspace of the FP32 cycles) are stored
// red/black split: red cells ((i+j+k) even) first, then black, each half in
// row-major order of the cells of that colour, i.e. cell g = (i N + j) N + k
// sits at colour * N^3/2 + g/2.  A one-colour half-sweep then reads the
// other colour's half and its own half contiguously, with no wasted sectors.
#pragma once
#include "isis_ff.cuh"
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
  T* aux;          // f(R): e^x (FIELD) or e^B expm1(x) (DELTA), kept in step with x
};

__device__ __forceinline__ size_t cidx(int lg, int i, int j, int k) {
  return ((((size_t)i << lg) + (size_t)j) << lg) + (size_t)k;
}

// Storage index of cell (i,j,k) in a grid of element type T (see above).
// FP32 grids have N <= 1024, so their indices fit in 32 bits.
template <class T>
__device__ __forceinline__ size_t lidx(int lg, int i, int j, int k) {
  if constexpr (sizeof(T) == 4) {
    const unsigned g = (((unsigned)i << lg | (unsigned)j) << lg) | (unsigned)k;
    return (size_t)((((unsigned)(i + j + k) & 1u) << (3 * lg - 1)) | (g >> 1));
  } else {
    return cidx(lg, i, j, k);
  }
}

// Storage indices of cell (i,j,k) and of its six neighbours (i+1, i-1, j+1,
// j-1, k+1, k-1) with periodic wrap.  For the red/black FP32 layout the
// neighbours all lie in the other colour's half: 32-bit arithmetic on the
// row index and k/2.
template <class T>
__device__ __forceinline__ size_t stencil_idx(int lg, int i, int j, int k, size_t* nb) {
  const int m = (1 << lg) - 1;
  if constexpr (sizeof(T) == 4) {
    const unsigned hN = 1u << (lg - 1), half = 1u << (3 * lg - 1);
    const unsigned ui = (unsigned)i, uj = (unsigned)j, uk = (unsigned)k, um = (unsigned)m;
    const unsigned col = (ui + uj + uk) & 1u, oth = col ? 0u : half;
    const unsigned row = (ui << lg) | uj, k2 = uk >> 1;
    nb[0] = oth + ((((ui + 1) & um) << lg | uj) << (lg - 1)) + k2;
    nb[1] = oth + ((((ui - 1) & um) << lg | uj) << (lg - 1)) + k2;
    nb[2] = oth + (((ui << lg) | ((uj + 1) & um)) << (lg - 1)) + k2;
    nb[3] = oth + (((ui << lg) | ((uj - 1) & um)) << (lg - 1)) + k2;
    nb[4] = oth + (row << (lg - 1)) + (((uk + 1) & um) >> 1);
    nb[5] = oth + (row << (lg - 1)) + (((uk - 1) & um) >> 1);
    (void)hN;
    return (col ? half : 0u) + (row << (lg - 1)) + k2;
  } else {
    nb[0] = cidx(lg, (i + 1) & m, j, k);
    nb[1] = cidx(lg, (i - 1) & m, j, k);
    nb[2] = cidx(lg, i, (j + 1) & m, k);
    nb[3] = cidx(lg, i, (j - 1) & m, k);
    nb[4] = cidx(lg, i, j, (k + 1) & m);
    nb[5] = cidx(lg, i, j, (k - 1) & m);
    return cidx(lg, i, j, k);
  }
}

// Cell (i,j,k) stored at position t of a grid of type T (inverse of lidx).
template <class T>
__device__ __forceinline__ void cell_of(size_t t, int lg, int& i, int& j, int& k) {
  const int m = (1 << lg) - 1;
  if constexpr (sizeof(T) == 4) {
    const unsigned half = 1u << (3 * lg - 1), u = (unsigned)t;
    const unsigned col = u >= half ? 1u : 0u, l = u - col * half;
    const unsigned k2 = l & ((1u << (lg - 1)) - 1), row = l >> (lg - 1);
    j = (int)(row & (unsigned)m);
    i = (int)(row >> lg);
    k = (int)(2 * k2 + (((unsigned)i + (unsigned)j + col) & 1u));
  } else {
    k = (int)(t & m);
    j = (int)((t >> lg) & m);
    i = (int)(t >> (2 * lg));
  }
}

// Neighbours of the cell stored at position t (storage order), for kernels
// whose threads run over a grid in storage order.  Red/black FP32: cell t of
// colour col sits in row r = i N + j at place k2 of that colour; its i and j
// neighbours are at the same place in rows r +- N, r +- 1 of the other
// colour, its k neighbours at places k2 + par, k2 + par - 1 of its own row.
template <class T>
__device__ __forceinline__ void stencil_of_storage(int lg, size_t t, size_t* nb) {
  if constexpr (sizeof(T) == 4) {
    const unsigned half = 1u << (3 * lg - 1), hN = 1u << (lg - 1), m = (1u << lg) - 1;
    const unsigned u = (unsigned)t, col = u >= half ? 1u : 0u, l = u - (col ? half : 0u);
    const unsigned k2 = l & (hN - 1), row = l >> (lg - 1), j = row & m, i = row >> lg;
    const unsigned par = (i + j + col) & 1u, oth = col ? 0u : half;
    nb[0] = oth + ((((i + 1) & m) << lg | j) << (lg - 1)) + k2;
    nb[1] = oth + ((((i - 1) & m) << lg | j) << (lg - 1)) + k2;
    nb[2] = oth + (((i << lg) | ((j + 1) & m)) << (lg - 1)) + k2;
    nb[3] = oth + (((i << lg) | ((j - 1) & m)) << (lg - 1)) + k2;
    nb[4] = oth + (row << (lg - 1)) + ((k2 + par) & (hN - 1));
    nb[5] = oth + (row << (lg - 1)) + ((k2 + par - 1) & (hN - 1));
  } else {
    int i, j, k;
    cell_of<T>(t, lg, i, j, k);
    stencil_idx<T>(lg, i, j, k, nb);
  }
}

// The f(R) per-cell exponentials of a gathered cell, from its values: e^x in the
// field form; w = e^B and m = w expm1(e) in the correction form.  Evaluated where
// they are used (one MUFU exponential each) instead of being kept in grids: the
// sweeps then read two grids of the other colour instead of four.
template <Model M, Form FM, class T>
__device__ __forceinline__ void fill_exps(Cell<T>& q) {
  if constexpr (M == FOFR) {
    if constexpr (FM == DELTA) {
      q.w = dexp<T>(q.B);
#pragma unroll
      for (int d = 0; d < 6; ++d) q.wn[d] = dexp<T>(q.Bn[d]);
    } else {
      q.w = T(0);
#pragma unroll
      for (int d = 0; d < 6; ++d) q.wn[d] = T(0);
    }
    q.a = aux_of<M, FM, T>(q.x, q.w);
#pragma unroll
    for (int d = 0; d < 6; ++d) q.an[d] = aux_of<M, FM, T>(q.xn[d], q.wn[d]);
  }
}

// FP64 grids keep e^x of every cell in L.aux (the FP64 path runs the field form only):
// an FP64 exponential per neighbour would cost more than the extra reads.
template <class T>
constexpr bool kExpCache = sizeof(T) == 8;

template <Model M, Form FM, class T, class IDX>
__device__ __forceinline__ void load_or_fill_exps(const LevelView<T>& L, IDX c, const IDX* nb, Cell<T>& q) {
  if constexpr (M == FOFR && kExpCache<T>) {
    q.w = T(0);
    q.a = L.aux[c];
#pragma unroll
    for (int d = 0; d < 6; ++d) {
      q.wn[d] = T(0);
      q.an[d] = L.aux[nb[d]];
    }
  } else {
    fill_exps<M, FM, T>(q);
  }
}

// Gather the cell stored at t and its neighbours.
template <Model M, Form FM, class T>
__device__ __forceinline__ Cell<T> gather_at(const LevelView<T>& L, size_t c) {
  size_t nb[6];
  stencil_of_storage<T>(L.lg, c, nb);
  Cell<T> q;
  q.x = L.x[c];
#pragma unroll
  for (int d = 0; d < 6; ++d) q.xn[d] = L.x[nb[d]];
  q.sig = L.sig ? L.sig[c] : T(0);
  if constexpr (uses_eta<M, FM>()) q.eta = L.eta[c]; else q.eta = T(0);
  if constexpr (FM == DELTA && M != POI) q.B = L.B[c]; else q.B = T(0);
  if constexpr (FM == DELTA && M == FOFR) {
#pragma unroll
    for (int d = 0; d < 6; ++d) q.Bn[d] = L.B[nb[d]];
  }
  load_or_fill_exps<M, FM, T, size_t>(L, c, nb, q);
  return q;
}

// Gather one cell and its neighbours from global memory (periodic wrap).
template <Model M, Form FM, class T>
__device__ __forceinline__ Cell<T> gather(const LevelView<T>& L, int i, int j, int k) {
  size_t nb[6];
  const size_t c = stencil_idx<T>(L.lg, i, j, k, nb);
  Cell<T> q;
  q.x = L.x[c];
#pragma unroll
  for (int d = 0; d < 6; ++d) q.xn[d] = L.x[nb[d]];
  q.sig = L.sig ? L.sig[c] : T(0);
  if constexpr (uses_eta<M, FM>()) q.eta = L.eta[c]; else q.eta = T(0);
  if constexpr (FM == DELTA && M != POI) q.B = L.B[c]; else q.B = T(0);
  if constexpr (FM == DELTA && M == FOFR) {
#pragma unroll
    for (int d = 0; d < 6; ++d) q.Bn[d] = L.B[nb[d]];
  }
  load_or_fill_exps<M, FM, T, size_t>(L, c, nb, q);
  return q;
}

// One colour (0 = red: (i+j+k) even) of a Newton-Gauss-Seidel sweep, in place.
// Thread t updates the cell of the requested colour in the pair (k = 2p, 2p+1)
// of row t / (N/2); for FP32 grids t is also that cell's place in its colour
// half, so a warp reads and writes 32 consecutive values of each array.
template <Model M, Form FM, class T>
__global__ void smooth_color(LevelView<T> L, CoefT<T> c, int color) {
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
  // FP32 cycles drive a correction: a 2-ulp quotient is ample there
  T xn;
  if constexpr (sizeof(T) == 4) xn = q.x - __fdividef(F, dF);
  else xn = q.x - F / dF;
  const size_t o = lidx<T>(L.lg, i, j, k);
  L.x[o] = xn;
  if constexpr (M == FOFR && kExpCache<T>) L.aux[o] = aux_of<M, FM, T>(xn, q.w);
}

// One colour of a Newton-Gauss-Seidel sweep on a red/black split FP32 grid.
// Thread t owns cell t of the colour's half: row r = t / (N/2) = i N + j,
// k = 2 (t mod N/2) + ((i + j + colour) mod 2).  Its i and j neighbours are
// cells of the other colour in rows r +- N and r +- 1 at the same place in
// the row; its k neighbours are places k2 + par and k2 + par - 1 of its own
// row in the other colour's half (par = parity of k), all in 32-bit
// arithmetic.
template <Model M, Form FM>
__global__ void __launch_bounds__(256) smooth_rb(LevelView<float> L, CoefT<float> c, int color) {
  const int lg = L.lg;
  const unsigned half = 1u << (3 * lg - 1), hN = (unsigned)L.N >> 1, m = (unsigned)L.N - 1;
  const unsigned t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= half) return;
  const unsigned k2 = t & (hN - 1), row = t >> (lg - 1), j = row & m, i = row >> lg;
  const unsigned par = (i + j + (unsigned)color) & 1u;
  const unsigned own = color ? half : 0u, oth = color ? 0u : half;
  const unsigned rip = (((i + 1) & m) << lg | j) * hN + k2, rim = (((i - 1) & m) << lg | j) * hN + k2;
  const unsigned rjp = ((i << lg) | ((j + 1) & m)) * hN + k2, rjm = ((i << lg) | ((j - 1) & m)) * hN + k2;
  const unsigned rkp = row * hN + ((k2 + par) & (hN - 1)), rkm = row * hN + ((k2 + par - 1) & (hN - 1));
  const unsigned nb[6] = {oth + rip, oth + rim, oth + rjp, oth + rjm, oth + rkp, oth + rkm};
  const unsigned o = own + t;
  Cell<float> q;
  q.x = L.x[o];
#pragma unroll
  for (int d = 0; d < 6; ++d) q.xn[d] = L.x[nb[d]];
  q.sig = L.sig ? L.sig[o] : 0.f;
  if constexpr (uses_eta<M, FM>()) q.eta = L.eta[o]; else q.eta = 0.f;
  if constexpr (FM == DELTA && M != POI) q.B = L.B[o]; else q.B = 0.f;
  if constexpr (FM == DELTA && M == FOFR) {
#pragma unroll
    for (int d = 0; d < 6; ++d) q.Bn[d] = L.B[nb[d]];
  }
  fill_exps<M, FM, float>(q);
  float F, dF;
  eval_cell<M, FM, float>(c, L.ih2, q, F, dF);
  // FP32 cycles drive a correction: a 2-ulp quotient is ample there
  const float xn = q.x - __fdividef(F, dF);
  L.x[o] = xn;
}

// Storage positions of the cells k = 2K-1, 2K, 2K+1, 2K+2 of row (i, j).
template <class T>
__device__ __forceinline__ void row4(int lg, int i, int j, int K, size_t* p) {
  if constexpr (sizeof(T) == 4) {
    const unsigned half = 1u << (3 * lg - 1), hm = (1u << (lg - 1)) - 1;
    const unsigned rp = (((unsigned)i << lg) | (unsigned)j) << (lg - 1);
    const unsigned ev = ((unsigned)(i + j) & 1u) ? half : 0u, od = ev ? 0u : half;  // colour halves of even / odd k
    p[0] = od + rp + (((unsigned)K - 1u) & hm);
    p[1] = ev + rp + (unsigned)K;
    p[2] = od + rp + (unsigned)K;
    p[3] = ev + rp + (((unsigned)K + 1u) & hm);
  } else {
    const int m = (1 << lg) - 1;
    const size_t rb = (((size_t)i << lg) + (size_t)j) << lg;
#pragma unroll
    for (int d = 0; d < 4; ++d) p[d] = rb + (size_t)((2 * K - 1 + d) & m);
  }
}

// Same half-sweep, two cells of the colour per thread (places k2a, k2a + 1
// of a row, float2 loads and stores; N >= 4).  The k neighbours of the pair
// are the other colour's places k2a + par - 1 .. k2a + par + 1.
template <Model M, Form FM, bool kFill = true>
__device__ __forceinline__ unsigned rb2_gather(const LevelView<float>& L, int color, unsigned t, Cell<float>& q0,
                                               Cell<float>& q1) {
  const int lg = L.lg;
  const unsigned half = 1u << (3 * lg - 1), hN = (unsigned)L.N >> 1, m = (unsigned)L.N - 1;
  const unsigned k2a = (t & ((hN >> 1) - 1)) << 1, row = t >> (lg - 2), j = row & m, i = row >> lg;
  const unsigned par = (i + j + (unsigned)color) & 1u;
  const unsigned own = color ? half : 0u, oth = color ? 0u : half;
  const unsigned o = own + row * hN + k2a;
  const unsigned pr[4] = {oth + ((((i + 1) & m) << lg) | j) * hN + k2a, oth + ((((i - 1) & m) << lg) | j) * hN + k2a,
                          oth + ((i << lg) | ((j + 1) & m)) * hN + k2a, oth + ((i << lg) | ((j - 1) & m)) * hN + k2a};
  const unsigned rk = oth + row * hN;
  const unsigned ks = par ? ((k2a + 2) & (hN - 1)) : ((k2a - 1) & (hN - 1));  // the scalar k neighbour place
  // six neighbours of both cells from one array of the other colour
  auto nbrs = [&](const float* __restrict__ a, float* n0, float* n1) {
#pragma unroll
    for (int d = 0; d < 4; ++d) {
      const float2 v = *reinterpret_cast<const float2*>(a + pr[d]);
      n0[d] = v.x;
      n1[d] = v.y;
    }
    const float2 v = *reinterpret_cast<const float2*>(a + rk + k2a);
    const float sc = a[rk + ks];
    if (par) { n0[4] = v.y; n0[5] = v.x; n1[4] = sc; n1[5] = v.y; }
    else { n0[4] = v.x; n0[5] = sc; n1[4] = v.y; n1[5] = v.x; }
  };
  const float2 x2 = *reinterpret_cast<const float2*>(L.x + o);
  q0.x = x2.x;
  q1.x = x2.y;
  nbrs(L.x, q0.xn, q1.xn);
  if (L.sig) {
    const float2 v = *reinterpret_cast<const float2*>(L.sig + o);
    q0.sig = v.x;
    q1.sig = v.y;
  } else {
    q0.sig = q1.sig = 0.f;
  }
  if constexpr (uses_eta<M, FM>()) {
    const float2 v = *reinterpret_cast<const float2*>(L.eta + o);
    q0.eta = v.x;
    q1.eta = v.y;
  } else {
    q0.eta = q1.eta = 0.f;
  }
  if constexpr (FM == DELTA && M != POI) {
    const float2 v = *reinterpret_cast<const float2*>(L.B + o);
    q0.B = v.x;
    q1.B = v.y;
  } else {
    q0.B = q1.B = 0.f;
  }
  if constexpr (FM == DELTA && M == FOFR) nbrs(L.B, q0.Bn, q1.Bn);
  if constexpr (kFill) {
    fill_exps<M, FM, float>(q0);
    fill_exps<M, FM, float>(q1);
  }
  return o;
}

// ---- f(R) on the pair of cells of an rb2 thread, in packed FP32x2 arithmetic ----
// Both cells go through the same operations, so they run as the two lanes of float2 instructions (one
// fused multiply-add, add or multiply for a pair of FP32 operations; sm_100 family).  The f(R) sweeps are
// bound by instruction issue, and this halves the issue count of their arithmetic.  The exponentials
// remain one MUFU operation per lane.
__device__ __forceinline__ float2 pk(float a, float b) { return make_float2(a, b); }
__device__ __forceinline__ float2 bc(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return __ffma2_rn(b, bc(-1.0f), a); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
// e^v = 2^(v log2 e): one packed multiply, then the hardware base-2 exponential (MUFU) of each lane.
// The .ftz form flushes subnormal inputs and results to zero (PTX ISA, ex2): it spares the subnormal
// handling around the MUFU operation.  A subnormal input gives 1 either way; a subnormal result needs
// v < -87, far outside the exponents of these fields (|u|, |B| and |u|/(n+1) stay below about 30).
__device__ __forceinline__ float ex2_approx(float t) {
  float r;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(t));
  return r;
}
__device__ __forceinline__ float2 exp_2(float2 v) {
  const float2 t = mul2(v, bc(1.4426950408889634f));
  return pk(ex2_approx(t.x), ex2_approx(t.y));
}

// e^v - 1 of both lanes by the series of dexpm1<float> of a fixed degree: DEG 3 for |v| <= 2^-7, DEG 8 for
// |v| <= 1/2, DEG 0 for expf(v) - 1.
template <int DEG>
__device__ __forceinline__ float2 expm1_2d(float2 v) {
  if constexpr (DEG == 3) {
    float2 p = fma2(v, bc(1.0f / 6.0f), bc(0.5f));
    p = fma2(p, v, bc(1.0f));
    return mul2(p, v);
  } else if constexpr (DEG == 8) {
    float2 p = fma2(v, bc(1.0f / 40320.0f), bc(1.0f / 5040.0f));
    p = fma2(p, v, bc(1.0f / 720.0f));
    p = fma2(p, v, bc(1.0f / 120.0f));
    p = fma2(p, v, bc(1.0f / 24.0f));
    p = fma2(p, v, bc(1.0f / 6.0f));
    p = fma2(p, v, bc(0.5f));
    p = fma2(p, v, bc(1.0f));
    return mul2(p, v);
  } else {
    return pk(expf(v.x) - 1.0f, expf(v.y) - 1.0f);
  }
}
// The same with the degree set by the larger |v| of the two lanes.
__device__ __forceinline__ float2 expm1_2(float2 v) {
  const float mx = fmaxf(fabsf(v.x), fabsf(v.y));
  if (mx <= 0.0078125f) return expm1_2d<3>(v);
  if (mx <= 0.5f) return expm1_2d<8>(v);
  return expm1_2d<0>(v);
}
// The largest of a non-negative float over the warp's lanes in `lanes` (non-negative floats order as their bits).
__device__ __forceinline__ float warp_max_nonneg(unsigned lanes, float v) {
  return __uint_as_float(__reduce_max_sync(lanes, __float_as_uint(v)));
}
// expm1_2 with the low degree taken only when every lane of the warp allows it: the threads of a warp then
// run one series rather than both in turn.  Degree 8 holds its bound for every |v| <= 1/2, the small ones
// included, so only lanes with |v| > 1/2 (rare) leave it for expf.
__device__ __forceinline__ float2 expm1_2w(unsigned lanes, float2 v) {
  const float mx = fmaxf(fabsf(v.x), fabsf(v.y));
  if (warp_max_nonneg(lanes, mx) <= 0.0078125f) return expm1_2d<3>(v);
  if (mx <= 0.5f) return expm1_2d<8>(v);
  return expm1_2d<0>(v);
}

// The correction-form flux sums of both cells with every e^e - 1 of one degree.  The face terms
// (1/2)(m + m_nb) dB + (1/2)(bt + bt_nb) de and (1/2) bt (dB + de) - (bt + bt_nb)/2 are summed through the
// five neighbour sums of dB, de, m_nb dB, bt_nb de and bt_nb, each term of which is of the size of the
// correction (no large terms cancel), at fewer operations per neighbour.
// em = e^{-e/(n+1)} - 1 of both cells comes with it, of the same degree (|e|/(n+1) <= |e|); the expf form
// (DEG 0) picks its own degree per lane.
template <int DEG>
__device__ __forceinline__ void fofr_delta_flux2(const Cell<float>& q0, const Cell<float>& q1, float2 x, float2 B,
                                                 float2 xm, float2& m, float2& flux, float2& dsum, float2& em) {
  em = DEG == 0 ? expm1_2(xm) : expm1_2d<DEG>(xm);
  const float2 w = exp_2(B);
  m = mul2(w, expm1_2d<DEG>(x));
  const float2 bt = add2(w, m);
  float2 sdB = bc(0.0f), sde = bc(0.0f), smn = bc(0.0f), sbn = bc(0.0f), sbt = bc(0.0f);
#pragma unroll
  for (int d = 0; d < 6; ++d) {
    const float2 Bn = pk(q0.Bn[d], q1.Bn[d]), en = pk(q0.xn[d], q1.xn[d]);
    const float2 wn = exp_2(Bn);
    const float2 mn = mul2(wn, expm1_2d<DEG>(en));
    const float2 btn = add2(wn, mn);
    const float2 dB = sub2(Bn, B), de = sub2(en, x);
    sdB = add2(sdB, dB);
    sde = add2(sde, de);
    smn = fma2(mn, dB, smn);
    sbn = fma2(btn, de, sbn);
    sbt = add2(sbt, btn);
  }
  const float2 half = bc(0.5f);
  // flux = (1/2) [m sum dB + bt sum de + sum m_nb dB + sum bt_nb de]
  flux = mul2(half, add2(fma2(m, sdB, mul2(bt, sde)), add2(smn, sbn)));
  // dsum = (1/2) bt (sum dB + sum de) - (6 bt + sum bt_nb) / 2
  dsum = sub2(mul2(mul2(half, bt), add2(sdB, sde)), mul2(half, fma2(bc(6.0f), bt, sbt)));
}

// F = L(x) - Sigma and dF = dL/dx of both cells (the f(R) operators of fofr_field_eval and fofr_delta_eval),
// from cells gathered without their exponentials.
// `lanes`: the warp's lanes that evaluate a pair here (the series degree is chosen per warp).
template <Form FM>
__device__ __forceinline__ void fofr_pair_eval(const CoefT<float>& c, float ih2, unsigned lanes, const Cell<float>& q0,
                                               const Cell<float>& q1, float2& F, float2& dF) {
  const float2 half = bc(0.5f);
  const float2 x = pk(q0.x, q1.x), sig = pk(q0.sig, q1.sig);
  float2 flux = bc(0.0f), dsum = bc(0.0f);
  if constexpr (FM == DELTA) {
    const float2 B = pk(q0.B, q1.B);
    // one series degree for the corrections of both cells and their neighbours
    float mx = fmaxf(fabsf(x.x), fabsf(x.y));
#pragma unroll
    for (int d = 0; d < 6; ++d) mx = fmaxf(mx, fmaxf(fabsf(q0.xn[d]), fabsf(q1.xn[d])));
    // one degree for the whole warp unless a lane needs expf (|e| > 1/2): then degree 8 or expf per lane
    const float2 minv = bc(-c.inv_np1), xm = mul2(x, minv);
    float2 m, em;
    if (warp_max_nonneg(lanes, mx) <= 0.0078125f) fofr_delta_flux2<3>(q0, q1, x, B, xm, m, flux, dsum, em);
    else if (mx <= 0.5f) fofr_delta_flux2<8>(q0, q1, x, B, xm, m, flux, dsum, em);
    else fofr_delta_flux2<0>(q0, q1, x, B, xm, m, flux, dsum, em);
    const float2 exB = exp_2(mul2(B, minv));
    const float2 K2 = bc(c.K2);
    F = sub2(fma2(flux, bc(ih2), mul2(K2, mul2(exB, em))), sig);
    dF = sub2(mul2(dsum, bc(ih2)), mul2(mul2(K2, bc(c.inv_np1)), mul2(exB, add2(em, bc(1.0f)))));
  } else {
    // flux = (1/2) [ex sum du + sum ex_nb du], dsum = (1/2) ex sum du - (6 ex + sum ex_nb) / 2
    const float2 ex = exp_2(x), hex = mul2(half, ex);
    float2 sdu = bc(0.0f), sexdu = bc(0.0f), sex = bc(0.0f);
#pragma unroll
    for (int d = 0; d < 6; ++d) {
      const float2 xn = pk(q0.xn[d], q1.xn[d]);
      const float2 du = sub2(xn, x), exn = exp_2(xn);
      sdu = add2(sdu, du);
      sexdu = fma2(exn, du, sexdu);
      sex = add2(sex, exn);
    }
    flux = fma2(hex, sdu, mul2(half, sexdu));
    dsum = sub2(mul2(hex, sdu), mul2(half, fma2(bc(6.0f), ex, sex)));
    const float2 fs = bc(c.fscale);
    flux = mul2(flux, fs);
    dsum = mul2(dsum, fs);
    const float2 inp1 = bc(c.inv_np1), Kx = bc(c.fKx);
    const float2 em = expm1_2w(lanes, mul2(x, bc(-c.inv_np1)));
    const float2 S = add2(sub2(mul2(bc(c.K1), sub2(pk(q0.eta, q1.eta), bc(1.0f))), mul2(Kx, em)),
                          bc(c.fK3x));
    F = sub2(sub2(mul2(flux, bc(ih2)), S), sig);
    dF = sub2(mul2(dsum, bc(ih2)), mul2(mul2(Kx, inp1), add2(em, bc(1.0f))));
  }
}

// Gather and evaluate the two cells of an rb2 thread: the packed path for f(R), two eval_cell otherwise.
// `lanes`: the lanes of the calling warp that are here (all of them call with the same mask).
template <Model M, Form FM>
__device__ __forceinline__ unsigned rb2_eval(const LevelView<float>& L, const CoefT<float>& c, int color, unsigned t,
                                             unsigned lanes, Cell<float>& q0, Cell<float>& q1, float2& F,
                                             float2& dF) {
  if constexpr (M == FOFR) {
    const unsigned o = rb2_gather<M, FM, false>(L, color, t, q0, q1);
    fofr_pair_eval<FM>(c, L.ih2, lanes, q0, q1, F, dF);
    return o;
  } else {
    (void)lanes;
    const unsigned o = rb2_gather<M, FM>(L, color, t, q0, q1);
    eval_cell<M, FM, float>(c, L.ih2, q0, F.x, dF.x);
    eval_cell<M, FM, float>(c, L.ih2, q1, F.y, dF.y);
    return o;
  }
}

template <Model M, Form FM>
__global__ void __launch_bounds__(256) smooth_rb2(LevelView<float> L, CoefT<float> c, int color) {
  const unsigned t = blockIdx.x * blockDim.x + threadIdx.x;
  const unsigned lanes = __ballot_sync(0xffffffffu, t < (1u << (3 * L.lg - 2)));  // blocks of whole warps
  if (t >= (1u << (3 * L.lg - 2))) return;
  Cell<float> q0, q1;
  float2 F, dF;
  const unsigned o = rb2_eval<M, FM>(L, c, color, t, lanes, q0, q1, F, dF);
  // FP32 cycles drive a correction: a 2-ulp quotient is ample there
  const float xn0 = q0.x - __fdividef(F.x, dF.x), xn1 = q1.x - __fdividef(F.y, dF.y);
  *reinterpret_cast<float2*>(L.x + o) = make_float2(xn0, xn1);
}

// Residual r = Sigma - L(x) of every cell of a red/black FP32 grid into res
// (two cells per thread; threads [0, N^3/4) red, then black).
template <Model M, Form FM>
__global__ void __launch_bounds__(256) resid_rb2(LevelView<float> L, CoefT<float> c, float* __restrict__ res) {
  const unsigned q4 = 1u << (3 * L.lg - 2);
  unsigned t = blockIdx.x * blockDim.x + threadIdx.x;
  const unsigned lanes = __ballot_sync(0xffffffffu, t < 2 * q4);  // blocks of whole warps
  if (t >= 2 * q4) return;
  const int color = t >= q4 ? 1 : 0;
  t -= color ? q4 : 0u;
  Cell<float> q0, q1;
  float2 F, dF;
  const unsigned o = rb2_eval<M, FM>(L, c, color, t, lanes, q0, q1, F, dF);
  *reinterpret_cast<float2*>(res + o) = make_float2(-F.x, -F.y);  // Sigma is inside F
}

// x_H = R x, x0_H = x_H, Sigma_H = R res (res from resid_rb2), f(R) cache of x_H;
// one thread per coarse cell in row-major order.
template <Model M, Form FM>
__global__ void restrict_xr(LevelView<float> F, const float* __restrict__ res, LevelView<float> C,
                            float* __restrict__ x0c, float* __restrict__ sigc) {
  const int lgc = F.lg - 1, lg = F.lg, m = F.N - 1, mc = (1 << lgc) - 1;
  size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= ((size_t)1 << (3 * lgc))) return;
  const int K = (int)(t & mc), J = (int)((t >> lgc) & mc), I = (int)(t >> (2 * lgc));
  float xs = 0.f, rs = 0.f;
#pragma unroll
  for (int a = 0; a < 2; ++a)
#pragma unroll
    for (int b = 0; b < 2; ++b) {
      size_t p[4];
      row4<float>(lg, (2 * I + a) & m, (2 * J + b) & m, K, p);
      xs += F.x[p[1]] + F.x[p[2]];
      rs += res[p[1]] + res[p[2]];
    }
  const size_t to = lidx<float>(lgc, I, J, K);
  const float xr = xs * 0.125f;
  C.x[to] = xr;
  x0c[to] = xr;
  sigc[to] = rs * 0.125f;
}

// One thread per coarse cell (I,J,K): residuals r = Sigma - L(x) of its 8
// children, x_H = R x, x0_H = x_H, Sigma_H = R r.  The 32 fine cells the 8
// stencils touch (block a, b, d = 0..3 at i = 2I-1+a, j = 2J-1+b, k = 2K-1+d,
// without the 4 corner rows) are loaded once.
// FP32 (but the f(R) correction form, whose neighbours' B and e^B need more): at least three blocks of 256 per
// SM (at most 85 registers); the compiler would otherwise keep every loaded cell and exponential in flight at
// once (89 registers, two blocks, 1.35x the time at 512^3 for the f(R) field form).
template <Model M, Form FM, class T>
__global__ void __launch_bounds__(256, (sizeof(T) == 4 && !(M == FOFR && FM == DELTA)) ? 3 : 1)
    resid_restrict(LevelView<T> F, CoefT<T> c, LevelView<T> C, T* __restrict__ x0c, T* __restrict__ sigc) {
  constexpr bool kAllB = (FM == DELTA && M == FOFR);   // neighbours' B (and e^B) needed
  constexpr bool kAux = (M == FOFR);
  T* __restrict__ xc = C.x;
  const int lgc = F.lg - 1, lg = F.lg, m = F.N - 1;
  size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  const unsigned lanes = __ballot_sync(0xffffffffu, t < ((size_t)1 << (3 * lgc)));  // blocks of whole warps
  if (t >= ((size_t)1 << (3 * lgc))) return;
  // threads in row-major coarse order: neighbouring threads touch neighbouring fine cells
  const int mc = (1 << lgc) - 1;
  const int K = (int)(t & mc), J = (int)((t >> lgc) & mc), I = (int)(t >> (2 * lgc));
  const size_t to = lidx<T>(lgc, I, J, K);
  T X[4][4][4], Ax[4][4][4], Bx[4][4][4], Wx[4][4][4];
  // storage positions of the loaded cells (FP32 grids: N <= 1024, 32-bit positions, half the registers)
  using Idx = std::conditional_t<sizeof(T) == 4, unsigned, size_t>;
  Idx P[4][4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      const bool ea = (a == 0 || a == 3), eb = (b == 0 || b == 3);
      if (ea && eb) continue;  // corner rows: not in any stencil
      size_t p[4];
      row4<T>(lg, (2 * I - 1 + a) & m, (2 * J - 1 + b) & m, K, p);
#pragma unroll
      for (int d = 0; d < 4; ++d) {
        if ((ea || eb) && (d == 0 || d == 3)) continue;
        P[a][b][d] = (Idx)p[d];
        X[a][b][d] = F.x[p[d]];
        // the f(R) exponentials of each loaded cell, once for the 8 stencils (fill_exps)
        if constexpr (kAllB) { Bx[a][b][d] = F.B[p[d]]; Wx[a][b][d] = dexp<T>(Bx[a][b][d]); }
        if constexpr (kAux) {
          if constexpr (kExpCache<T>) Ax[a][b][d] = F.aux[p[d]];
          else Ax[a][b][d] = aux_of<M, FM, T>(X[a][b][d], kAllB ? Wx[a][b][d] : T(0));
        }
      }
    }
  T xs = 0, rs = 0;
  if constexpr (M == FOFR && FM == FIELD && sizeof(T) == 4) {
    // the f(R) field form in packed FP32x2: the children k = 2K, 2K+1 of each (i, j) row as the two lanes
    // (the algebra of fofr_pair_eval, with the loaded cells' exponentials)
    const float2 half = bc(0.5f), fs = bc(c.fscale), ih2 = bc(F.ih2);
    float2 xs2 = bc(0.f), rs2 = bc(0.f);
#pragma unroll
    for (int a = 1; a < 3; ++a)
#pragma unroll
      for (int b = 1; b < 3; ++b) {
        const float2 x2 = pk(X[a][b][1], X[a][b][2]), ex2 = pk(Ax[a][b][1], Ax[a][b][2]);
        const float2 xn[6] = {pk(X[a + 1][b][1], X[a + 1][b][2]), pk(X[a - 1][b][1], X[a - 1][b][2]),
                              pk(X[a][b + 1][1], X[a][b + 1][2]), pk(X[a][b - 1][1], X[a][b - 1][2]),
                              pk(X[a][b][2], X[a][b][3]), pk(X[a][b][0], X[a][b][1])};
        const float2 en[6] = {pk(Ax[a + 1][b][1], Ax[a + 1][b][2]), pk(Ax[a - 1][b][1], Ax[a - 1][b][2]),
                              pk(Ax[a][b + 1][1], Ax[a][b + 1][2]), pk(Ax[a][b - 1][1], Ax[a][b - 1][2]),
                              pk(Ax[a][b][2], Ax[a][b][3]), pk(Ax[a][b][0], Ax[a][b][1])};
        float2 sdu = bc(0.f), sexdu = bc(0.f);
#pragma unroll
        for (int d = 0; d < 6; ++d) {
          const float2 du = sub2(xn[d], x2);
          sdu = add2(sdu, du);
          sexdu = fma2(en[d], du, sexdu);
        }
        const float2 flux = mul2(fs, fma2(mul2(half, ex2), sdu, mul2(half, sexdu)));
        const float2 em = expm1_2w(lanes, mul2(x2, bc(-c.inv_np1)));
        const float2 eta2 = pk(F.eta[P[a][b][1]], F.eta[P[a][b][2]]);
        const float2 sig2 = F.sig ? pk(F.sig[P[a][b][1]], F.sig[P[a][b][2]]) : bc(0.f);
        const float2 S = add2(sub2(mul2(bc(c.K1), sub2(eta2, bc(1.0f))), mul2(bc(c.fKx), em)), bc(c.fK3x));
        const float2 Fv = sub2(sub2(mul2(flux, ih2), S), sig2);
        xs2 = add2(xs2, x2);
        rs2 = sub2(rs2, Fv);  // r = Sigma - L(x)
      }
    xs = xs2.x + xs2.y;
    rs = rs2.x + rs2.y;
  } else {
  (void)lanes;
#pragma unroll
  for (int a = 1; a < 3; ++a)
#pragma unroll
    for (int b = 1; b < 3; ++b)
#pragma unroll
      for (int d = 1; d < 3; ++d) {
        Cell<T> q;
        const Idx pc = P[a][b][d];
        q.x = X[a][b][d];
        q.xn[0] = X[a + 1][b][d]; q.xn[1] = X[a - 1][b][d];
        q.xn[2] = X[a][b + 1][d]; q.xn[3] = X[a][b - 1][d];
        q.xn[4] = X[a][b][d + 1]; q.xn[5] = X[a][b][d - 1];
        q.sig = F.sig ? F.sig[pc] : T(0);
        if constexpr (uses_eta<M, FM>()) q.eta = F.eta[pc]; else q.eta = T(0);
        if constexpr (FM == DELTA && M != POI) q.B = F.B[pc]; else q.B = T(0);
        if constexpr (kAllB) {
          q.w = Wx[a][b][d];
          q.Bn[0] = Bx[a + 1][b][d]; q.Bn[1] = Bx[a - 1][b][d]; q.Bn[2] = Bx[a][b + 1][d];
          q.Bn[3] = Bx[a][b - 1][d]; q.Bn[4] = Bx[a][b][d + 1]; q.Bn[5] = Bx[a][b][d - 1];
          q.wn[0] = Wx[a + 1][b][d]; q.wn[1] = Wx[a - 1][b][d]; q.wn[2] = Wx[a][b + 1][d];
          q.wn[3] = Wx[a][b - 1][d]; q.wn[4] = Wx[a][b][d + 1]; q.wn[5] = Wx[a][b][d - 1];
        }
        if constexpr (kAux) {
          q.a = Ax[a][b][d];
          q.an[0] = Ax[a + 1][b][d]; q.an[1] = Ax[a - 1][b][d]; q.an[2] = Ax[a][b + 1][d];
          q.an[3] = Ax[a][b - 1][d]; q.an[4] = Ax[a][b][d + 1]; q.an[5] = Ax[a][b][d - 1];
        }
        T Fv, dF;
        eval_cell<M, FM, T>(c, F.ih2, q, Fv, dF);
        xs += q.x;
        rs -= Fv;  // r = Sigma - L(x)
      }
  }
  (void)Bx;
  (void)Wx;
  (void)Ax;
  const T xr = xs * T(0.125);
  xc[to] = xr;
  x0c[to] = xr;
  sigc[to] = rs * T(0.125);
  if constexpr (M == FOFR && kExpCache<T>) C.aux[to] = aux_of<M, FM, T>(xr, T(0));
}

// resid_restrict for FP32 red/black grids of the canonical models (Poisson, symmetron), two coarse cells
// (K, K+1; K even) per thread: each fine row of the 16 children's stencils, k = 2K-1 .. 2K+4, comes in as one
// float2 per colour half (k = 2K, 2K+2 and k = 2K+1, 2K+3) and two scalars, and the per-cell arrays of the
// children as float2 likewise.  Coarse side >= 4.
template <Model M, Form FM>
__global__ void __launch_bounds__(256) resid_restrict2(LevelView<float> F, CoefT<float> c, LevelView<float> C,
                                                       float* __restrict__ x0c, float* __restrict__ sigc) {
  static_assert(M != FOFR, "the f(R) operators keep the one-cell kernel");
  const int lg = F.lg, lgc = lg - 1, m = F.N - 1;
  const unsigned hN = (unsigned)F.N >> 1, half = 1u << (3 * lg - 1);
  const unsigned long long npairs = 1ull << (3 * lgc - 1);
  const unsigned t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= npairs) return;
  const int mc = (1 << lgc) - 1;
  const int K = (int)((t << 1) & mc), J = (int)((t >> (lgc - 1)) & mc), I = (int)(t >> (2 * lgc - 1));
  // X[a][b][d]: fine (2I-1+a, 2J-1+b, 2K-1+d); corner rows (a, b both in {0, 3}) unused
  float X[4][4][6];
  auto row = [&](int a, int b, bool halo) {
    const int fi = (2 * I - 1 + a) & m, fj = (2 * J - 1 + b) & m;
    const unsigned rb = (((unsigned)fi << lg) | (unsigned)fj) * hN;
    const unsigned c0 = ((unsigned)(fi + fj) & 1u) ? half : 0u, c1 = c0 ? 0u : half;
    const float2 v0 = *reinterpret_cast<const float2*>(F.x + c0 + rb + (unsigned)K);  // k = 2K, 2K+2
    const float2 v1 = *reinterpret_cast<const float2*>(F.x + c1 + rb + (unsigned)K);  // k = 2K+1, 2K+3
    X[a][b][1] = v0.x;
    X[a][b][2] = v1.x;
    X[a][b][3] = v0.y;
    X[a][b][4] = v1.y;
    if (halo) {
      X[a][b][0] = F.x[c1 + rb + (((unsigned)K - 1u) & (hN - 1u))];  // k = 2K-1
      X[a][b][5] = F.x[c0 + rb + (((unsigned)K + 2u) & (hN - 1u))];  // k = 2K+4
    }
  };
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      const bool ea = (a == 0 || a == 3), eb = (b == 0 || b == 3);
      if (ea && eb) continue;
      row(a, b, !(ea || eb));
    }
  // the children's own arrays (a, b in {1, 2}; d = 1..4), same float2 pattern
  float E[2][2][4], S[2][2][4], Bv[2][2][4];
#pragma unroll
  for (int a = 0; a < 2; ++a)
#pragma unroll
    for (int b = 0; b < 2; ++b) {
      const int fi = (2 * I + a) & m, fj = (2 * J + b) & m;
      const unsigned rb = (((unsigned)fi << lg) | (unsigned)fj) * hN;
      const unsigned c0 = ((unsigned)(fi + fj) & 1u) ? half : 0u, c1 = c0 ? 0u : half;
      auto get4 = [&](const float* __restrict__ arr, float* out) {
        const float2 v0 = *reinterpret_cast<const float2*>(arr + c0 + rb + (unsigned)K);
        const float2 v1 = *reinterpret_cast<const float2*>(arr + c1 + rb + (unsigned)K);
        out[0] = v0.x;
        out[1] = v1.x;
        out[2] = v0.y;
        out[3] = v1.y;
      };
      if (F.sig) get4(F.sig, S[a][b]);
      else S[a][b][0] = S[a][b][1] = S[a][b][2] = S[a][b][3] = 0.f;
      if constexpr (uses_eta<M, FM>()) get4(F.eta, E[a][b]);
      if constexpr (FM == DELTA && M != POI) get4(F.B, Bv[a][b]);
    }
  float xs[2] = {0.f, 0.f}, rs[2] = {0.f, 0.f};
#pragma unroll
  for (int a = 1; a < 3; ++a)
#pragma unroll
    for (int b = 1; b < 3; ++b)
#pragma unroll
      for (int d = 1; d < 5; ++d) {
        Cell<float> q;
        q.x = X[a][b][d];
        q.xn[0] = X[a + 1][b][d];
        q.xn[1] = X[a - 1][b][d];
        q.xn[2] = X[a][b + 1][d];
        q.xn[3] = X[a][b - 1][d];
        q.xn[4] = X[a][b][d + 1];
        q.xn[5] = X[a][b][d - 1];
        q.sig = S[a - 1][b - 1][d - 1];
        if constexpr (uses_eta<M, FM>()) q.eta = E[a - 1][b - 1][d - 1]; else q.eta = 0.f;
        if constexpr (FM == DELTA && M != POI) q.B = Bv[a - 1][b - 1][d - 1]; else q.B = 0.f;
        float Fv, dF;
        eval_cell<M, FM, float>(c, F.ih2, q, Fv, dF);
        const int s = (d - 1) >> 1;  // children of K (d = 1, 2) or of K+1 (d = 3, 4)
        xs[s] += q.x;
        rs[s] -= Fv;
      }
  (void)E;
  (void)Bv;
#pragma unroll
  for (int s = 0; s < 2; ++s) {
    const size_t to = lidx<float>(lgc, I, J, K + s);
    const float xr = xs[s] * 0.125f;
    C.x[to] = xr;
    x0c[to] = xr;
    sigc[to] = rs[s] * 0.125f;
  }
}

// Sigma_H += L_H(x_H) on a red/black FP32 level (the FAS coarse source, Sect. 3.2): two cells per thread through
// the smoother's gather and evaluation (threads [0, N^3/4) red, then black; N >= 4).  sig is the level's own
// Sigma array, read and written here only.
template <Model M, Form FM>
__global__ void __launch_bounds__(256) sigma_rb2(LevelView<float> L, CoefT<float> c, float* __restrict__ sig) {
  const unsigned q4 = 1u << (3 * L.lg - 2);
  unsigned t = blockIdx.x * blockDim.x + threadIdx.x;
  const unsigned lanes = __ballot_sync(0xffffffffu, t < 2 * q4);  // blocks of whole warps
  if (t >= 2 * q4) return;
  const int color = t >= q4 ? 1 : 0;
  t -= color ? q4 : 0u;
  L.sig = nullptr;  // L(x) itself
  Cell<float> q0, q1;
  float2 F, dF;
  const unsigned o = rb2_eval<M, FM>(L, c, color, t, lanes, q0, q1, F, dF);
  float2* sp = reinterpret_cast<float2*>(sig + o);
  const float2 v = *sp;
  *sp = make_float2(v.x + F.x, v.y + F.y);
}

// Sigma_H += L_H(x_H) (the FAS coarse source, Sect. 3.2).
template <Model M, Form FM, class T>
__global__ void coarse_sigma_add(LevelView<T> L, CoefT<T> c, T* __restrict__ sig) {
  size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= ((size_t)1 << (3 * L.lg))) return;
  LevelView<T> L0 = L;
  L0.sig = nullptr;
  Cell<T> q = gather_at<M, FM, T>(L0, t);
  T F, dF;
  eval_cell<M, FM, T>(c, L.ih2, q, F, dF);
  sig[t] += F;
}

// x_h += P(x_H - x0_H): one thread per coarse cell (I,J,K) writes its 8
// children.  P is cell-centred trilinear, applied one axis at a time: the
// child at offset 0 (1) along an axis takes 3/4 of the coarse value and 1/4
// of the coarse neighbour below (above).  f(R): the cached exponential of
// each child follows its new value.
template <Model M, Form FM, class T>
__global__ void prolong_correct(LevelView<T> Fv, const T* __restrict__ xc, const T* __restrict__ x0c, int lgc) {
  T* __restrict__ xf = Fv.x;
  const int lgf = lgc + 1, mc = (1 << lgc) - 1;
  size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= ((size_t)1 << (3 * lgc))) return;
  // threads in row-major coarse order: the 8 children of neighbouring threads are contiguous
  const int K = (int)(t & mc), J = (int)((t >> lgc) & mc), I = (int)(t >> (2 * lgc));
  T D[3][3][3];
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int b = 0; b < 3; ++b)
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        const size_t q = lidx<T>(lgc, (I + a - 1) & mc, (J + b - 1) & mc, (K + d - 1) & mc);
        D[a][b][d] = xc[q] - x0c[q];
      }
  const T w3 = T(0.75), w1 = T(0.25);
  T Tk[3][3][2], Tj[3][2][2];
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int b = 0; b < 3; ++b) {
      Tk[a][b][0] = w3 * D[a][b][1] + w1 * D[a][b][0];
      Tk[a][b][1] = w3 * D[a][b][1] + w1 * D[a][b][2];
    }
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int d = 0; d < 2; ++d) {
      Tj[a][0][d] = w3 * Tk[a][1][d] + w1 * Tk[a][0][d];
      Tj[a][1][d] = w3 * Tk[a][1][d] + w1 * Tk[a][2][d];
    }
#pragma unroll
  for (int ca = 0; ca < 2; ++ca)
#pragma unroll
    for (int cb = 0; cb < 2; ++cb)
#pragma unroll
      for (int cd = 0; cd < 2; ++cd) {
        const T v = w3 * Tj[1][cb][cd] + w1 * Tj[ca ? 2 : 0][cb][cd];
        const size_t o = lidx<T>(lgf, 2 * I + ca, 2 * J + cb, 2 * K + cd);
        const T xn = xf[o] + v;
        xf[o] = xn;
        if constexpr (M == FOFR && kExpCache<T>) Fv.aux[o] = aux_of<M, FM, T>(xn, T(0));
      }
}

// The same correction for FP32 red/black grids with at least 32 coarse cells per side, tiled: a block of
// 2 x 4 x 32 coarse cells first stages the coarse correction D = xc - x0c of its tile and a one-cell halo
// (4 x 6 x 34 values) in shared memory, so each D is read from global memory once per block instead of by
// 27 threads, and each thread then updates the 8 children of its coarse cell (consecutive threads write
// consecutive places of one colour half).
constexpr int kPTI = 2, kPTJ = 4, kPTK = 32;
template <Model M, Form FM>
__global__ void __launch_bounds__(kPTI * kPTJ * kPTK) prolong_tiled(LevelView<float> Fv, const float* __restrict__ xc,
                                                                   const float* __restrict__ x0c, int lgc) {
  __shared__ float D[kPTI + 2][kPTJ + 2][kPTK + 2];
  float* __restrict__ xf = Fv.x;
  const int Nc = 1 << lgc, mc = Nc - 1, lgf = lgc + 1;
  const int tk_blocks = Nc / kPTK, tj_blocks = Nc / kPTJ;
  const int b = blockIdx.x;
  const int K0 = (b % tk_blocks) * kPTK, J0 = ((b / tk_blocks) % tj_blocks) * kPTJ,
            I0 = (b / (tk_blocks * tj_blocks)) * kPTI;
  constexpr int kHalo = (kPTI + 2) * (kPTJ + 2) * (kPTK + 2);
  for (int e = threadIdx.x; e < kHalo; e += blockDim.x) {
    const int d = e % (kPTK + 2), r = e / (kPTK + 2), bb = r % (kPTJ + 2), a = r / (kPTJ + 2);
    const size_t q = lidx<float>(lgc, (I0 + a - 1) & mc, (J0 + bb - 1) & mc, (K0 + d - 1) & mc);
    D[a][bb][d] = xc[q] - x0c[q];
  }
  __syncthreads();
  const int tk = threadIdx.x % kPTK, tj = (threadIdx.x / kPTK) % kPTJ, ti = threadIdx.x / (kPTK * kPTJ);
  const float w3 = 0.75f, w1 = 0.25f;
  float Tk[3][3][2], Tj[3][2][2];
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int bb = 0; bb < 3; ++bb) {
      const float c0 = D[ti + a][tj + bb][tk], c1 = D[ti + a][tj + bb][tk + 1], c2 = D[ti + a][tj + bb][tk + 2];
      Tk[a][bb][0] = w3 * c1 + w1 * c0;
      Tk[a][bb][1] = w3 * c1 + w1 * c2;
    }
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int d = 0; d < 2; ++d) {
      Tj[a][0][d] = w3 * Tk[a][1][d] + w1 * Tk[a][0][d];
      Tj[a][1][d] = w3 * Tk[a][1][d] + w1 * Tk[a][2][d];
    }
  const int I = I0 + ti, J = J0 + tj, K = K0 + tk;
#pragma unroll
  for (int ca = 0; ca < 2; ++ca)
#pragma unroll
    for (int cb = 0; cb < 2; ++cb)
#pragma unroll
      for (int cd = 0; cd < 2; ++cd) {
        const float v = w3 * Tj[1][cb][cd] + w1 * Tj[ca ? 2 : 0][cb][cd];
        const size_t o = lidx<float>(lgf, 2 * I + ca, 2 * J + cb, 2 * K + cd);
        xf[o] += v;
      }
}

// The tiled prolongation with two coarse cells per thread along k (tile 2 x 4 x 64): the children of cells
// K and K+1 at the same (ca, cb, cd) are neighbours in one colour half, so every fine access is a float2
// and all 8 loads are issued before the 8 stores.
constexpr int kP2K = 64;
template <Model M, Form FM>
__global__ void __launch_bounds__(kPTI * kPTJ * kPTK) prolong_tiled2(LevelView<float> Fv, const float* __restrict__ xc,
                                                                    const float* __restrict__ x0c, int lgc) {
  __shared__ float D[kPTI + 2][kPTJ + 2][kP2K + 2];
  float* __restrict__ xf = Fv.x;
  const int Nc = 1 << lgc, mc = Nc - 1, lgf = lgc + 1;
  const int tk_blocks = Nc / kP2K, tj_blocks = Nc / kPTJ;
  const int b = blockIdx.x;
  const int K0 = (b % tk_blocks) * kP2K, J0 = ((b / tk_blocks) % tj_blocks) * kPTJ,
            I0 = (b / (tk_blocks * tj_blocks)) * kPTI;
  constexpr int kHalo = (kPTI + 2) * (kPTJ + 2) * (kP2K + 2);
  for (int e = threadIdx.x; e < kHalo; e += blockDim.x) {
    const int d = e % (kP2K + 2), r = e / (kP2K + 2), bb = r % (kPTJ + 2), a = r / (kPTJ + 2);
    const size_t q = lidx<float>(lgc, (I0 + a - 1) & mc, (J0 + bb - 1) & mc, (K0 + d - 1) & mc);
    D[a][bb][d] = xc[q] - x0c[q];
  }
  __syncthreads();
  const int tk = threadIdx.x % kPTK, tj = (threadIdx.x / kPTK) % kPTJ, ti = threadIdx.x / (kPTK * kPTJ);
  const float w3 = 0.75f, w1 = 0.25f;
  // values of the 8 children of coarse cell K0 + 2 tk + s (s = 0, 1), index [ca][cb][cd]
  float V[2][2][2][2];
#pragma unroll
  for (int sidx = 0; sidx < 2; ++sidx) {
    const int kk = 2 * tk + sidx;
    float Tk[3][3][2], Tj[3][2][2];
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int bb = 0; bb < 3; ++bb) {
        const float c0 = D[ti + a][tj + bb][kk], c1 = D[ti + a][tj + bb][kk + 1], c2 = D[ti + a][tj + bb][kk + 2];
        Tk[a][bb][0] = w3 * c1 + w1 * c0;
        Tk[a][bb][1] = w3 * c1 + w1 * c2;
      }
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int d = 0; d < 2; ++d) {
        Tj[a][0][d] = w3 * Tk[a][1][d] + w1 * Tk[a][0][d];
        Tj[a][1][d] = w3 * Tk[a][1][d] + w1 * Tk[a][2][d];
      }
#pragma unroll
    for (int ca = 0; ca < 2; ++ca)
#pragma unroll
      for (int cb = 0; cb < 2; ++cb)
#pragma unroll
        for (int cd = 0; cd < 2; ++cd) V[sidx][ca][cb][cd] = w3 * Tj[1][cb][cd] + w1 * Tj[ca ? 2 : 0][cb][cd];
  }
  const int I = I0 + ti, J = J0 + tj, K = K0 + 2 * tk;
  // children (2I+ca, 2J+cb, 2K+cd) and (2I+ca, 2J+cb, 2K+2+cd): places g/2 and g/2 + 1 of one colour half
  size_t o[2][2][2];
  float2 xv[2][2][2];
#pragma unroll
  for (int ca = 0; ca < 2; ++ca)
#pragma unroll
    for (int cb = 0; cb < 2; ++cb)
#pragma unroll
      for (int cd = 0; cd < 2; ++cd) {
        o[ca][cb][cd] = lidx<float>(lgf, 2 * I + ca, 2 * J + cb, 2 * K + cd);
        xv[ca][cb][cd] = *reinterpret_cast<const float2*>(xf + o[ca][cb][cd]);
      }
#pragma unroll
  for (int ca = 0; ca < 2; ++ca)
#pragma unroll
    for (int cb = 0; cb < 2; ++cb)
#pragma unroll
      for (int cd = 0; cd < 2; ++cd) {
        const float2 v = xv[ca][cb][cd];
        *reinterpret_cast<float2*>(xf + o[ca][cb][cd]) =
            make_float2(v.x + V[0][ca][cb][cd], v.y + V[1][ca][cb][cd]);
      }
}

// coarse = mean of the 8 children of fine (plain restriction of a field).
template <class Tin, class Tout>
__global__ void restrict_mean(const Tin* __restrict__ f, Tout* __restrict__ c, int lgc) {
  size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= ((size_t)1 << (3 * lgc))) return;
  int lgf = lgc + 1, mc = (1 << lgc) - 1;
  const int K = (int)(t & mc), J = (int)((t >> lgc) & mc), I = (int)(t >> (2 * lgc));
  Tin s = 0;
#pragma unroll
  for (int a = 0; a < 2; ++a)
#pragma unroll
    for (int b = 0; b < 2; ++b)
#pragma unroll
      for (int d = 0; d < 2; ++d) s += f[lidx<Tin>(lgf, 2 * I + a, 2 * J + b, 2 * K + d)];
  c[lidx<Tout>(lgc, I, J, K)] = (Tout)(s * Tin(0.125));
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
__global__ void __launch_bounds__(kNormThreads) norm_partial(LevelView<T> L, CoefT<T> c, double* __restrict__ part) {
  size_t n = (size_t)1 << (3 * L.lg);
  double acc = 0.0;
  for (size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (size_t)gridDim.x * blockDim.x) {
    Cell<T> q = gather_at<M, FM, T>(L, t);
    T F, dF;
    eval_cell<M, FM, T>(c, L.ih2, q, F, dF);
    acc += (double)F * (double)F;
  }
  block_sum_store<T>(acc, part);
}

// Block partial sums of (L(x) - Sigma)^2 over a red/black FP32 grid, two cells per thread
// and iteration (the smoother's gather), a grid-stride loop over the pairs of both colours
// with a fixed assignment: reproducible.
template <Model M, Form FM>
__global__ void __launch_bounds__(kNormThreads) norm_rb2(LevelView<float> L, CoefT<float> c, double* __restrict__ part) {
  const unsigned q4 = 1u << (3 * L.lg - 2);
  float acc = 0.f;
  // the loop runs while any lane of the warp has a pair (warp-uniform trip count, blocks of whole warps)
  for (unsigned tt = blockIdx.x * blockDim.x + threadIdx.x; __any_sync(0xffffffffu, tt < 2 * q4);
       tt += gridDim.x * blockDim.x) {
    const unsigned lanes = __ballot_sync(0xffffffffu, tt < 2 * q4);
    if (tt < 2 * q4) {
      const int color = tt >= q4 ? 1 : 0;
      Cell<float> q0, q1;
      float2 F, dF;
      rb2_eval<M, FM>(L, c, color, tt - (color ? q4 : 0u), lanes, q0, q1, F, dF);
      acc = fmaf(F.x, F.x, fmaf(F.y, F.y, acc));
    }
  }
  block_sum_store<double>((double)acc, part);
}


// Sum of (v - shift)^2 and of v over an array (for the reference residual
// and the Poisson mean).
template <class T, bool kFast = false>
__global__ void __launch_bounds__(kNormThreads) moments_partial(const T* __restrict__ v, size_t n, double shift,
                                                                double* __restrict__ part2,
                                                                double* __restrict__ part1) {
  double a2 = 0.0, a1 = 0.0;
  if constexpr (sizeof(T) == 8 && kFast) {
    // FP64 fields without the FP64 units (the mixed-precision solves): the sum in float-float (Poisson needs
    // the mean to ~1e-14), the square sum (a scale for the tolerance) in FP32 per thread
    ff s1 = {0.f, 0.f};
    float s2 = 0.f;
    const float sh = (float)shift;  // 0 or 1: exact
    for (size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (size_t)gridDim.x * blockDim.x) {
      const ff x = ff_split_bits((double)v[t]);
      s1 = ff_add(s1, x);
      const float d = ff_add_f(x, -sh).hi;
      s2 = fmaf(d, d, s2);
    }
    a1 = (double)s1.hi + (double)s1.lo;
    a2 = (double)s2;
  } else {
    for (size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (size_t)gridDim.x * blockDim.x) {
      double d = (double)v[t] - shift;
      a2 += d * d;
      a1 += (double)v[t];
    }
  }
  block_sum_store<T>(a2, part2);
  __syncthreads();
  block_sum_store<T>(a1, part1);
}

// moments_partial<double, true> of the density (shift 1) and, in the same pass, its FP32 copy in the
// red/black layout (the value truncated to 24 bits, as to_rb writes it): the density is read once.
__global__ void __launch_bounds__(kNormThreads) moments_to_rb(const double* __restrict__ v, float* __restrict__ rb,
                                                              int lg, double* __restrict__ part2,
                                                              double* __restrict__ part1);
// Sum (float-float per thread) of an FP32 array, block partials: the Poisson mean of the FP32 grids.
__global__ void __launch_bounds__(kNormThreads) sum_f32_partial(const float* __restrict__ v, size_t n,
                                                                double* __restrict__ part);

// One block sums nparts partials in a fixed order into *out.
__global__ void reduce_final(const double* __restrict__ part, int nparts, double* __restrict__ out);
// Scalars and flags for the host, written by a kernel into mapped pinned memory (hd, hi: its device
// addresses): the per-cycle readback of the solvers uses no copy engine, so it never queues behind the
// caller's bulk host<->device copies on other streams.
__global__ void publish_scalars(const double* __restrict__ scal, int ns, const int* __restrict__ iflags, int ni,
                                double* hd, int* hi);

}  // namespace isis
