// isis_fofr_staged.cuh -- the f(R) Newton-Gauss-Seidel half-sweep (Sect. 3.4, Eqs. (disc_non_canonical) and
// (dbeq); Sect. 4.2) on FP32 red/black grids of side N >= 128, with the per-cell exponentials of the other
// colour staged in shared memory.
//
// Every cell of the other colour is a neighbour of six cells of the colour being updated.  The flux form needs
// per neighbour its e^u (field form), or e^B and e^B expm1(e) (correction form about the base B).  Evaluated
// where they are used, as in smooth_rb2, they cost seven exponentials per updated cell; here a block streams
// along i over a slab of TJ rows in j (full rows in k), computes the other colour's per-cell values once per
// plane (with one halo row on either side in j) into a ring of three planes in shared memory, and updates its
// own cells of plane i from planes i-1, i, i+1 of the ring.  The arithmetic of the update is that of
// fofr_field_eval / fofr_delta_eval (isis_model.cuh); the exponentials are the hardware base-2 exponential of
// the packed kernels.
#pragma once
#include "isis_kernels.cuh"

namespace isis {

constexpr int kSTThreads = 256;
constexpr int kSTRows = 4;     // TJ: rows in j updated by a block
constexpr int kSTChunk = 32;   // planes in i streamed by a block

// e^v through ex2 (the exponential of the packed f(R) kernels)
__device__ __forceinline__ float st_exp(float v) { return ex2_approx(v * 1.4426950408889634f); }

// Per-cell values of the other colour: field form (x, b = e^x); correction form (e, B, m = e^B expm1(e),
// bt = e^B + m).
template <Form FM>
struct StagedVal;
template <>
struct StagedVal<FIELD> { using T = float2; };
template <>
struct StagedVal<DELTA> { using T = float4; };

template <Form FM>
__device__ __forceinline__ typename StagedVal<FM>::T st_values(float x, float B) {
  if constexpr (FM == FIELD) {
    (void)B;
    return make_float2(x, st_exp(x));
  } else {
    const float w = st_exp(B), m = w * dexpm1<float>(x);
    return make_float4(x, B, m, w + m);
  }
}

// Shared memory of one block: 3 planes x (TJ + 2) rows x N/2 places.
template <Form FM>
inline size_t staged_smem_bytes(int N) {
  return 3 * (size_t)(kSTRows + 2) * (size_t)(N / 2) * sizeof(typename StagedVal<FM>::T);
}

// Blocks: (N / TJ) slabs in j times (N / kSTChunk) chunks in i; N = 2^LG >= 128.
// kResid: instead of updating x, write the residual r = Sigma - L(x) of the colour's cells into res (same
// layout as x); two launches (colour 0, 1) give the residual of the grid.
// The global loads of plane i + 2 (to be staged) and of the own cells of plane i + 1 are issued into registers
// before plane i is updated, so their latency overlaps the update and the block barriers.
template <Form FM, bool kResid, int LG>
__global__ void __launch_bounds__(kSTThreads) fofr_smooth_staged(LevelView<float> L, Coef c, int color,
                                                                 float* __restrict__ res) {
  using V = typename StagedVal<FM>::T;
  constexpr unsigned N = 1u << LG, m = N - 1, hN = N >> 1, half = 1u << (3 * LG - 1);
  constexpr unsigned kR = kSTRows + 2;        // staged rows: j0 - 1 .. j0 + TJ
  constexpr unsigned plane_vals = kR * hN;    // values per staged plane
  constexpr unsigned kFill = (plane_vals + kSTThreads - 1) / kSTThreads;  // staged values per thread
  constexpr unsigned kOwn = kSTRows * hN / kSTThreads;                    // own cells per thread and plane
  static_assert(kSTRows * hN % kSTThreads == 0, "own cells must divide evenly among the threads");
  extern __shared__ float4 st_dyn[];
  V* ring = reinterpret_cast<V*>(st_dyn);
  const unsigned own = color ? half : 0u, oth = color ? 0u : half;
  constexpr unsigned nslab = N / kSTRows;
  const unsigned j0 = (blockIdx.x % nslab) * kSTRows, i0 = (blockIdx.x / nslab) * kSTChunk;

  // raw values (x, B) of the other colour's staged rows of plane p
  float rx[kFill], rB[kFill];
  auto load_raw = [&](unsigned p) {
#pragma unroll
    for (unsigned u = 0; u < kFill; ++u) {
      const unsigned t = threadIdx.x + u * kSTThreads;
      if (t < plane_vals) {
        const unsigned r = t / hN, k2 = t - r * hN, jj = (j0 + r - 1) & m;
        const unsigned g = oth + ((((p & m) << LG) | jj) << (LG - 1)) + k2;
        rx[u] = L.x[g];
        rB[u] = (FM == DELTA) ? L.B[g] : 0.f;
      }
    }
  };
  auto store_raw = [&](unsigned s) {
    V* dst = ring + s * plane_vals;
#pragma unroll
    for (unsigned u = 0; u < kFill; ++u) {
      const unsigned t = threadIdx.x + u * kSTThreads;
      if (t < plane_vals) dst[t] = st_values<FM>(rx[u], rB[u]);
    }
  };
  // the own cells of plane i: x, Sigma and eta (field form) or B (correction form)
  float ox[kOwn], osig[kOwn], oe[kOwn];
  auto load_own = [&](unsigned i) {
#pragma unroll
    for (unsigned u = 0; u < kOwn; ++u) {
      const unsigned t = threadIdx.x + u * kSTThreads, r = t / hN, k2 = t - r * hN, j = j0 + r;
      const unsigned o = own + (((i << LG) | j) << (LG - 1)) + k2;
      ox[u] = L.x[o];
      osig[u] = L.sig ? L.sig[o] : 0.f;
      oe[u] = (FM == FIELD) ? L.eta[o] : L.B[o];
    }
  };

  const float ih2 = L.ih2;
  load_raw(i0 - 1);
  store_raw(0);
  load_raw(i0);
  store_raw(1);
  load_raw(i0 + 1);
  load_own(i0);
  for (unsigned q = 1; q <= kSTChunk; ++q) {
    const unsigned i = i0 + q - 1;
    store_raw((q + 1) % 3);  // plane i + 1
    float cx[kOwn], csig[kOwn], ce[kOwn];
#pragma unroll
    for (unsigned u = 0; u < kOwn; ++u) { cx[u] = ox[u]; csig[u] = osig[u]; ce[u] = oe[u]; }
    if (q < kSTChunk) {
      load_raw(i + 2);
      load_own(i + 1);
    }
    __syncthreads();
    const V* pm = ring + ((q + 2) % 3) * plane_vals;  // plane i - 1
    const V* pc = ring + (q % 3) * plane_vals;        // plane i
    const V* pp = ring + ((q + 1) % 3) * plane_vals;  // plane i + 1
#pragma unroll
    for (unsigned u = 0; u < kOwn; ++u) {
      const unsigned t = threadIdx.x + u * kSTThreads, r = t / hN, k2 = t - r * hN, j = j0 + r;
      const unsigned par = (i + j + (unsigned)color) & 1u;
      const unsigned o = own + (((i << LG) | j) << (LG - 1)) + k2;
      const unsigned rc = (r + 1) * hN;  // the own row in the staged planes
      const V nb[6] = {pp[rc + k2], pm[rc + k2], pc[rc + hN + k2], pc[rc - hN + k2],
                       pc[rc + ((k2 + par) & (hN - 1))], pc[rc + ((k2 + par - 1) & (hN - 1))]};
      const float x = cx[u], sig = csig[u];
      float F, dF;
      if constexpr (FM == FIELD) {
        const float ex = st_exp(x);
        float sdu = 0.f, sexdu = 0.f, sex = 0.f;
#pragma unroll
        for (int d = 0; d < 6; ++d) {
          const float du = nb[d].x - x;
          sdu += du;
          sexdu = fmaf(nb[d].y, du, sexdu);
          sex += nb[d].y;
        }
        // flux = (1/2)[e^x sum du + sum e^x_nb du], dsum = (1/2) e^x sum du - (6 e^x + sum e^x_nb)/2 (fscale e^x = b)
        const float fs = (float)c.fscale;
        const float flux = fs * 0.5f * fmaf(ex, sdu, sexdu);
        const float dsum = fs * 0.5f * (fmaf(ex, sdu, -6.0f * ex) - sex);
        const float inp1 = (float)c.inv_np1, Kx = (float)c.fKx;
        const float em = dexpm1<float>(-x * inp1);
        const float S = (float)c.K1 * (ce[u] - 1.0f) - Kx * em + (float)c.fK3x;
        F = flux * ih2 - S - sig;
        dF = dsum * ih2 - Kx * inp1 * (em + 1.0f);
      } else {
        const float B = ce[u];
        const float w = st_exp(B), mm = w * dexpm1<float>(x), bt = w + mm;
        float sdB = 0.f, sde = 0.f, smn = 0.f, sbn = 0.f, sbt = 0.f;
#pragma unroll
        for (int d = 0; d < 6; ++d) {
          const float dB = nb[d].y - B, de = nb[d].x - x;
          sdB += dB;
          sde += de;
          smn = fmaf(nb[d].z, dB, smn);
          sbn = fmaf(nb[d].w, de, sbn);
          sbt += nb[d].w;
        }
        // flux = (1/2)[m sum dB + bt sum de + sum m_nb dB + sum bt_nb de]
        // dsum = (1/2) bt (sum dB + sum de) - (6 bt + sum bt_nb)/2
        const float flux = 0.5f * (fmaf(mm, sdB, bt * sde) + (smn + sbn));
        const float dsum = 0.5f * bt * (sdB + sde) - 0.5f * fmaf(6.0f, bt, sbt);
        const float inp1 = (float)c.inv_np1, K2 = (float)c.K2;
        const float exB = st_exp(-B * inp1), em = dexpm1<float>(-x * inp1);
        F = fmaf(flux, ih2, K2 * exB * em) - sig;
        dF = dsum * ih2 - K2 * inp1 * exB * (em + 1.0f);
      }
      if constexpr (kResid) res[o] = -F;  // Sigma is inside F
      else L.x[o] = x - __fdividef(F, dF);
    }
    __syncthreads();
  }
}

// Launch one colour on grids of side 128 .. 1024.
template <Form FM, bool kResid>
inline cudaError_t launch_fofr_staged(const LevelView<float>& L, const Coef& c, int color, float* res,
                                      cudaStream_t st) {
  const unsigned blocks = (unsigned)((L.N / kSTRows) * (L.N / kSTChunk));
  const size_t smem = staged_smem_bytes<FM>(L.N);
  switch (L.lg) {
    case 7: fofr_smooth_staged<FM, kResid, 7><<<blocks, kSTThreads, smem, st>>>(L, c, color, res); break;
    case 8: fofr_smooth_staged<FM, kResid, 8><<<blocks, kSTThreads, smem, st>>>(L, c, color, res); break;
    case 9: fofr_smooth_staged<FM, kResid, 9><<<blocks, kSTThreads, smem, st>>>(L, c, color, res); break;
    case 10: fofr_smooth_staged<FM, kResid, 10><<<blocks, kSTThreads, smem, st>>>(L, c, color, res); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

// Allow each instantiation its largest shared memory (called once per device).
template <Form FM, bool kResid>
inline cudaError_t allow_fofr_staged_smem() {
  cudaError_t e = cudaSuccess;
  auto set = [&](auto kern, int lg) {
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)staged_smem_bytes<FM>(1 << lg));
  };
  set(fofr_smooth_staged<FM, kResid, 7>, 7);
  set(fofr_smooth_staged<FM, kResid, 8>, 8);
  set(fofr_smooth_staged<FM, kResid, 9>, 9);
  set(fofr_smooth_staged<FM, kResid, 10>, 10);
  return e;
}

}  // namespace isis
