// isis_stream.cuh -- temporally blocked red-black Newton-Gauss-Seidel
// smoother (Sect. 3.2) for FP32 grids: NSW full sweeps (2 NSW colour
// half-sweeps) in one pass over HBM.
//
// Layout of the work
//   - A CTA owns a (j, k) tile of TJ x 64 cells including a halo of
//     H = 2 NSW cells on each side, and streams along i through TI planes
//     (plus H halo planes below and above).  Each half-sweep invalidates one
//     more layer of the halo, so after 2 NSW half-sweeps exactly the interior
//     (TJ - 2H) x (64 - 2H) x TI cells hold the result of NSW sequential
//     red-black sweeps; only those are stored.
//   - A thread owns a pair of cells (k = 2 lane, 2 lane + 1) in one j row:
//     one red and one black cell per plane, so every thread updates one cell
//     per half-sweep.  Red = (i + j + k) even, updated first.
//   - Half-sweep s (colour s mod 2) runs on plane q - 1 - s when plane q
//     arrives.  The i-neighbours of a thread's cell are in its own register
//     ring of planes; the k-neighbours are its other cell or a warp shuffle;
//     the j-neighbours come from a shared-memory ring of planes.  A half-sweep
//     only reads, in shared memory, cells of the other colour written in the
//     previous plane step, so one barrier per plane orders everything.
//   - Input and output are different buffers (the halo reads of one CTA must
//     see the old values that a neighbouring CTA is overwriting).
#pragma once
#include <type_traits>

#include "isis_kernels.cuh"

namespace isis {

// What a neighbour needs to know about a cell.
template <Model M, Form FM>
struct SState {
  float x;
};
template <>
struct SState<FOFR, FIELD> {
  float x, b;  // b = e^x
};
template <>
struct SState<FOFR, DELTA> {
  float x, B, m, bt;  // correction e, base B, m = e^B expm1(e), bt = e^(B+e)
};

template <Model M, Form FM, int NSW>
struct StreamCfg {
  // rows per CTA including the halo: as many as the register file allows
  static constexpr int TJ = (M == FOFR && FM == DELTA) ? 16 : (NSW == 1 ? 32 : 24);
};

template <Model M, Form FM>
__device__ __forceinline__ SState<M, FM> make_state(float x, float B, float w) {
  SState<M, FM> s;
  s.x = x;
  if constexpr (M == FOFR && FM == FIELD) s.b = __expf(x);
  if constexpr (M == FOFR && FM == DELTA) {
    s.B = B;
    s.m = w * expm1f(x);
    s.bt = w + s.m;
  }
  (void)B;
  (void)w;
  return s;
}

template <Model M, Form FM>
__device__ __forceinline__ float own_B(const SState<M, FM>& s) {
  if constexpr (M == FOFR && FM == DELTA) return s.B;
  (void)s;
  return 0.f;
}

template <Model M, Form FM>
__device__ __forceinline__ float stream_update(const Coef& c, float ih2, const SState<M, FM>& o,
                                               const SState<M, FM>* nb, float eta, float sig, float B, float w) {
  float F, dF;
  if constexpr (M == FOFR && FM == FIELD) {
    float xn[6], bn[6];
#pragma unroll
    for (int d = 0; d < 6; ++d) { xn[d] = nb[d].x; bn[d] = nb[d].b; }
    fofr_field_eval<float>(c, ih2, o.x, o.b, xn, bn, eta, sig, F, dF);
  } else if constexpr (M == FOFR && FM == DELTA) {
    float en[6], Bn[6], mn[6], btn[6];
#pragma unroll
    for (int d = 0; d < 6; ++d) { en[d] = nb[d].x; Bn[d] = nb[d].B; mn[d] = nb[d].m; btn[d] = nb[d].bt; }
    fofr_delta_eval<float>(c, ih2, o.x, o.B, o.m, o.bt, en, Bn, mn, btn, sig, F, dF);
    (void)w;
  } else {
    Cell<float> q;
    q.x = o.x;
#pragma unroll
    for (int d = 0; d < 6; ++d) q.xn[d] = nb[d].x;
    q.eta = eta;
    q.sig = sig;
    q.B = B;
    eval_cell<M, FM, float>(c, ih2, q, F, dF);
    (void)w;
  }
  // the FP32 cycles only drive the correction; a 2-ulp quotient changes the
  // Newton step by far less than its own error
  return o.x - __fdividef(F, dF);
}

template <Model M, Form FM>
__device__ __forceinline__ SState<M, FM> shfl_up1(const SState<M, FM>& v) {
  SState<M, FM> r;
  const float* a = reinterpret_cast<const float*>(&v);
  float* b = reinterpret_cast<float*>(&r);
#pragma unroll
  for (int t = 0; t < (int)(sizeof(v) / 4); ++t) b[t] = __shfl_up_sync(0xffffffffu, a[t], 1);
  return r;
}
template <Model M, Form FM>
__device__ __forceinline__ SState<M, FM> shfl_down1(const SState<M, FM>& v) {
  SState<M, FM> r;
  const float* a = reinterpret_cast<const float*>(&v);
  float* b = reinterpret_cast<float*>(&r);
#pragma unroll
  for (int t = 0; t < (int)(sizeof(v) / 4); ++t) b[t] = __shfl_down_sync(0xffffffffu, a[t], 1);
  return r;
}

// Per-cell read-only inputs staged in shared memory with each plane.
template <Model M, Form FM>
struct SUse {
  static constexpr bool eta = (FM == FIELD) || (M == SYM);  // f(R) and Poisson corrections need no eta
  static constexpr bool B = (FM == DELTA && M == SYM);      // f(R) keeps B in its state
  static constexpr bool w = (FM == DELTA && M == FOFR);
  static constexpr int nd = 1 + (eta ? 1 : 0) + (B ? 1 : 0) + (w ? 1 : 0);  // + Sigma
};

template <Model M, Form FM>
struct PlaneRegs {  // one plane of a thread's pair, as loaded from global memory
  float2 x, eta, sig, B, w;
};

template <Model M, Form FM>
__device__ __forceinline__ void load_plane(PlaneRegs<M, FM>& r, const LevelView<float>& L, size_t off) {
  using U = SUse<M, FM>;
  r.x = *reinterpret_cast<const float2*>(L.x + off);
  if constexpr (U::eta) r.eta = *reinterpret_cast<const float2*>(L.eta + off);
  r.sig = L.sig ? *reinterpret_cast<const float2*>(L.sig + off) : make_float2(0.f, 0.f);
  if constexpr (U::B || (M == FOFR && FM == DELTA)) r.B = *reinterpret_cast<const float2*>(L.B + off);
  if constexpr (U::w) r.w = *reinterpret_cast<const float2*>(L.w + off);
}

// xin: current field (read only); xout: receives the interior after NSW sweeps.
// Grid: (ceil(N / (64 - 2H)), ceil(N / (TJ - 2H)), N / TI); block 32 x TJ threads;
// dynamic shared memory stream_smem<M, FM, NSW>().
template <Model M, Form FM, int NSW>
__global__ void __launch_bounds__(32 * StreamCfg<M, FM, NSW>::TJ) smooth_stream(LevelView<float> L, float* __restrict__ xout,
                                                                          Coef c, int TI) {
  using S = SState<M, FM>;
  using U = SUse<M, FM>;
  constexpr int TJ = StreamCfg<M, FM, NSW>::TJ;
  constexpr int H = 2 * NSW, R = 2 * NSW + 2, TK = 64, KI = TK - 2 * H, JI = TJ - 2 * H;
  constexpr int PL = TJ * TK;  // cells per plane slot
  extern __shared__ __align__(16) unsigned char smraw[];
  S* sm = reinterpret_cast<S*>(smraw);                     // [R][TJ][TK] states
  float* sd = reinterpret_cast<float*>(sm + R * PL);       // [nd][R][TJ][TK] inputs: Sigma, eta, B, w
  float* sdSig = sd;
  float* sdEta = sd + (size_t)R * PL;
  float* sdB = sdEta + (U::eta ? (size_t)R * PL : 0);
  float* sdW = sdB + (U::B ? (size_t)R * PL : 0);

  const int lane = threadIdx.x & 31, wj = threadIdx.x >> 5;
  const int N = L.N, lg = L.lg, msk = N - 1;
  const int kA = (int)blockIdx.x * KI - H + 2 * lane;  // first cell of the pair, unwrapped (even)
  const int jg = (int)blockIdx.y * JI - H + wj;         // unwrapped row
  const int i0 = (int)blockIdx.z * TI;
  const int ilo = i0 - H, ihi = i0 + TI - 1 + H;
  const int kw = kA & msk, jw = jg & msk;
  const bool st_j = (wj >= H) && (wj < TJ - H) && (jg < N);
  const bool st_k0 = (2 * lane >= H) && (2 * lane < TK - H) && (kA < N);
  const bool st_k1 = (2 * lane + 1 >= H) && (2 * lane + 1 < TK - H) && (kA + 1 < N);
  const int jup = wj + 1 < TJ ? wj + 1 : wj, jdn = wj > 0 ? wj - 1 : wj;  // edge rows read themselves (halo)
  const float ih2 = L.ih2;
  auto plane_off = [&](int q) -> size_t { return cidx(lg, q & msk, jw, kw); };

  S ring[R][2];
  // two planes in flight: pre[0] holds even (q - ilo), pre[1] odd
  PlaneRegs<M, FM> pre[2];
  load_plane<M, FM>(pre[0], L, plane_off(ilo));
  load_plane<M, FM>(pre[1], L, plane_off(ilo + 1));

  for (int base = ilo; base <= ihi; base += R) {
#pragma unroll
    for (int u = 0; u < R; ++u) {
      const int q = base + u;
      if (q > ihi) break;  // CTA-uniform
      // plane q arrives: states into the register and shared rings, inputs into shared memory
      {
        const PlaneRegs<M, FM> cur = pre[u & 1];
        if (q + 2 <= ihi) load_plane<M, FM>(pre[u & 1], L, plane_off(q + 2));
        S s0 = make_state<M, FM>(cur.x.x, cur.B.x, cur.w.x), s1 = make_state<M, FM>(cur.x.y, cur.B.y, cur.w.y);
        ring[u][0] = s0;
        ring[u][1] = s1;
        const int o = u * PL + wj * TK + 2 * lane;
        sm[o] = s0;
        sm[o + 1] = s1;
        *reinterpret_cast<float2*>(sdSig + o) = cur.sig;
        if constexpr (U::eta) *reinterpret_cast<float2*>(sdEta + o) = cur.eta;
        if constexpr (U::B) *reinterpret_cast<float2*>(sdB + o) = cur.B;
        if constexpr (U::w) *reinterpret_cast<float2*>(sdW + o) = cur.w;
      }
      __syncthreads();
#pragma unroll
      for (int s = 0; s < 2 * NSW; ++s) {
        const int p = q - 1 - s;
        if (p >= ilo + s + 1) {  // CTA-uniform: stage s has valid input at p
          const int sl = (u - 1 - s + 2 * R) % R, slp = (u - s + 2 * R) % R, slm = (u - 2 - s + 2 * R) % R;
          // the cell of the pair with this colour: (p + jg + kk + colour) even; p - base has
          // the parity of u - 1 - s (base and i0 are even), so only the row's parity is run-time
          const int kpar = (s + (u - 1 - s) + ilo) & 1;
          auto stage = [&](auto KK) {
            constexpr int kk = decltype(KK)::value;
            const S own = ring[sl][kk];
            S nb[6];
            nb[0] = ring[slp][kk];
            nb[1] = ring[slm][kk];
            nb[2] = sm[sl * PL + jup * TK + 2 * lane + kk];
            nb[3] = sm[sl * PL + jdn * TK + 2 * lane + kk];
            if constexpr (kk == 0) {
              nb[4] = ring[sl][1];
              nb[5] = shfl_up1<M, FM>(ring[sl][1]);
            } else {
              nb[4] = shfl_down1<M, FM>(ring[sl][0]);
              nb[5] = ring[sl][0];
            }
            const int od = sl * PL + wj * TK + 2 * lane + kk;
            const float sig = sdSig[od];
            const float eta = U::eta ? sdEta[od] : 0.f;
            const float Bc = U::B ? sdB[od] : own_B(own);
            const float wc = U::w ? sdW[od] : 0.f;
            const float xn = stream_update<M, FM>(c, ih2, own, nb, eta, sig, Bc, wc);
            const S ns = make_state<M, FM>(xn, Bc, wc);
            ring[sl][kk] = ns;
            sm[od] = ns;
          };
          if (((kpar + jg) & 1) == 0) stage(std::integral_constant<int, 0>{});
          else stage(std::integral_constant<int, 1>{});
        }
      }
      // plane q - 2 NSW is final
      const int pf = q - 2 * NSW;
      if (pf >= i0 && pf < i0 + TI && st_j) {
        const int sl = (u - 2 * NSW + 2 * R) % R;
        float* o = xout + cidx(lg, pf & msk, jw, kw);
        if (st_k0 && st_k1) *reinterpret_cast<float2*>(o) = make_float2(ring[sl][0].x, ring[sl][1].x);
        else {
          if (st_k0) o[0] = ring[sl][0].x;
          if (st_k1) o[1] = ring[sl][1].x;
        }
      }
    }
  }
}

template <Model M, Form FM, int NSW>
constexpr size_t stream_smem() {
  return (size_t)(2 * NSW + 2) * StreamCfg<M, FM, NSW>::TJ * 64 * (sizeof(SState<M, FM>) + 4 * SUse<M, FM>::nd);
}

}  // namespace isis
