// isis_unet.cu -- kernels of the learned initial guess: a small 3-D U-Net whose
// 3x3x3 periodic convolutions are implicit GEMMs on the 5th-generation tensor
// cores (tcgen05.mma, BF16 operands in shared memory, FP32 accumulators in
// tensor memory), trained by the library's own backward and Adam kernels.
// The paper has no learned part; the net only proposes the initial guess and
// the multigrid solver always finishes the solve.
//
// Tensors: a grid of n = 2^lg cells per side, V = n^3 voxels in row-major
// order, C channels (a multiple of 16), BF16, voxel-major: element [v][c].
// A 3x3x3 convolution with periodic wrap:
//     out[v][o] = b[o] + sum_{t < 27} sum_i X[v + d_t][i] W[t][o][i]
// tap t = (di+1)*9 + (dj+1)*3 + (dk+1), d_t = (di, dj, dk) in {-1, 0, 1}^3.
// X is the channel concatenation of src1 (c1 channels, optionally on the grid
// of half resolution and read by nearest-neighbour upsampling) and src2 (c2
// channels on the output grid).
//
// GEMM view (forward): rows m = 128 consecutive voxels, columns n = output
// channels, k = (tap, input channel) in chunks of 16.  The input-gradient
// uses the same kernel with offsets -d_t and W transposed per tap.  The weight
// gradient is a GEMM with k = voxels and both operands M/N-major.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>

#include "../../include/isis_unet.h"
#include "isis_prof.cuh"

namespace isis {
namespace unet {

typedef __nv_bfloat16 bf16;

__device__ __forceinline__ uint32_t su32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Shared-memory matrix descriptor, no swizzle: lbo = byte stride between core
// matrices along K, sbo = along M/N (a core matrix is 8 rows of 16 bytes).
__device__ __forceinline__ uint64_t sdesc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((addr >> 4) & 0x3FFF) | ((uint64_t)((lbo >> 4) & 0x3FFF) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFF) << 32) | ((uint64_t)1 << 46);
}

// Instruction descriptor of kind::f16 with BF16 A/B and FP32 D.
__device__ __forceinline__ uint32_t idesc_bf16(int M, int N, int a_mn_major, int b_mn_major) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)a_mn_major << 15) | ((uint32_t)b_mn_major << 16) |
         ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void cp16(uint32_t dst, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_zero16(uint32_t dst) {
  asm volatile("st.shared.v4.u32 [%0], {%1, %1, %1, %1};" ::"r"(dst), "r"(0u) : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

__device__ __forceinline__ void mbar_init(uint64_t* bar) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(su32(bar)) : "memory");
}

// Bounded wait for the phase with this parity; false if it gave up.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
  uint32_t done = 0;
  for (int it = 0; it < (1 << 22) && !done; ++it) {
    asm volatile(
        "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(su32(bar)), "r"(parity)
        : "memory");
  }
  return done != 0;
}

__device__ __forceinline__ void mma_bf16(uint32_t tmem, uint64_t ad, uint64_t bd, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
      "l"(ad), "l"(bd), "r"(idesc), "r"(acc)
      : "memory");
}
__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(su32(bar))
               : "memory");
}

// 16 FP32 columns of this warp's 32 TMEM lanes starting at column col.
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* v) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int j = 0; j < 16; ++j) v[j] = __uint_as_float(r[j]);
}

// TMEM allocation (a power of two >= 32 columns) holding n columns; n <= 512.
__host__ __device__ __forceinline__ uint32_t tmem_cols(int n) {
  return n <= 32 ? 32u : (n <= 64 ? 64u : (n <= 128 ? 128u : (n <= 256 ? 256u : 512u)));
}

// voxel index of (i + di, j + dj, k + dk) on a grid of side 2^lg, periodic
__device__ __forceinline__ int shift_vox(int i, int j, int k, int di, int dj, int dk, int lg) {
  const int m = (1 << lg) - 1;
  return ((((i + di) & m) << lg | ((j + dj) & m)) << lg) | ((k + dk) & m);
}

// ---------------------------------------------------------------------------
// Implicit-GEMM convolution: forward (MODE 0) and input gradient (MODE 1)
// ---------------------------------------------------------------------------

struct ConvArgs {
  const bf16* s1;  // c1 channels, grid lg1 (= lg, or lg - 1 read by nearest upsampling)
  const bf16* s2;  // c2 channels, grid lg (nullptr if c2 == 0)
  const bf16* w;   // [27][ncol][c1 + c2]
  const float* bias;
  bf16* out_bf;    // forward: [V][ncol]
  float* out_f;    // input gradient: [V][ncol]
  int c1, lg1, c2, lg, ncol, relu, sgn;  // sgn: +1 forward taps, -1 flipped
  int* err;
};

constexpr int kStages = 4;
constexpr int kKC = 2;  // 16-wide K chunks per pipeline stage

__host__ __device__ constexpr int conv_stage_bytes(int ncol) { return 128 * 32 * kKC + ncol * 32 * kKC; }

template <int MODE>
__global__ void __launch_bounds__(128) igemm_conv(ConvArgs a) {
  extern __shared__ __align__(1024) unsigned char smem[];
  __shared__ __align__(8) uint64_t bars[kStages];
  __shared__ uint32_t tmem_slot;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int lg = a.lg, V = 1 << (3 * lg), m = (1 << lg) - 1;
  const int kin = a.c1 + a.c2, kch = kin / 16, nch = 27 * kch, nst = (nch + kKC - 1) / kKC;
  const int ncol = a.ncol;
  const int stage_bytes = conv_stage_bytes(ncol), a_bytes = 128 * 32 * kKC;
  const uint32_t sbase = su32(smem);
  // this thread's voxel row
  const int v = blockIdx.x * 128 + tid;
  const bool vok = v < V;
  const int vi = v >> (2 * lg), vj = (v >> lg) & m, vk = v & m;

  const uint32_t ncols = tmem_cols(ncol);
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(&tmem_slot)),
                 "r"(ncols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid < kStages) mbar_init(&bars[tid]);
  if (tid == 0) asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_slot;
  const uint32_t idesc = idesc_bf16(128, ncol, 0, 0);
  bool ok = true;

  // K-major canonical stage layout, K = 16 kKC per stage: element (r, kk) at
  // (r/8)*SBO + (kk/8)*128 + (r%8)*16 + (kk%8)*2, SBO = 256 kKC
  const uint32_t SBO = 256u * kKC, LBO = 128u;
  auto load_stage = [&](int st, int s) {
    const uint32_t sa = sbase + st * stage_bytes, sb = sa + a_bytes;
#pragma unroll
    for (int q = 0; q < kKC; ++q) {
      const int ch = s * kKC + q;
      const uint32_t koff = (uint32_t)q * 256u;  // two k-cores per 16-wide chunk
      if (ch >= nch) {
        cp_zero16(sa + (tid / 8) * SBO + koff + (tid % 8) * 16);
        cp_zero16(sa + (tid / 8) * SBO + koff + 128 + (tid % 8) * 16);
        for (int n = tid; n < ncol; n += 128) {
          cp_zero16(sb + (n / 8) * SBO + koff + (n % 8) * 16);
          cp_zero16(sb + (n / 8) * SBO + koff + 128 + (n % 8) * 16);
        }
        continue;
      }
      const int tap = ch / kch, c0 = (ch % kch) * 16;
      const int di = a.sgn * (tap / 9 - 1), dj = a.sgn * ((tap / 3) % 3 - 1), dk = a.sgn * (tap % 3 - 1);
      // A: this thread's voxel row
      const uint32_t da = sa + (tid / 8) * SBO + koff + (tid % 8) * 16;
      if (vok) {
        const bf16* src;
        if (c0 < a.c1) {
          const int u = shift_vox(vi, vj, vk, di, dj, dk, lg);
          int uu = u;
          if (a.lg1 != lg) {  // nearest upsampling from the half-resolution grid
            const int ui = u >> (2 * lg), uj = (u >> lg) & m, uk = u & m;
            uu = (((ui >> 1) << (lg - 1) | (uj >> 1)) << (lg - 1)) | (uk >> 1);
          }
          src = a.s1 + (size_t)uu * a.c1 + c0;
        } else {
          const int u = shift_vox(vi, vj, vk, di, dj, dk, lg);
          src = a.s2 + (size_t)u * a.c2 + (c0 - a.c1);
        }
        cp16(da, src);
        cp16(da + 128, src + 8);
      } else {
        cp_zero16(da);
        cp_zero16(da + 128);
      }
      // B: rows n of W[tap][n][c0 .. c0+15]
      for (int n = tid; n < ncol; n += 128) {
        const bf16* src = a.w + ((size_t)tap * ncol + n) * kin + c0;
        const uint32_t db = sb + (n / 8) * SBO + koff + (n % 8) * 16;
        cp16(db, src);
        cp16(db + 128, src + 8);
      }
    }
  };

  // prologue
#pragma unroll
  for (int s = 0; s < kStages - 1; ++s) {
    if (s < nst) load_stage(s, s);
    cp_commit();
  }
  for (int s = 0; s < nst; ++s) {
    const int sn = s + kStages - 1;
    if (sn < nst) {
      // stage sn % kStages was last read by the MMAs of step sn - kStages
      if (sn >= kStages && ok) ok = mbar_wait(&bars[sn % kStages], ((sn - kStages) / kStages) & 1);
      load_stage(sn % kStages, sn);
    }
    cp_commit();
    cp_wait<kStages - 1>();
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    if (tid == 0 && ok) {
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t sa = sbase + (s % kStages) * stage_bytes, sb = sa + a_bytes;
#pragma unroll
      for (int q = 0; q < kKC; ++q)
        mma_bf16(tmem, sdesc(sa + q * 256, LBO, SBO), sdesc(sb + q * 256, LBO, SBO), idesc,
                 (s > 0 || q > 0) ? 1u : 0u);
      mma_commit(&bars[s % kStages]);
    }
  }
  // all MMAs done: the last commit covers every earlier one
  if (ok) ok = mbar_wait(&bars[(nst - 1) % kStages], ((nst - 1) / kStages) & 1);
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (!ok) {
    if (tid == 0) atomicOr(a.err, 1);
  } else {
    // epilogue: this warp's 32 lanes are voxel rows 32 warp .. 32 warp + 31
    for (int c0 = 0; c0 < ncol; c0 += 16) {
      float acc[16];
      tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, acc);
      if (vok) {
        if (MODE == 0) {
          __align__(16) bf16 o[16];
#pragma unroll
          for (int j = 0; j < 16; ++j) {
            float y = acc[j] + a.bias[c0 + j];
            if (a.relu) y = fmaxf(y, 0.f);
            o[j] = __float2bfloat16(y);
          }
          uint4* dst = reinterpret_cast<uint4*>(a.out_bf + (size_t)v * ncol + c0);
          dst[0] = reinterpret_cast<const uint4*>(o)[0];
          dst[1] = reinterpret_cast<const uint4*>(o)[1];
        } else {
          float4* dst = reinterpret_cast<float4*>(a.out_f + (size_t)v * ncol + c0);
#pragma unroll
          for (int j = 0; j < 4; ++j) dst[j] = make_float4(acc[4 * j], acc[4 * j + 1], acc[4 * j + 2], acc[4 * j + 3]);
        }
      }
    }
  }
  (void)lane;
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(ncols));
}

// ---------------------------------------------------------------------------
// Weight gradient: dW[t][o][i] += sum_v dZ[v][o] X[v + d_t][i]
// GEMM rows m = (tap in the tile, input channel), columns n = o, k = voxels;
// both operands M/N-major (channels contiguous for a voxel).
// ---------------------------------------------------------------------------

struct WgradArgs {
  const bf16* s1;
  const bf16* s2;
  const bf16* dz;  // [V][cout]
  float* dw;       // [27][cout][c1 + c2], accumulated (atomic)
  int c1, lg1, c2, lg, cout, vper;  // vper: voxels per CTA (multiple of 16 kKC)
  int* err;
};

__host__ __device__ constexpr int wgrad_stage_bytes(int cout) { return 128 * 32 * kKC + cout * 32 * kKC; }

__global__ void __launch_bounds__(128) igemm_wgrad(WgradArgs a) {
  extern __shared__ __align__(1024) unsigned char smem[];
  __shared__ __align__(8) uint64_t bars[kStages];
  __shared__ uint32_t tmem_slot;
  const int tid = threadIdx.x, warp = tid >> 5;
  const int lg = a.lg, V = 1 << (3 * lg), m = (1 << lg) - 1;
  const int kin = a.c1 + a.c2, tpt = kin >= 128 ? 1 : 128 / kin;  // taps per M tile
  const int rows = tpt * kin;                                    // <= 128 used rows
  const int tap0 = blockIdx.x * tpt;
  const int vb = blockIdx.y * a.vper, ve = min(V, vb + a.vper);
  const int kvox = 16 * kKC, nst = (ve - vb + kvox - 1) / kvox;
  const int cout = a.cout;
  const int stage_bytes = wgrad_stage_bytes(cout), a_bytes = 128 * 32 * kKC;
  const uint32_t sbase = su32(smem);
  const uint32_t ncols = tmem_cols(cout);
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(&tmem_slot)),
                 "r"(ncols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid < kStages) mbar_init(&bars[tid]);
  if (tid == 0) asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_slot;
  const uint32_t idesc = idesc_bf16(128, cout, 1, 1);
  bool ok = true;
  // M/N-major canonical layout: element (r, kv) at (r/8)*128 + (kv/8)*LBO + (kv%8)*16 + (r%8)*2;
  // A: 16 row-cores, LBO_A = 2048; B: cout/8 row-cores, LBO_B = 16 cout
  const uint32_t LBOA = 2048u, LBOB = (uint32_t)cout * 16u;
  const int agroups = 16;  // 8-row groups of the 128-row A tile

  auto load_stage = [&](int st, int s) {
    const uint32_t sa = sbase + st * stage_bytes, sb = sa + a_bytes;
    // A: (voxel kv, row group g) pairs, 16 bytes each
    for (int e = tid; e < kvox * agroups; e += 128) {
      const int kv = e / agroups, g = e % agroups;
      const uint32_t dst = sa + g * 128 + (kv / 8) * LBOA + (kv % 8) * 16;
      const int vv = vb + s * kvox + kv;
      const int r0 = g * 8, tl = r0 / kin, ci = r0 % kin, tap = tap0 + tl;
      if (vv >= ve || r0 >= rows || tap >= 27) {
        cp_zero16(dst);
        continue;
      }
      const int i = vv >> (2 * lg), j = (vv >> lg) & m, k = vv & m;
      const int u = shift_vox(i, j, k, tap / 9 - 1, (tap / 3) % 3 - 1, tap % 3 - 1, lg);
      const bf16* src;
      if (ci < a.c1) {
        int uu = u;
        if (a.lg1 != lg) {
          const int ui = u >> (2 * lg), uj = (u >> lg) & m, uk = u & m;
          uu = (((ui >> 1) << (lg - 1) | (uj >> 1)) << (lg - 1)) | (uk >> 1);
        }
        src = a.s1 + (size_t)uu * a.c1 + ci;
      } else {
        src = a.s2 + (size_t)u * a.c2 + (ci - a.c1);
      }
      cp16(dst, src);
    }
    // B: (voxel kv, column group g)
    const int bgroups = cout / 8;
    for (int e = tid; e < kvox * bgroups; e += 128) {
      const int kv = e / bgroups, g = e % bgroups;
      const uint32_t dst = sb + g * 128 + (kv / 8) * LBOB + (kv % 8) * 16;
      const int vv = vb + s * kvox + kv;
      if (vv >= ve) cp_zero16(dst);
      else cp16(dst, a.dz + (size_t)vv * cout + g * 8);
    }
  };

#pragma unroll
  for (int s = 0; s < kStages - 1; ++s) {
    if (s < nst) load_stage(s, s);
    cp_commit();
  }
  for (int s = 0; s < nst; ++s) {
    const int sn = s + kStages - 1;
    if (sn < nst) {
      if (sn >= kStages && ok) ok = mbar_wait(&bars[sn % kStages], ((sn - kStages) / kStages) & 1);
      load_stage(sn % kStages, sn);
    }
    cp_commit();
    cp_wait<kStages - 1>();
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    if (tid == 0 && ok) {
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t sa = sbase + (s % kStages) * stage_bytes, sb = sa + a_bytes;
#pragma unroll
      for (int q = 0; q < kKC; ++q)
        mma_bf16(tmem, sdesc(sa + q * 2 * LBOA, LBOA, 128), sdesc(sb + q * 2 * LBOB, LBOB, 128), idesc,
                 (s > 0 || q > 0) ? 1u : 0u);
      mma_commit(&bars[s % kStages]);
    }
  }
  if (nst > 0 && ok) ok = mbar_wait(&bars[(nst - 1) % kStages], ((nst - 1) / kStages) & 1);
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (!ok) {
    if (tid == 0) atomicOr(a.err, 1);
  } else if (nst > 0) {
    const int r = warp * 32 + (threadIdx.x & 31);  // this thread's D row
    const int tl = r / kin, ci = r % kin, tap = tap0 + tl;
    for (int c0 = 0; c0 < cout; c0 += 16) {
      float acc[16];
      tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, acc);
      if (r < rows && tap < 27) {
#pragma unroll
        for (int j = 0; j < 16; ++j) atomicAdd(&a.dw[((size_t)tap * cout + c0 + j) * kin + ci], acc[j]);
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(ncols));
}

// ---------------------------------------------------------------------------
// First layer: the two input features f0 (normalised ln eta) and f1 (the
// expansion-factor feature) to 16 channels.  One GEMM per 128 voxels with
// K = 2 x 27 = 54 (padded to 64): A[v][t] = f0(v + d_t), A[v][27 + t] = f1(v + d_t),
// B[o][t] = W[t][o][0], B[o][27 + t] = W[t][o][1].  The result equals the
// 16-channel convolution of an input whose channels 2..15 are zero.
// ---------------------------------------------------------------------------

__global__ void __launch_bounds__(128) stem_conv(const __nv_bfloat162* __restrict__ f2, int lg,
                                                 const bf16* __restrict__ w, int wcin, const float* __restrict__ bias,
                                                 bf16* __restrict__ out, int* err) {
  __shared__ __align__(1024) unsigned char sm[128 * 128 + 16 * 128];
  __shared__ __align__(8) uint64_t bar;
  __shared__ uint32_t tmem_slot;
  const int tid = threadIdx.x, warp = tid >> 5;
  const int V = 1 << (3 * lg), m = (1 << lg) - 1;
  const int v = blockIdx.x * 128 + tid;
  const bool vok = v < V;
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(&tmem_slot)),
                 "r"(32));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 0) {
    mbar_init(&bar);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  // K-major canonical layout, element (r, kk) at (r/8)*1024 + (kk/8)*128 + (r%8)*16 + (kk%8)*2
  const uint32_t sa = su32(sm), sb = sa + 128 * 128;
  {
    __align__(16) bf16 row[64];
#pragma unroll
    for (int kk = 0; kk < 64; ++kk) row[kk] = __float2bfloat16(0.f);
    if (vok) {
      const int i = v >> (2 * lg), j = (v >> lg) & m, k = v & m;
#pragma unroll
      for (int t = 0; t < 27; ++t) {
        const __nv_bfloat162 x = f2[shift_vox(i, j, k, t / 9 - 1, (t / 3) % 3 - 1, t % 3 - 1, lg)];
        row[t] = x.x;
        row[27 + t] = x.y;
      }
    }
    const uint32_t d = sa + (tid / 8) * 1024 + (tid % 8) * 16;
#pragma unroll
    for (int c = 0; c < 8; ++c) {
      const uint4 q = reinterpret_cast<const uint4*>(row)[c];
      asm volatile("st.shared.v4.u32 [%0], {%1, %2, %3, %4};" ::"r"(d + c * 128), "r"(q.x), "r"(q.y), "r"(q.z),
                   "r"(q.w)
                   : "memory");
    }
  }
  if (tid < 16) {
    __align__(16) bf16 row[64];
#pragma unroll
    for (int kk = 0; kk < 64; ++kk) row[kk] = __float2bfloat16(0.f);
#pragma unroll
    for (int t = 0; t < 27; ++t) {
      row[t] = w[((size_t)t * 16 + tid) * wcin];
      row[27 + t] = w[((size_t)t * 16 + tid) * wcin + 1];
    }
    const uint32_t d = sb + (tid / 8) * 1024 + (tid % 8) * 16;
#pragma unroll
    for (int c = 0; c < 8; ++c) {
      const uint4 q = reinterpret_cast<const uint4*>(row)[c];
      asm volatile("st.shared.v4.u32 [%0], {%1, %2, %3, %4};" ::"r"(d + c * 128), "r"(q.x), "r"(q.y), "r"(q.z),
                   "r"(q.w)
                   : "memory");
    }
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_slot;
  if (tid == 0) {
    const uint32_t idesc = idesc_bf16(128, 16, 0, 0);
#pragma unroll
    for (int q = 0; q < 4; ++q)
      mma_bf16(tmem, sdesc(sa + q * 256, 128, 1024), sdesc(sb + q * 256, 128, 1024), idesc, q > 0 ? 1u : 0u);
    mma_commit(&bar);
  }
  const bool ok = __syncthreads_and(mbar_wait(&bar, 0)) != 0;
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (!ok) {
    if (tid == 0) atomicOr(err, 1);
  } else {
    float acc[16];
    tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16), acc);
    if (vok) {
      __align__(16) bf16 o[16];
#pragma unroll
      for (int j = 0; j < 16; ++j) o[j] = __float2bfloat16(fmaxf(acc[j] + bias[j], 0.f));
      uint4* dst = reinterpret_cast<uint4*>(out + (size_t)v * 16);
      dst[0] = reinterpret_cast<const uint4*>(o)[0];
      dst[1] = reinterpret_cast<const uint4*>(o)[1];
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(32));
}

// ---------------------------------------------------------------------------
// Line convolution (forward, grids of n >= 32 cells per side).
//
// One CTA computes a unit of P = max(n, 128) output positions: one grid row
// (i, j, 0..n-1) when n >= 128, else R = 128/n consecutive rows of plane i.
// For every (di, dj) and every 16-channel slice it stages the R source rows
// (i+di, j+r+dj), all n voxels along k, as the A operand (rows = positions,
// no gather), and one MMA with N = 3 cout multiplies it by the weights of the
// three taps dk = -1, 0, 1 at once:
//     Acc[dk][u][o] += sum_c X[(i+di, j+r+dj, u)][c] W[(di,dj,dk)][o][c].
// The k shift is applied once, in the epilogue:
//     out[(i, j+r, k)][o] = b[o] + sum_dk Acc[dk][(k + dk) mod n][o].
// A source read by nearest upsampling from the half-resolution grid is staged
// at its own resolution along k (n/2 positions per row, half the MMAs); its
// epilogue index is ((k + dk) mod n) / 2.
// ---------------------------------------------------------------------------

struct LineArgs {
  const bf16* s1;  // c1 channels; grid lg, or lg - 1 when up1
  const bf16* s2;  // c2 channels on grid lg, or nullptr
  const bf16* w;   // [27][cout][c1 + c2]
  const float* bias;
  bf16* out;       // [V][cout]
  int c1, up1, c2, lg, cout, relu;
  int* err;
};

constexpr int kLS = 6;  // pipeline stages
constexpr int kStg = 49;  // floats per staged (position, channel group): 3 x 16 + 1 (bank offset)

__host__ __device__ inline int line_tiles(int lg) { return lg >= 7 ? 1 << (lg - 7) : 1; }
__host__ __device__ inline int line_stage_bytes(int lg, int cout) { return 4096 * line_tiles(lg) + 96 * cout; }
__host__ __device__ inline int line_tiles1(int lg, int up1) {
  const int T = line_tiles(lg);
  return up1 ? (T > 1 ? T / 2 : 1) : T;
}
__host__ __device__ inline int line_tmem_cols(int lg, int up1, int c2, int cout) {
  return 3 * cout * (line_tiles1(lg, up1) + (c2 > 0 ? line_tiles(lg) : 0));
}
__host__ __device__ inline int line_smem(int lg, int up1, int c2, int cout) {
  const int pipe = kLS * line_stage_bytes(lg, cout);
  const int stg = 128 * (line_tiles1(lg, up1) + (c2 > 0 ? line_tiles(lg) : 0)) * kStg * 4;
  return pipe > stg ? pipe : stg;
}

__global__ void __launch_bounds__(128) line_conv(LineArgs a) {
  extern __shared__ __align__(1024) unsigned char smem[];
  __shared__ __align__(8) uint64_t bars[kLS];
  __shared__ uint32_t tmem_slot;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int lg = a.lg, n = 1 << lg, msk = n - 1;
  const int T = line_tiles(lg), R = lg >= 7 ? 1 : 128 >> lg, P = R * n;
  const int T1 = line_tiles1(lg, a.up1);
  const int cout = a.cout, N3 = 3 * cout, kin = a.c1 + a.c2;
  const int S1 = a.c1 / 16, S2 = a.c2 / 16, nst = 9 * (S1 + S2);
  const int upp = n / R;  // units per plane
  const int pi = blockIdx.x / upp, j0 = (blockIdx.x % upp) * R;
  const int a_bytes = 4096 * T, stage_bytes = a_bytes + 96 * cout;
  const uint32_t LBOA = 2048u * T, LBOB = 16u * N3;
  const uint32_t col2 = (uint32_t)(T1 * N3);
  const uint32_t ncols = tmem_cols(line_tmem_cols(lg, a.up1, a.c2, cout));
  const uint32_t sbase = su32(smem);

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(&tmem_slot)),
                 "r"(ncols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid < kLS) mbar_init(&bars[tid]);
  if (tid == 0) asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_slot;
  const uint32_t idesc = idesc_bf16(128, N3, 0, 0);
  bool ok = true;

  // A: position p of chunk c (channels 8c..8c+7 of the slice) at c*LBOA + p*16;
  // B: row dk*cout + o of chunk c at c*LBOB + (dk*cout + o)*16.
  auto load_stage = [&](int slot, int s) {
    const int src = s < 9 * S1 ? 0 : 1;
    const int qq = src ? s - 9 * S1 : s;
    const int slice = qq / 9, line = qq % 9;
    const int di = line / 3 - 1, dj = line % 3 - 1;
    const uint32_t sa = sbase + slot * stage_bytes, sb = sa + a_bytes;
    const int ri = (pi + di) & msk;
    const bool up = src == 0 && a.up1;
    const bf16* base = src ? a.s2 : a.s1;
    const int C = src ? a.c2 : a.c1, c0 = slice * 16;
    const int hl = up ? lg - 1 : lg;             // log2 of the staged positions per row
    const int lv = hl + (lg >= 7 ? 0 : 7 - lg);  // log2 of the staged positions per unit
    const int nv = 1 << lv;
    for (int q = tid; q < 2 * nv; q += 128) {
      const int c = q >> lv, e = q & (nv - 1);
      const int r = e >> hl, k = e & ((1 << hl) - 1);
      const int rj = (j0 + r + dj) & msk;
      const int vox = up ? ((((ri >> 1) << (lg - 1)) | (rj >> 1)) << (lg - 1)) | k : (((ri << lg) | rj) << lg) | k;
      cp16(sa + c * LBOA + (uint32_t)(r * n + k) * 16u, base + (size_t)vox * C + c0 + 8 * c);
    }
    const int tap0 = (di + 1) * 9 + (dj + 1) * 3;
    const int coff = (src ? a.c1 : 0) + c0;
    for (int q = tid; q < 2 * N3; q += 128) {
      const int c = q / N3, nn = q - c * N3;
      const int dki = nn / cout, o = nn - dki * cout;
      cp16(sb + c * LBOB + (uint32_t)nn * 16u, a.w + ((size_t)(tap0 + dki) * cout + o) * kin + coff + 8 * c);
    }
  };

  // prologue: stages 0 .. kLS-3 in flight; stage s + kLS - 2 is loaded at step s
  // into the slot last read by the MMAs of step s - 2.
#pragma unroll
  for (int s = 0; s < kLS - 2; ++s) {
    if (s < nst) load_stage(s, s);
    cp_commit();
  }
  for (int s = 0; s < nst; ++s) {
    const int sn = s + kLS - 2;
    if (sn < nst) {
      if (sn >= kLS && ok) ok = mbar_wait(&bars[sn % kLS], ((sn - kLS) / kLS) & 1);
      if (ok) load_stage(sn % kLS, sn);
    }
    cp_commit();
    cp_wait<kLS - 2>();
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    if (tid == 0 && ok) {
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const int src = s < 9 * S1 ? 0 : 1;
      const bool first = src ? s == 9 * S1 : s == 0;
      const int Ts = src ? T : T1;
      const uint32_t col = src ? col2 : 0u;
      const uint32_t sa = sbase + (s % kLS) * stage_bytes, sb = sa + a_bytes;
      const uint64_t bd = sdesc(sb, LBOB, 128);
      for (int t = 0; t < Ts; ++t)
        mma_bf16(tmem + col + (uint32_t)(t * N3), sdesc(sa + t * 2048, LBOA, 128), bd, idesc, first ? 0u : 1u);
      mma_commit(&bars[s % kLS]);
    }
  }
  cp_wait<0>();
  if (ok) ok = mbar_wait(&bars[(nst - 1) % kLS], ((nst - 1) / kLS) & 1);
  ok = __syncthreads_and(ok) != 0;  // block-uniform from here on
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (!ok && tid == 0) atomicOr(a.err, 1);
  // epilogue, one group of 16 output channels at a time, through shared memory
  float* stg = reinterpret_cast<float*>(smem);
  const int off2 = 128 * T1 * kStg;
  for (int g = 0; g < cout / 16 && ok; ++g) {
    for (int src = 0; src < (S2 ? 2 : 1); ++src) {
      const int Ts = src ? T : T1;
      const uint32_t col = src ? col2 : 0u;
      for (int t = 0; t < Ts; ++t)
        for (int dki = 0; dki < 3; ++dki) {
          float v[16];
          tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + col + (uint32_t)(t * N3 + dki * cout + g * 16), v);
          float* d = stg + (src ? off2 : 0) + (t * 128 + warp * 32 + lane) * kStg + dki * 16;
#pragma unroll
          for (int j = 0; j < 16; ++j) d[j] = v[j];
        }
    }
    __syncthreads();
    for (int p = tid; p < P; p += 128) {
      const int r = p >> lg, k = p & msk;
      float acc[16];
#pragma unroll
      for (int j = 0; j < 16; ++j) acc[j] = a.bias[g * 16 + j];
#pragma unroll
      for (int dki = 0; dki < 3; ++dki) {
        const int kk = (k + dki - 1) & msk;
        const float* s1p = stg + (r * n + (a.up1 ? kk >> 1 : kk)) * kStg + dki * 16;
#pragma unroll
        for (int j = 0; j < 16; ++j) acc[j] += s1p[j];
        if (S2) {
          const float* s2p = stg + off2 + (r * n + kk) * kStg + dki * 16;
#pragma unroll
          for (int j = 0; j < 16; ++j) acc[j] += s2p[j];
        }
      }
      __align__(16) bf16 o[16];
#pragma unroll
      for (int j = 0; j < 16; ++j) o[j] = __float2bfloat16(a.relu ? fmaxf(acc[j], 0.f) : acc[j]);
      uint4* dst = reinterpret_cast<uint4*>(a.out + ((((size_t)pi << lg | (size_t)(j0 + r)) << lg) | k) * cout +
                                            g * 16);
      dst[0] = reinterpret_cast<const uint4*>(o)[0];
      dst[1] = reinterpret_cast<const uint4*>(o)[1];
    }
    __syncthreads();
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(ncols));
}

// ---------------------------------------------------------------------------
// Element-wise and transfer kernels
// ---------------------------------------------------------------------------

// Input features: channel 0 = (ln eta - mu) / sd, channel 1 = (a - a0) / sa, others 0.
__global__ void input_features(const double* __restrict__ eta, int V, float mu, float isd, float afeat,
                               bf16* __restrict__ x, __nv_bfloat162* __restrict__ f2) {
  int v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= V) return;
  const bf16 f0 = __float2bfloat16((logf((float)fmax(eta[v], 1e-30)) - mu) * isd), f1 = __float2bfloat16(afeat);
  if (f2) f2[v] = __halves2bfloat162(f0, f1);
  if (!x) return;
  __align__(16) bf16 o[16];
#pragma unroll
  for (int c = 0; c < 16; ++c) o[c] = __float2bfloat16(0.f);
  o[0] = f0;
  o[1] = f1;
  uint4* dst = reinterpret_cast<uint4*>(x + (size_t)v * 16);
  dst[0] = reinterpret_cast<const uint4*>(o)[0];
  dst[1] = reinterpret_cast<const uint4*>(o)[1];
}

// Mean over the 8 children (lg: coarse grid).
__global__ void pool_fwd(const bf16* __restrict__ x, int C, int lg, bf16* __restrict__ y) {
  const int Vc = 1 << (3 * lg), m = (1 << lg) - 1, lgf = lg + 1;
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= Vc * C) return;
  const int u = t / C, c = t % C;
  const int I = u >> (2 * lg), J = (u >> lg) & m, K = u & m;
  float s = 0.f;
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    const int f = (((2 * I + (q >> 2)) << lgf | (2 * J + ((q >> 1) & 1))) << lgf) | (2 * K + (q & 1));
    s += __bfloat162float(x[(size_t)f * C + c]);
  }
  y[t] = __float2bfloat16(0.125f * s);
}

// dX[fine] += dY[parent] / 8 (lg: coarse grid).
__global__ void pool_bwd(const float* __restrict__ dy, int C, int lg, float* __restrict__ dx) {
  const int lgf = lg + 1, Vf = 1 << (3 * lgf), mf = (1 << lgf) - 1;
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= Vf * C) return;
  const int f = t / C, c = t % C;
  const int i = f >> (2 * lgf), j = (f >> lgf) & mf, k = f & mf;
  const int u = (((i >> 1) << lg | (j >> 1)) << lg) | (k >> 1);
  dx[t] += 0.125f * dy[(size_t)u * C + c];
}

// dZ = dY where the stored activation is positive (ReLU), else 0; BF16 for the GEMMs.
__global__ void relu_bwd(const float* __restrict__ dy, const bf16* __restrict__ y, size_t n, bf16* __restrict__ dz) {
  size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n) return;
  dz[t] = __float2bfloat16(__bfloat162float(y[t]) > 0.f ? dy[t] : 0.f);
}

// Split the gradient of a concatenated input: channels [0, c1) belong to src1
// (summed over the 8 fine voxels of its half-resolution cell when upsampled),
// channels [c1, c1 + c2) are added into the gradient of src2.
__global__ void split_up_bwd(const float* __restrict__ dx, int c1, int c2, int lg, int up, float* __restrict__ d1,
                             float* __restrict__ d2) {
  const int kin = c1 + c2, V = 1 << (3 * lg), m = (1 << lg) - 1;
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (up) {
    const int lgc = lg - 1, Vc = 1 << (3 * lgc), mc = (1 << lgc) - 1;
    if (t < Vc * c1) {
      const int u = t / c1, c = t % c1;
      const int I = u >> (2 * lgc), J = (u >> lgc) & mc, K = u & mc;
      float s = 0.f;
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const int f = (((2 * I + (q >> 2)) << lg | (2 * J + ((q >> 1) & 1))) << lg) | (2 * K + (q & 1));
        s += dx[(size_t)f * kin + c];
      }
      d1[t] = s;
    }
  } else if (t < V * c1) {
    const int v = t / c1, c = t % c1;
    d1[t] = dx[(size_t)v * kin + c];
  }
  if (c2 > 0 && t < V * c2) {
    const int v = t / c2, c = t % c2;
    d2[t] += dx[(size_t)v * kin + c1 + c];
  }
  (void)m;
}

// Output head (1x1x1 convolution to one channel) and squared-error loss:
//   p[v] = b + sum_c h[c] y[v][c];  r = p - target;  loss += r^2 / V
// and its gradients dY[v][c] = (2 r / V) h[c], dh[c] += sum (2 r / V) y[v][c], db += sum 2 r / V.
// pred (optional) receives p.
__global__ void head_fwd_bwd(const bf16* __restrict__ y, int C, int V, const float* __restrict__ hb,
                             const float* __restrict__ target, float tscale, float* __restrict__ pred,
                             float* __restrict__ dy, float* __restrict__ dhb, double* __restrict__ loss) {
  __shared__ float sdh[65];
  __shared__ double sl;
  if (threadIdx.x <= C) sdh[threadIdx.x] = 0.f;
  if (threadIdx.x == 0) sl = 0.0;
  __syncthreads();
  int v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v < V) {
    float p = hb[C];
    for (int c = 0; c < C; ++c) p += hb[c] * __bfloat162float(y[(size_t)v * C + c]);
    if (pred) pred[v] = p;
    if (target) {
      const float r = p - tscale * target[v];
      const float g = 2.f * r / (float)V;
      atomicAdd(&sl, (double)r * r / V);
      if (dy)
        for (int c = 0; c < C; ++c) {
          dy[(size_t)v * C + c] = g * hb[c];
          atomicAdd(&sdh[c], g * __bfloat162float(y[(size_t)v * C + c]));
        }
      atomicAdd(&sdh[C], g);
    }
  }
  __syncthreads();
  if (target && dhb && threadIdx.x <= C) atomicAdd(&dhb[threadIdx.x], sdh[threadIdx.x]);
  if (target && loss && threadIdx.x == 0) atomicAdd(loss, sl);
}

// Bias gradient db[o] += sum_v dZ[v][o].
__global__ void bias_grad(const bf16* __restrict__ dz, int C, int V, float* __restrict__ db) {
  __shared__ float s[64];
  if (threadIdx.x < C) s[threadIdx.x] = 0.f;
  __syncthreads();
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < V * C; t += gridDim.x * blockDim.x)
    atomicAdd(&s[t % C], __bfloat162float(dz[t]));
  __syncthreads();
  if (threadIdx.x < C) atomicAdd(&db[threadIdx.x], s[threadIdx.x]);
}

// Adam on FP32 master parameters (bias-corrected step sizes passed in), then
// the BF16 copy used by the convolutions.
__global__ void adam_step(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m1,
                          float* __restrict__ m2, int n, float lr1, float lr2c, float b1, float b2, float eps,
                          bf16* __restrict__ pb) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n) return;
  const float gi = g[t];
  const float a = b1 * m1[t] + (1.f - b1) * gi, b = b2 * m2[t] + (1.f - b2) * gi * gi;
  m1[t] = a;
  m2[t] = b;
  const float q = p[t] - lr1 * a / (sqrtf(b * lr2c) + eps);
  p[t] = q;
  if (pb) pb[t] = __float2bfloat16(q);
}

// Wt[t][i][o] = W[t][o][i] (BF16), the operand of the input gradient.
__global__ void transpose_w(const bf16* __restrict__ w, int cout, int cin, bf16* __restrict__ wt) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= 27 * cout * cin) return;
  const int tap = t / (cout * cin), r = t % (cout * cin), o = r / cin, i = r % cin;
  wt[((size_t)tap * cin + i) * cout + o] = w[t];
}

__global__ void to_bf16(const float* __restrict__ a, bf16* __restrict__ b, size_t n) {
  size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t < n) b[t] = __float2bfloat16(a[t]);
}

// Initial guess from the net: phi = bg + scale * p.
__global__ void guess_out(const float* __restrict__ p, int V, double bg, double scale, double* __restrict__ phi) {
  int v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v < V) phi[v] = bg + scale * (double)p[v];
}

inline unsigned nb(size_t n, int t) { return (unsigned)((n + t - 1) / t); }

static bool aligned16(const void* p) { return ((uintptr_t)p & 15u) == 0; }

}  // namespace unet
}  // namespace isis

using namespace isis::unet;

#define UNET_LAUNCH(kind, bytes, st, ...) ISIS_LAUNCH(kind, bytes, st, __VA_ARGS__)

extern "C" {

isis_status isis_unet_conv3_fwd(const void* src1, int c1, int lg1, const void* src2, int c2, int lg, const void* w,
                                const float* bias, int cout, int relu, void* out, int* err, void* stream) {
  if (!src1 || !w || !bias || !out || !err || lg < 2 || lg > 10 || (lg1 != lg && lg1 != lg - 1)) return ISIS_EINVAL;
  if (c1 < 16 || c1 % 16 || c2 < 0 || c2 % 16 || (c2 > 0 && !src2) || cout < 16 || cout > 64 || cout % 16)
    return ISIS_EINVAL;
  if (!aligned16(src1) || (src2 && !aligned16(src2)) || !aligned16(w) || !aligned16(out)) return ISIS_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  const size_t V = (size_t)1 << (3 * lg);
  const double flops = 2.0 * 27.0 * (c1 + c2) * cout * (double)V;
  const int up1 = lg1 != lg;
  if (lg >= 5 && lg <= 9 && line_tmem_cols(lg, up1, c2, cout) <= 512 && line_smem(lg, up1, c2, cout) <= 200 * 1024) {
    static bool lattr = false;
    if (!lattr) {
      if (cudaFuncSetAttribute(line_conv, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024) != cudaSuccess)
        return ISIS_ECUDA;
      lattr = true;
    }
    LineArgs la{(const bf16*)src1, (const bf16*)src2, (const bf16*)w, bias, (bf16*)out, c1, up1, c2, lg, cout,
                relu, err};
    const int P = lg >= 7 ? 1 << lg : 128;
    UNET_LAUNCH(isis::KK_UNET_CONV, flops, st,
                (line_conv<<<(unsigned)(V / P), 128, line_smem(lg, up1, c2, cout), st>>>(la)));
    return ISIS_OK;
  }
  ConvArgs a{(const bf16*)src1, (const bf16*)src2, (const bf16*)w, bias, (bf16*)out, nullptr,
             c1, lg1, c2, lg, cout, relu, +1, err};
  const size_t smem = (size_t)kStages * conv_stage_bytes(cout);
  static bool attr = false;
  if (!attr) {
    if (cudaFuncSetAttribute(igemm_conv<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, 96 * 1024) != cudaSuccess)
      return ISIS_ECUDA;
    attr = true;
  }
  UNET_LAUNCH(isis::KK_UNET_CONV, flops, st, (igemm_conv<0><<<nb(V, 128), 128, smem, st>>>(a)));
  return ISIS_OK;
}

isis_status isis_unet_conv3_dgrad(const void* dz, int cout, int lg, const void* wt, int cin, float* din, int* err,
                                  void* stream) {
  if (!dz || !wt || !din || !err || lg < 2 || lg > 10 || cout < 16 || cout % 16 || cin < 16 || cin > 128 ||
      cin % 16)
    return ISIS_EINVAL;
  ConvArgs a{(const bf16*)dz, nullptr, (const bf16*)wt, nullptr, nullptr, din, cout, lg, 0, lg, cin, 0, -1, err};
  cudaStream_t st = (cudaStream_t)stream;
  const size_t smem = (size_t)kStages * conv_stage_bytes(cin);
  static bool attr = false;
  if (!attr) {
    if (cudaFuncSetAttribute(igemm_conv<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, 96 * 1024) != cudaSuccess)
      return ISIS_ECUDA;
    attr = true;
  }
  const size_t V = (size_t)1 << (3 * lg);
  const double flops = 2.0 * 27.0 * cin * cout * (double)V;
  UNET_LAUNCH(isis::KK_UNET_CONV, flops, st, (igemm_conv<1><<<nb(V, 128), 128, smem, st>>>(a)));
  return ISIS_OK;
}

isis_status isis_unet_conv3_wgrad(const void* src1, int c1, int lg1, const void* src2, int c2, int lg,
                                  const void* dz, int cout, float* dw, int* err, void* stream) {
  if (!src1 || !dz || !dw || !err || lg < 2 || lg > 10 || (lg1 != lg && lg1 != lg - 1)) return ISIS_EINVAL;
  if (c1 < 16 || c1 % 16 || c2 < 0 || c2 % 16 || (c2 > 0 && !src2) || cout < 16 || cout > 64 || cout % 16 ||
      c1 + c2 > 128)
    return ISIS_EINVAL;
  const int kin = c1 + c2, tpt = kin >= 128 ? 1 : 128 / kin, mt = (27 + tpt - 1) / tpt;
  const size_t V = (size_t)1 << (3 * lg);
  // about 4 CTAs per SM in total, each over a whole number of 32-voxel stages
  size_t target = (size_t)(152 * 4 / mt) + 1;
  size_t vper = (V + target - 1) / target;
  vper = ((vper + 31) / 32) * 32;
  if (vper < 512) vper = 512;
  WgradArgs a{(const bf16*)src1, (const bf16*)src2, (const bf16*)dz, dw, c1, lg1, c2, lg, cout, (int)vper, err};
  cudaStream_t st = (cudaStream_t)stream;
  const size_t smem = (size_t)kStages * wgrad_stage_bytes(cout);
  static bool attr = false;
  if (!attr) {
    if (cudaFuncSetAttribute(igemm_wgrad, cudaFuncAttributeMaxDynamicSharedMemorySize, 96 * 1024) != cudaSuccess)
      return ISIS_ECUDA;
    attr = true;
  }
  dim3 grid((unsigned)mt, (unsigned)((V + vper - 1) / vper));
  const double flops = 2.0 * 27.0 * kin * cout * (double)V;
  UNET_LAUNCH(isis::KK_UNET_CONV, flops, st, (igemm_wgrad<<<grid, 128, smem, st>>>(a)));
  return ISIS_OK;
}

isis_status isis_unet_input(const double* eta, int lg, float mu, float isd, float afeat, void* x16, void* f2,
                            void* stream) {
  if (!eta || (!x16 && !f2) || lg < 2 || lg > 10) return ISIS_EINVAL;
  if ((x16 && !aligned16(x16)) || (f2 && ((uintptr_t)f2 & 3u))) return ISIS_EINVAL;
  const int V = 1 << (3 * lg);
  cudaStream_t st = (cudaStream_t)stream;
  UNET_LAUNCH(isis::KK_UNET_ELEM, (8.0 + (x16 ? 32.0 : 0.0) + (f2 ? 4.0 : 0.0)) * V, st,
              (input_features<<<nb(V, 256), 256, 0, st>>>(eta, V, mu, isd, afeat, (bf16*)x16,
                                                          (__nv_bfloat162*)f2)));
  return ISIS_OK;
}

isis_status isis_unet_stem_fwd(const void* f2, int lg, const void* w, int wcin, const float* bias, void* out,
                               int* err, void* stream) {
  if (!f2 || !w || !bias || !out || !err || lg < 2 || lg > 10 || wcin < 2 || wcin % 8) return ISIS_EINVAL;
  if (((uintptr_t)f2 & 3u) || !aligned16(out)) return ISIS_EINVAL;
  const size_t V = (size_t)1 << (3 * lg);
  cudaStream_t st = (cudaStream_t)stream;
  const double flops = 2.0 * 27.0 * 2.0 * 16.0 * (double)V;
  UNET_LAUNCH(isis::KK_UNET_CONV, flops, st,
              (stem_conv<<<nb(V, 128), 128, 0, st>>>((const __nv_bfloat162*)f2, lg, (const bf16*)w, wcin, bias,
                                                       (bf16*)out, err)));
  return ISIS_OK;
}

isis_status isis_unet_pool_fwd(const void* x, int C, int lgc, void* y, void* stream) {
  if (!x || !y || C < 1 || lgc < 1) return ISIS_EINVAL;
  const size_t n = ((size_t)1 << (3 * lgc)) * C;
  cudaStream_t st = (cudaStream_t)stream;
  UNET_LAUNCH(isis::KK_UNET_ELEM, 18.0 * n, st,
              (pool_fwd<<<nb(n, 256), 256, 0, st>>>((const bf16*)x, C, lgc, (bf16*)y)));
  return ISIS_OK;
}

isis_status isis_unet_pool_bwd(const float* dy, int C, int lgc, float* dx, void* stream) {
  if (!dy || !dx || C < 1 || lgc < 1) return ISIS_EINVAL;
  const size_t n = ((size_t)1 << (3 * (lgc + 1))) * C;
  cudaStream_t st = (cudaStream_t)stream;
  UNET_LAUNCH(isis::KK_UNET_ELEM, 12.0 * n, st, (pool_bwd<<<nb(n, 256), 256, 0, st>>>(dy, C, lgc, dx)));
  return ISIS_OK;
}

isis_status isis_unet_relu_bwd(const float* dy, const void* y, int64_t n, void* dz, void* stream) {
  if (!dy || !y || !dz || n < 1) return ISIS_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  UNET_LAUNCH(isis::KK_UNET_ELEM, 8.0 * n, st,
              (relu_bwd<<<nb((size_t)n, 256), 256, 0, st>>>(dy, (const bf16*)y, (size_t)n, (bf16*)dz)));
  return ISIS_OK;
}

isis_status isis_unet_split_bwd(const float* dx, int c1, int c2, int lg, int up, float* d1, float* d2,
                                void* stream) {
  if (!dx || !d1 || (c2 > 0 && !d2) || lg < 1) return ISIS_EINVAL;
  const size_t V = (size_t)1 << (3 * lg);
  const size_t n = V * (size_t)(c1 > c2 ? c1 : c2);
  cudaStream_t st = (cudaStream_t)stream;
  UNET_LAUNCH(isis::KK_UNET_ELEM, 8.0 * V * (c1 + c2), st,
              (split_up_bwd<<<nb(n, 256), 256, 0, st>>>(dx, c1, c2, lg, up, d1, d2)));
  return ISIS_OK;
}

isis_status isis_unet_head(const void* y, int C, int lg, const float* hb, const float* target, float tscale,
                           float* pred, float* dy, float* dhb, double* loss, void* stream) {
  if (!y || !hb || C < 1 || C > 64 || lg < 1) return ISIS_EINVAL;
  const int V = 1 << (3 * lg);
  cudaStream_t st = (cudaStream_t)stream;
  UNET_LAUNCH(isis::KK_UNET_ELEM, (2.0 * C + 8.0) * V, st,
              (head_fwd_bwd<<<nb(V, 256), 256, 0, st>>>((const bf16*)y, C, V, hb, target, tscale, pred, dy, dhb,
                                                          loss)));
  return ISIS_OK;
}

isis_status isis_unet_bias_grad(const void* dz, int C, int lg, float* db, void* stream) {
  if (!dz || !db || C < 1 || C > 64) return ISIS_EINVAL;
  const int V = 1 << (3 * lg);
  cudaStream_t st = (cudaStream_t)stream;
  UNET_LAUNCH(isis::KK_UNET_ELEM, 2.0 * V * C, st,
              (bias_grad<<<608, 256, 0, st>>>((const bf16*)dz, C, V, db)));
  return ISIS_OK;
}

isis_status isis_unet_adam(float* p, const float* g, float* m1, float* m2, int64_t n, float lr, float b1, float b2,
                           float eps, int step, void* pbf16, void* stream) {
  if (!p || !g || !m1 || !m2 || n < 1 || step < 1) return ISIS_EINVAL;
  // bias corrections folded into the step: p -= lr/(1-b1^t) m / (sqrt(v/(1-b2^t)) + eps)
  double c1 = 1.0 - pow((double)b1, step), c2 = 1.0 - pow((double)b2, step);
  cudaStream_t st = (cudaStream_t)stream;
  UNET_LAUNCH(isis::KK_UNET_ELEM, 22.0 * n, st,
              (adam_step<<<nb((size_t)n, 256), 256, 0, st>>>(p, g, m1, m2, (int)n, (float)(lr / c1), (float)(1.0 / c2),
                                                              b1, b2, eps, (bf16*)pbf16)));
  return ISIS_OK;
}

isis_status isis_unet_transpose_w(const void* w, int cout, int cin, void* wt, void* stream) {
  if (!w || !wt) return ISIS_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  const size_t n = (size_t)27 * cout * cin;
  UNET_LAUNCH(isis::KK_UNET_ELEM, 4.0 * n, st,
              (transpose_w<<<nb(n, 256), 256, 0, st>>>((const bf16*)w, cout, cin, (bf16*)wt)));
  return ISIS_OK;
}

isis_status isis_unet_to_bf16(const float* a, int64_t n, void* b, void* stream) {
  if (!a || !b || n < 1) return ISIS_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  UNET_LAUNCH(isis::KK_UNET_ELEM, 6.0 * n, st,
              (to_bf16<<<nb((size_t)n, 256), 256, 0, st>>>(a, (bf16*)b, (size_t)n)));
  return ISIS_OK;
}

isis_status isis_unet_guess(const float* pred, int lg, double bg, double scale, double* phi, void* stream) {
  if (!pred || !phi) return ISIS_EINVAL;
  const int V = 1 << (3 * lg);
  cudaStream_t st = (cudaStream_t)stream;
  UNET_LAUNCH(isis::KK_UNET_ELEM, 12.0 * V, st, (guess_out<<<nb(V, 256), 256, 0, st>>>(pred, V, bg, scale, phi)));
  return ISIS_OK;
}

}  // extern "C"
