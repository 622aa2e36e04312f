// isis_unet.cu -- kernels of the learned initial guess: a small 3-D U-Net whose
// 3x3x3 periodic convolutions are implicit GEMMs on the 5th-generation tensor
// cores (tcgen05.mma, BF16 operands in shared memory, FP32 accumulators in
// tensor memory), trained by the library's own backward and Adam kernels.
// The paper has no learned part; the net only proposes the initial guess and
// the multigrid solver always finishes the solve.
//
// Tensors: a grid of n = 2^lg cells per side, V = n^3 voxels in row-major
// order, C channels (a multiple of 16), stored channel-planar in groups of 8:
// element (v, c) at ((c / 8) V + v) 8 + c % 8.  A grid row of one 8-channel
// group is then one contiguous block (n x 16 bytes for BF16), which the line
// convolution fetches with single bulk copies.
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
#include <cstring>

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

// Polling wait (mbarrier.test_wait never suspends the thread), then the bounded
// blocking wait above; false if both gave up.
__device__ __forceinline__ bool mbar_wait_spin(uint64_t* bar, uint32_t parity) {
  for (int it = 0; it < (1 << 14); ++it) {
    uint32_t done;
    asm volatile(
        "{\n.reg .pred p;\nmbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(su32(bar)), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return mbar_wait(bar, parity);
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

// element (v, c) of a channel-planar tensor with V voxels
__device__ __forceinline__ size_t pidx(size_t v, int c, size_t V) { return (((size_t)(c >> 3) * V + v) << 3) | (c & 7); }

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
        const bf16 *src, *src8;  // channels c0..c0+7 and c0+8..c0+15 (two 8-channel planes)
        if (c0 < a.c1) {
          const int u = shift_vox(vi, vj, vk, di, dj, dk, lg);
          int uu = u;
          if (a.lg1 != lg) {  // nearest upsampling from the half-resolution grid
            const int ui = u >> (2 * lg), uj = (u >> lg) & m, uk = u & m;
            uu = (((ui >> 1) << (lg - 1) | (uj >> 1)) << (lg - 1)) | (uk >> 1);
          }
          const size_t V1 = (size_t)1 << (3 * a.lg1);
          src = a.s1 + pidx(uu, c0, V1);
          src8 = a.s1 + pidx(uu, c0 + 8, V1);
        } else {
          const int u = shift_vox(vi, vj, vk, di, dj, dk, lg);
          src = a.s2 + pidx(u, c0 - a.c1, (size_t)V);
          src8 = a.s2 + pidx(u, c0 - a.c1 + 8, (size_t)V);
        }
        cp16(da, src);
        cp16(da + 128, src8);
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
          *reinterpret_cast<uint4*>(a.out_bf + pidx(v, c0, (size_t)V)) = reinterpret_cast<const uint4*>(o)[0];
          *reinterpret_cast<uint4*>(a.out_bf + pidx(v, c0 + 8, (size_t)V)) = reinterpret_cast<const uint4*>(o)[1];
        } else {
          float4* d0 = reinterpret_cast<float4*>(a.out_f + pidx(v, c0, (size_t)V));
          float4* d1 = reinterpret_cast<float4*>(a.out_f + pidx(v, c0 + 8, (size_t)V));
          d0[0] = make_float4(acc[0], acc[1], acc[2], acc[3]);
          d0[1] = make_float4(acc[4], acc[5], acc[6], acc[7]);
          d1[0] = make_float4(acc[8], acc[9], acc[10], acc[11]);
          d1[1] = make_float4(acc[12], acc[13], acc[14], acc[15]);
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
        src = a.s1 + pidx(uu, ci, (size_t)1 << (3 * a.lg1));
      } else {
        src = a.s2 + pidx(u, ci - a.c1, (size_t)V);
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
      else cp16(dst, a.dz + pidx(vv, g * 8, (size_t)V));
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
      *reinterpret_cast<uint4*>(out + pidx(v, 0, (size_t)V)) = reinterpret_cast<const uint4*>(o)[0];
      *reinterpret_cast<uint4*>(out + pidx(v, 8, (size_t)V)) = reinterpret_cast<const uint4*>(o)[1];
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(32));
}

// ---------------------------------------------------------------------------
// Line convolution (forward, grids of n >= 32 cells per side).
//
// A unit is P = max(n, 128) output positions: one grid row (i, j, 0..n-1)
// when n >= 128, else R = 128/n consecutive rows of plane i.  For every
// (di, dj) and every 16-channel slice of a source, the R source rows
// (i+di, j+r+dj), all voxels along k, are the A operand (rows = positions, no
// gather), and one MMA with N = 3 cout multiplies it by the weights of the
// three taps dk = -1, 0, 1 at once:
//     Acc[dk][u][o] += sum_c X[(i+di, j+r+dj, u)][c] W[(di,dj,dk)][o][c].
// The k shift is applied once, in the epilogue:
//     out[(i, j+r, k)][o] = b[o] + sum_dk Acc[dk][(k + dk) mod n][o].
// A source read by nearest upsampling from the half-resolution grid is staged
// at its own resolution along k (n/2 positions per row, half the MMAs); its
// epilogue index is ((k + dk) mod n) / 2.
//
// Persistent CTAs with three roles: warp 0 issues the bulk copies (a source
// row of one 8-channel plane is one contiguous block, so a stage is 2R + 1
// copies: the A rows of both planes of the slice and the stage's pre-packed
// weights), warp 1 the tcgen05 MMAs, warps 2..5 the epilogue.  Accumulators
// are double buffered in TMEM so the epilogue of one unit overlaps the MMAs
// of the next.  Operands use the no-swizzle K-major layout: 8-channel chunk
// planes of 16-byte rows.
// ---------------------------------------------------------------------------

struct LineArgs {
  const bf16* s1;  // c1 channels; grid lg, or lg - 1 when up1 (channel-planar)
  const bf16* s2;  // c2 channels on grid lg (channel-planar), or nullptr
  const bf16* wl;  // weights packed per stage (isis_unet_pack_w)
  const float* bias;
  bf16* out;  // cout channels on grid lg (channel-planar)
  int c1, up1, c2, lg, cout, relu, nunits, nls;
  int* err;
};

#ifndef ISIS_LINE_STAGES
#define ISIS_LINE_STAGES 4
#endif
constexpr int kLS = ISIS_LINE_STAGES;  // pipeline stages
constexpr int kStg = 52;  // floats per staged (position, channel group): 3 x 16 + 4

__host__ __device__ inline int line_tiles(int lg) { return lg >= 7 ? 1 << (lg - 7) : 1; }
__host__ __device__ inline int line_tiles1(int lg, int up1) {
  const int T = line_tiles(lg);
  return up1 ? (T > 1 ? T / 2 : 1) : T;
}
// positions (16-byte rows) per chunk plane of a stage: the source rows j-1..j+1 (n >= 128) or
// j0-1 .. j0+R of the R output rows (n < 128), n positions each
__host__ __device__ inline int line_pa(int lg) { return lg >= 7 ? 3 << lg : 128 + (2 << lg); }
__host__ __device__ inline int line_stage_bytes(int lg, int cout) { return 32 * line_pa(lg) + 288 * cout; }
__host__ __device__ inline int line_unit_cols(int lg, int up1, int c2, int cout) {
  return 3 * cout * (line_tiles1(lg, up1) + (c2 > 0 ? line_tiles(lg) : 0));
}
__host__ __device__ inline int line_nbuf(int lg, int up1, int c2, int cout) {
  return 2 * line_unit_cols(lg, up1, c2, cout) <= 512 ? 2 : 1;
}
__host__ __device__ inline int line_stg_bytes(int lg, int up1, int c2) {
  return 128 * (line_tiles1(lg, up1) + (c2 > 0 ? line_tiles(lg) : 0)) * kStg * 4;
}
__host__ __device__ inline int line_smem_n(int lg, int up1, int c2, int cout, int nls) {
  return 1024 + nls * line_stage_bytes(lg, cout) + line_stg_bytes(lg, up1, c2);
}
// the most pipeline stages (2..kLS) whose shared memory fits 220 KB; 0 if none
__host__ __device__ inline int line_nls(int lg, int up1, int c2, int cout) {
  for (int k = kLS; k >= 2; --k)
    if (line_smem_n(lg, up1, c2, cout, k) <= 220 * 1024) return k;
  return 0;
}

// Bulk asynchronous copy of `bytes` (a multiple of 16, both addresses 16-byte
// aligned) from global to shared memory, completing on the mbarrier's tx count.
__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
               "l"(src), "r"(bytes), "r"(bar)
               : "memory");
}
__device__ __forceinline__ void mbar_init_n(uint64_t* bar, int n) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(su32(bar)), "r"(n) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(su32(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(su32(bar)) : "memory");
}

__global__ void __launch_bounds__(192, 1) line_conv(const __grid_constant__ LineArgs a) {
  extern __shared__ unsigned char smem_raw[];
  __shared__ __align__(8) uint64_t full[kLS], empty[kLS], accf[2], acce[2];
  __shared__ uint32_t tmem_slot;
  __shared__ volatile int s_err, s_stop;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int lg = a.lg, n = 1 << lg, msk = n - 1;
  const int T = line_tiles(lg), R = lg >= 7 ? 1 : 128 >> lg, P = R * n;
  const int T1 = line_tiles1(lg, a.up1);
  const int cout = a.cout, N3 = 3 * cout;
  const int S1 = a.c1 / 16, S2 = a.c2 / 16;
  const int upp = n / R;  // units per plane
  const int PA = line_pa(lg), a_bytes = 32 * PA, stage_bytes = a_bytes + 288 * cout;
  const uint32_t ucols = (uint32_t)line_unit_cols(lg, a.up1, a.c2, cout);
  const int nbuf = line_nbuf(lg, a.up1, a.c2, cout);
  const uint32_t ncols = tmem_cols(nbuf * ucols);
  const uint32_t col2 = (uint32_t)(T1 * N3);
  // A: position p of chunk plane c at c * LBOA + p * 16 (source row slot q at positions q n);
  // B: block dj (of 3), row dk * cout + o of chunk c at dj * 96 cout + c * LBOB + row * 16
  const uint32_t LBOA = 16u * PA, LBOB = 16u * N3;
  // 1024-byte aligned base for the swizzled stages, then the epilogue staging
  const uint32_t sraw = su32(smem_raw), sbase = (sraw + 1023u) & ~1023u;
  float* stg = reinterpret_cast<float*>(smem_raw + (sbase - sraw) + a.nls * stage_bytes);
  const int nit = (a.nunits - (int)blockIdx.x + (int)gridDim.x - 1) / (int)gridDim.x;  // units of this CTA
  const int nls = a.nls;  // pipeline stages in use (<= kLS)

  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(&tmem_slot)),
                 "r"(ncols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 0) {
    for (int s = 0; s < kLS; ++s) {  // all kLS barriers initialised; nls in use
      mbar_init_n(&full[s], 1);
      mbar_init_n(&empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init_n(&accf[b], 1);
      mbar_init_n(&acce[b], 128);
    }
    s_err = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_slot;

  if (warp == 0) {
    // ---------------- producer ----------------
    // A stage is (source, 16-channel slice, di): the source rows of the three lines dj = -1, 0, 1
    // of both 8-channel planes (consecutive grid rows are contiguous: one copy per plane, two at
    // the periodic wrap) and the packed weights of the three lines (one copy).
    if (lane == 0) {
      int slot = 0, round = 0, g = 0;  // g = round * nls + slot
      for (int it = 0; it < nit && !s_err; ++it) {
        const int u = blockIdx.x + it * gridDim.x;
        const int pi = u / upp, j0 = (u % upp) * R;
        for (int src = 0; src < (S2 ? 2 : 1) && !s_err; ++src) {
          const bool up = src == 0 && a.up1;
          const int lgs = up ? lg - 1 : lg, nc = 1 << lgs, mc = nc - 1;
          const size_t Vs = (size_t)1 << (3 * lgs);
          const uint32_t rb = (uint32_t)nc * 16u;  // bytes of one source row of one plane
          const uint32_t tx = 2u * rb * (uint32_t)(lg >= 7 ? (up ? 2 : 3) : R + 2) + 288u * (uint32_t)cout;
          const int ns = 3 * (src ? S2 : S1), rot = (int)(blockIdx.x % (unsigned)ns);
          const bf16* wsrc = a.wl + (size_t)(src ? 9 * S1 : 0) * 48 * cout;
          for (int q = 0; q < ns; ++q) {
            // per-CTA rotation of the stage order: concurrent CTAs read different weight blocks
            int qr = q + rot;
            if (qr >= ns) qr -= ns;
            const int slice = qr / 3, di = qr - 3 * slice - 1;
            if (g >= nls && !mbar_wait_spin(&empty[slot], (round - 1) & 1)) {
              s_err = 1;
              break;
            }
            const int ri = ((pi + di) & msk) >> (up ? 1 : 0);
            const bf16* p0 = (src ? a.s2 : a.s1) + (size_t)slice * 16 * Vs + ((size_t)ri << (2 * lgs + 3));
            const size_t p1 = 8 * Vs;  // plane 1 - plane 0
            const uint32_t sa = sbase + slot * stage_bytes, fb = su32(&full[slot]);
            mbar_expect_tx(&full[slot], tx);
            // rows [r0, r0 + cnt) of the source grid plane to positions [pos, pos + cnt nc)
            auto rows = [&](int r0, int cnt, int pos) {
              const bf16* g0 = p0 + ((size_t)r0 << (lgs + 3));
              bulk_g2s(sa + (uint32_t)pos * 16u, g0, rb * (uint32_t)cnt, fb);
              bulk_g2s(sa + LBOA + (uint32_t)pos * 16u, g0 + p1, rb * (uint32_t)cnt, fb);
            };
            if (lg >= 7) {
              const int j = j0;
              if (!up) {  // fine rows j-1, j, j+1 to slots 0, 1, 2
                if (j >= 1 && j <= n - 2) {
                  rows(j - 1, 3, 0);
                } else if (j == 0) {
                  rows(n - 1, 1, 0);
                  rows(0, 2, n);
                } else {
                  rows(n - 2, 2, 0);
                  rows(0, 1, 2 * n);
                }
              } else {  // the two coarse rows under j-1 .. j+1, to slots 0 and 1 (nc positions each)
                const int clo = ((j - 1) & msk) >> 1, chi = ((j + 1) & msk) >> 1;
                if (chi == clo + 1) {
                  rows(clo, 2, 0);
                } else {
                  rows(clo, 1, 0);
                  rows(chi, 1, nc);
                }
              }
            } else if (!up) {  // fine rows j0-1 .. j0+R to slots 0 .. R+1
              if (j0 >= 1 && j0 + R <= n - 1) {
                rows(j0 - 1, R + 2, 0);
              } else if (j0 == 0) {
                rows(n - 1, 1, 0);
                rows(0, R + 1, n);
              } else {
                rows(j0 - 1, R + 1, 0);
                rows(0, 1, (R + 1) * n);
              }
            } else {  // slot q holds the coarse row under fine row j0-1+q
              for (int qq = 0; qq < R + 2; ++qq) rows(((j0 - 1 + qq) & msk) >> 1 & mc, 1, qq * n);
            }
            bulk_g2s(sa + a_bytes, wsrc + (size_t)(9 * slice + 3 * (di + 1)) * 48 * cout, 288u * (uint32_t)cout, fb);
            ++g;
            if (++slot == nls) {
              slot = 0;
              ++round;
            }
          }
        }
      }
      // drain: the copies of the last stages land before this CTA may exit
      for (int h = (g > nls ? g - nls : 0); h < g; ++h)
        if (!mbar_wait_spin(&full[h % nls], (h / nls) & 1)) s_err = 1;
    }
  } else if (warp == 1) {
    // ---------------- MMA issuer ----------------
    if (lane == 0) {
      const uint32_t idesc = idesc_bf16(128, N3, 0, 0);
      // descriptors of slot 0; a slot or tile offset adds (bytes >> 4) to the start-address field
      const uint64_t a0 = sdesc(sbase, LBOA, 128), b0 = sdesc(sbase + a_bytes, LBOB, 128);
      int slot = 0, round = 0;
      bool issued = false;
      int last_slot = 0, last_round = 0;
      for (int it = 0; it < nit && !s_err; ++it) {
        const int buf = it % nbuf;
        if (it >= nbuf && !mbar_wait_spin(&acce[buf], ((it / nbuf) - 1) & 1)) {
          s_err = 1;
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t dbase = tmem + (uint32_t)buf * ucols;
        const int j = (blockIdx.x + it * (int)gridDim.x) % upp * R;  // the unit's (first) row
        for (int src = 0; src < (S2 ? 2 : 1) && !s_err; ++src) {
          const bool up = src == 0 && a.up1;
          const int Ts = src ? T : T1, ns = 3 * (src ? S2 : S1), nc = up ? n / 2 : n;
          const uint32_t d0 = dbase + (src ? col2 : 0u);
          const int clo = ((j - 1) & msk) >> 1;
          for (int q = 0; q < ns; ++q) {
            if (!mbar_wait_spin(&full[slot], round & 1)) {
              s_err = 1;
              break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint64_t so = (uint64_t)((slot * stage_bytes) >> 4);
            for (int dji = 0; dji < 3; ++dji) {
              // position of line dj's first source row in the stage
              int pos = dji * n;
              if (lg >= 7 && up) pos = (((((j + dji - 1) & msk) >> 1) == clo) ? 0 : 1) * nc;
              const uint64_t bd = b0 + so + (uint64_t)(dji * 6 * cout);  // 96 cout bytes per line
              for (int t = 0; t < Ts; ++t)
                mma_bf16(d0 + (uint32_t)(t * N3), a0 + so + (uint64_t)(pos + t * 128), bd, idesc,
                         (q == 0 && dji == 0) ? 0u : 1u);
            }
            mma_commit(&empty[slot]);
            issued = true;
            last_slot = slot;
            last_round = round;
            if (++slot == nls) {
              slot = 0;
              ++round;
            }
          }
        }
        if (s_err) break;
        mma_commit(&accf[buf]);
      }
      // drain: the last MMAs complete before TMEM is released
      if (issued && !mbar_wait_spin(&empty[last_slot], last_round & 1)) s_err = 1;
    }
  } else {
    // ---------------- epilogue (warps 2..5) ----------------
    const int ew = warp & 3;  // TMEM lane quarter of this warp
    const int et = tid - 64;  // 0..127
    const int off2 = 128 * T1 * kStg;
    const size_t Vout = (size_t)1 << (3 * lg);
    for (int it = 0; it < nit; ++it) {
      const int u = blockIdx.x + it * gridDim.x;
      const int pi = u / upp, j0 = (u % upp) * R;
      const int buf = it % nbuf;
      const bool ok = !s_err && mbar_wait_spin(&accf[buf], (it / nbuf) & 1);
      if (!ok) s_err = 1;
      // one snapshot of the flag, so all four warps stop at the same unit
      asm volatile("bar.sync 1, 128;" ::: "memory");
      if (et == 0) s_stop = s_err;
      asm volatile("bar.sync 1, 128;" ::: "memory");
      if (s_stop) break;
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t dbase = tmem + (uint32_t)buf * ucols + ((uint32_t)(ew * 32) << 16);
      for (int g = 0; g < cout / 16; ++g) {
        for (int src = 0; src < (S2 ? 2 : 1); ++src) {
          const int Ts = src ? T : T1;
          for (int t = 0; t < Ts; ++t)
            for (int dki = 0; dki < 3; ++dki) {
              float v[16];
              tmem_ld16(dbase + (src ? col2 : 0u) + (uint32_t)(t * N3 + dki * cout + g * 16), v);
              float4* d = reinterpret_cast<float4*>(stg + (src ? off2 : 0) + (t * 128 + ew * 32 + lane) * kStg +
                                                    dki * 16);
#pragma unroll
              for (int q = 0; q < 4; ++q) d[q] = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
            }
        }
        if (g == cout / 16 - 1) {  // TMEM of this unit fully read
          asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
          mbar_arrive(&acce[buf]);
        }
        asm volatile("bar.sync 1, 128;" ::: "memory");
        float bb[16];
#pragma unroll
        for (int j = 0; j < 16; ++j) bb[j] = a.bias[g * 16 + j];
        for (int p = et; p < P; p += 128) {
          const int r = p >> lg, k = p & msk;
          float acc[16];
#pragma unroll
          for (int j = 0; j < 16; ++j) acc[j] = bb[j];
#pragma unroll
          for (int dki = 0; dki < 3; ++dki) {
            const int kk = (k + dki - 1) & msk;
            const float4* s1p =
                reinterpret_cast<const float4*>(stg + (r * n + (a.up1 ? kk >> 1 : kk)) * kStg + dki * 16);
#pragma unroll
            for (int q = 0; q < 4; ++q) {
              const float4 x = s1p[q];
              acc[4 * q] += x.x;
              acc[4 * q + 1] += x.y;
              acc[4 * q + 2] += x.z;
              acc[4 * q + 3] += x.w;
            }
            if (S2) {
              const float4* s2p = reinterpret_cast<const float4*>(stg + off2 + (r * n + kk) * kStg + dki * 16);
#pragma unroll
              for (int q = 0; q < 4; ++q) {
                const float4 x = s2p[q];
                acc[4 * q] += x.x;
                acc[4 * q + 1] += x.y;
                acc[4 * q + 2] += x.z;
                acc[4 * q + 3] += x.w;
              }
            }
          }
          __align__(16) bf16 o[16];
#pragma unroll
          for (int j = 0; j < 16; ++j) o[j] = __float2bfloat16(a.relu ? fmaxf(acc[j], 0.f) : acc[j]);
          const size_t v = (((size_t)pi << lg | (size_t)(j0 + r)) << lg) | (size_t)k;
          *reinterpret_cast<uint4*>(a.out + pidx(v, g * 16, Vout)) = reinterpret_cast<const uint4*>(o)[0];
          *reinterpret_cast<uint4*>(a.out + pidx(v, g * 16 + 8, Vout)) = reinterpret_cast<const uint4*>(o)[1];
        }
        asm volatile("bar.sync 1, 128;" ::: "memory");
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (tid == 0 && s_err) atomicOr(a.err, 1);
  if (warp == 1) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(ncols));
}

// Weights packed per line-convolution stage s (slice s / 9 of the concatenated
// input channels, line s % 9 = (di + 1) * 3 + (dj + 1)), K-major no-swizzle:
//   wl[s][c][dk * cout + o][e] = W[3 (s % 9) + dk][o][16 (s / 9) + 8 c + e].
__global__ void pack_w(const bf16* __restrict__ w, int cout, int cin, bf16* __restrict__ wl) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;  // one 16-byte row
  const int N3 = 3 * cout, nrow = 9 * (cin / 16) * 2 * N3;
  if (t >= nrow) return;
  const int nn = t % N3, c = (t / N3) & 1, s = t / (2 * N3);
  const int dk = nn / cout, o = nn % cout;
  const int tap = 3 * (s % 9) + dk, ch = 16 * (s / 9) + 8 * c;
  *reinterpret_cast<uint4*>(wl + (size_t)t * 8) = *reinterpret_cast<const uint4*>(w + ((size_t)tap * cout + o) * cin + ch);
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
  __align__(16) bf16 o[8];
#pragma unroll
  for (int c = 0; c < 8; ++c) o[c] = __float2bfloat16(0.f);
  *reinterpret_cast<uint4*>(x + pidx(v, 8, (size_t)V)) = reinterpret_cast<const uint4*>(o)[0];
  o[0] = f0;
  o[1] = f1;
  *reinterpret_cast<uint4*>(x + pidx(v, 0, (size_t)V)) = reinterpret_cast<const uint4*>(o)[0];
}

// Mean over the 8 children (lg: coarse grid).
__global__ void pool_fwd(const bf16* __restrict__ x, int C, int lg, bf16* __restrict__ y) {
  const size_t Vc = (size_t)1 << (3 * lg), Vf = Vc << 3;
  const int m = (1 << lg) - 1, lgf = lg + 1;
  const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;  // element of y in memory order
  if (t >= Vc * C) return;
  const size_t pl = t / (Vc * 8);
  const int u = (int)((t >> 3) % Vc), e = (int)(t & 7);
  const int I = u >> (2 * lg), J = (u >> lg) & m, K = u & m;
  float s = 0.f;
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    const int f = (((2 * I + (q >> 2)) << lgf | (2 * J + ((q >> 1) & 1))) << lgf) | (2 * K + (q & 1));
    s += __bfloat162float(x[((pl * Vf + f) << 3) | e]);
  }
  y[t] = __float2bfloat16(0.125f * s);
}

// dX[fine] += dY[parent] / 8 (lg: coarse grid).
__global__ void pool_bwd(const float* __restrict__ dy, int C, int lg, float* __restrict__ dx) {
  const int lgf = lg + 1, mf = (1 << lgf) - 1;
  const size_t Vf = (size_t)1 << (3 * lgf), Vc = Vf >> 3;
  const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= Vf * C) return;
  const size_t pl = t / (Vf * 8);
  const int f = (int)((t >> 3) % Vf), e = (int)(t & 7);
  const int i = f >> (2 * lgf), j = (f >> lgf) & mf, k = f & mf;
  const int u = (((i >> 1) << lg | (j >> 1)) << lg) | (k >> 1);
  dx[t] += 0.125f * dy[((pl * Vc + u) << 3) | e];
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
  const size_t V = (size_t)1 << (3 * lg);
  const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  // channel-planar: the planes of src1's channels come first, then those of src2
  if (up) {
    const int lgc = lg - 1, mc = (1 << lgc) - 1;
    const size_t Vc = V >> 3;
    if (t < Vc * c1) {
      const size_t pl = t / (Vc * 8);
      const int u = (int)((t >> 3) % Vc), e = (int)(t & 7);
      const int I = u >> (2 * lgc), J = (u >> lgc) & mc, K = u & mc;
      float s = 0.f;
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const int f = (((2 * I + (q >> 2)) << lg | (2 * J + ((q >> 1) & 1))) << lg) | (2 * K + (q & 1));
        s += dx[((pl * V + f) << 3) | e];
      }
      d1[t] = s;
    }
  } else if (t < V * c1) {
    d1[t] = dx[t];
  }
  if (c2 > 0 && t < V * c2) d2[t] += dx[V * c1 + t];
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
    for (int c = 0; c < C; ++c) p += hb[c] * __bfloat162float(y[pidx(v, c, (size_t)V)]);
    if (pred) pred[v] = p;
    if (target) {
      const float r = p - tscale * target[v];
      const float g = 2.f * r / (float)V;
      atomicAdd(&sl, (double)r * r / V);
      if (dy)
        for (int c = 0; c < C; ++c) {
          dy[pidx(v, c, (size_t)V)] = g * hb[c];
          atomicAdd(&sdh[c], g * __bfloat162float(y[pidx(v, c, (size_t)V)]));
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
  const size_t n = (size_t)V * C;
  for (size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (size_t)gridDim.x * blockDim.x)
    atomicAdd(&s[(int)(t / ((size_t)V * 8)) * 8 + (int)(t & 7)], __bfloat162float(dz[t]));
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

// Features of the mean density over each coarse cell (eta on grid lg + 1, features on grid lg):
// f0 = (ln(mean of the 8 children) - mu) * isd, f1 = afeat.
__global__ void input_pooled(const double* __restrict__ eta, int lg, float mu, float isd, float afeat,
                             __nv_bfloat162* __restrict__ f2) {
  const int V = 1 << (3 * lg), m = (1 << lg) - 1, lgf = lg + 1;
  const int u = blockIdx.x * blockDim.x + threadIdx.x;
  if (u >= V) return;
  const int I = u >> (2 * lg), J = (u >> lg) & m, K = u & m;
  double s = 0.0;
#pragma unroll
  for (int q = 0; q < 8; ++q)
    s += eta[(((2 * I + (q >> 2)) << lgf | (2 * J + ((q >> 1) & 1))) << lgf) | (2 * K + (q & 1))];
  f2[u] = __halves2bfloat162(__float2bfloat16((logf((float)fmax(0.125 * s, 1e-30)) - mu) * isd),
                             __float2bfloat16(afeat));
}

// Guess on the grid lg + 1 from the net's output on grid lg: phi = bg + scale * P(pred), P the
// cell-centred trilinear interpolation (weights 3/4 and 1/4 per axis, periodic).
__global__ void guess_fine(const float* __restrict__ p, int lg, double bg, double scale, double* __restrict__ phi) {
  const int lgf = lg + 1, Vf = 1 << (3 * lgf), mf = (1 << lgf) - 1, m = (1 << lg) - 1;
  const int f = blockIdx.x * blockDim.x + threadIdx.x;
  if (f >= Vf) return;
  const int i = f >> (2 * lgf), j = (f >> lgf) & mf, k = f & mf;
  // coarse neighbours along each axis: the parent and the one on the side of the fine cell
  const int I0 = i >> 1, J0 = j >> 1, K0 = k >> 1;
  const int I1 = (I0 + ((i & 1) ? 1 : -1)) & m, J1 = (J0 + ((j & 1) ? 1 : -1)) & m, K1 = (K0 + ((k & 1) ? 1 : -1)) & m;
  const int Is[2] = {I0, I1}, Js[2] = {J0, J1}, Ks[2] = {K0, K1};
  // FP32 interpolation (the net's output is BF16-accurate); FP64 only for phi = bg + scale s
  const float w[2] = {0.75f, 0.25f};
  float s = 0.f;
#pragma unroll
  for (int a = 0; a < 2; ++a)
#pragma unroll
    for (int b = 0; b < 2; ++b) {
      const float* row = p + ((Is[a] << lg | Js[b]) << lg);
      s += w[a] * w[b] * (0.75f * row[Ks[0]] + 0.25f * row[Ks[1]]);
    }
  phi[f] = bg + scale * (double)s;
}

inline unsigned nb(size_t n, int t) { return (unsigned)((n + t - 1) / t); }

static bool aligned16(const void* p) { return ((uintptr_t)p & 15u) == 0; }

}  // namespace unet
}  // namespace isis

using namespace isis::unet;

#define UNET_LAUNCH(kind, bytes, st, ...) ISIS_LAUNCH(kind, bytes, st, __VA_ARGS__)

static int sm_count() {
  static int n = 0;
  if (!n) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
      n = 0;
  }
  return n;
}

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

isis_status isis_unet_pack_w(const void* w, int cout, int cin, void* wl, void* stream) {
  if (!w || !wl || cout < 16 || cout > 64 || cout % 16 || cin < 16 || cin % 16 || !aligned16(w) || !aligned16(wl))
    return ISIS_EINVAL;
  const int nrow = 9 * (cin / 16) * 6 * cout;
  cudaStream_t st = (cudaStream_t)stream;
  UNET_LAUNCH(isis::KK_UNET_ELEM, 32.0 * nrow, st,
              (pack_w<<<nb(nrow, 256), 256, 0, st>>>((const bf16*)w, cout, cin, (bf16*)wl)));
  return ISIS_OK;
}

int isis_unet_line_ok(int c1, int lg1, int c2, int lg, int cout) {
  const int up1 = lg1 != lg;
  return lg >= 5 && lg <= 9 && (lg1 == lg || lg1 == lg - 1) && c1 >= 16 && c1 % 16 == 0 && c2 >= 0 && c2 % 16 == 0 &&
         cout >= 16 && cout <= 64 && cout % 16 == 0 && line_unit_cols(lg, up1, c2, cout) <= 512 &&
         line_nls(lg, up1, c2, cout) >= 2;
}

isis_status isis_unet_line_fwd(const void* src1, int c1, int lg1, const void* src2, int c2, int lg, const void* wl,
                               const float* bias, int cout, int relu, void* out, int* err, void* stream) {
  if (!src1 || !wl || !bias || !out || !err || (c2 > 0 && !src2) || !isis_unet_line_ok(c1, lg1, c2, lg, cout))
    return ISIS_EINVAL;
  if (!aligned16(src1) || (src2 && !aligned16(src2)) || !aligned16(wl) || !aligned16(out)) return ISIS_EINVAL;
  static bool attr = false;
  if (!attr) {
    if (cudaFuncSetAttribute(line_conv, cudaFuncAttributeMaxDynamicSharedMemorySize, 220 * 1024) != cudaSuccess)
      return ISIS_ECUDA;
    attr = true;
  }
  const int up1 = lg1 != lg, n = 1 << lg, R = lg >= 7 ? 1 : 128 >> lg;
  const size_t V = (size_t)1 << (3 * lg);
  const int nls = line_nls(lg, up1, c2, cout);
  LineArgs la{(const bf16*)src1, (const bf16*)src2, (const bf16*)wl, bias, (bf16*)out, c1, up1, c2, lg, cout, relu,
              (int)(V / (size_t)(R * n)), nls, err};
  const int nsm = sm_count();
  if (nsm <= 0) return ISIS_ECUDA;
  const unsigned grid = (unsigned)(la.nunits < nsm ? la.nunits : nsm);
  cudaStream_t st = (cudaStream_t)stream;
  const double flops = 2.0 * 27.0 * (c1 + c2) * cout * (double)V;
  UNET_LAUNCH(isis::KK_UNET_CONV, flops, st, (line_conv<<<grid, 192, line_smem_n(lg, up1, c2, cout, nls), st>>>(la)));
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

isis_status isis_unet_input_pooled(const double* eta, int lg, float mu, float isd, float afeat, void* f2,
                                   void* stream) {
  if (!eta || !f2 || lg < 2 || lg > 9 || ((uintptr_t)f2 & 3u)) return ISIS_EINVAL;
  const int V = 1 << (3 * lg);
  cudaStream_t st = (cudaStream_t)stream;
  UNET_LAUNCH(isis::KK_UNET_ELEM, 68.0 * V, st,
              (input_pooled<<<nb(V, 256), 256, 0, st>>>(eta, lg, mu, isd, afeat, (__nv_bfloat162*)f2)));
  return ISIS_OK;
}

isis_status isis_unet_guess_fine(const float* pred, int lg, double bg, double scale, double* phi, void* stream) {
  if (!pred || !phi || lg < 2 || lg > 9) return ISIS_EINVAL;
  const int Vf = 1 << (3 * (lg + 1));
  cudaStream_t st = (cudaStream_t)stream;
  UNET_LAUNCH(isis::KK_UNET_ELEM, 8.5 * Vf, st, (guess_fine<<<nb(Vf, 256), 256, 0, st>>>(pred, lg, bg, scale, phi)));
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
