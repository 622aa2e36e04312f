/*
 * isis_unet.h -- C ABI of the learned initial guess for the scalar-field
 * solve: the kernels of a small 3-D U-Net (convolutions on the tcgen05 tensor
 * cores, BF16 operands, FP32 accumulation) and of its training.
 *
 * The paper (arXiv:1307.6748) has no learned component.  Its solver starts
 * every FAS solve from a guess (Sect. 3.2); here a network trained on
 * converged solutions of isis_scalar_solve proposes that guess, and the
 * multigrid solver always finishes the solve, so the net never changes the
 * answer, only the number of cycles.
 *
 * Conventions
 *   - A grid has n = 2^lg cells per side (2 <= lg <= 10), V = n^3 voxels in
 *     row-major order ((i n + j) n + k), periodic.
 *   - Activations are BF16 with C channels (a multiple of 16), stored
 *     channel-planar in groups of 8: element (v, c) at ((c / 8) V + v) 8 + c % 8,
 *     so that one grid row of one 8-channel group is a contiguous block of
 *     n x 16 bytes.  Gradients of activations are FP32 in the same layout.  All
 *     pointers are device pointers owned by the caller, 16-byte aligned.
 *   - 3x3x3 convolution, tap t = (di+1)*9 + (dj+1)*3 + (dk+1) for the offset
 *     (di, dj, dk) in {-1,0,1}^3, periodic wrap:
 *       out[v][o] = b[o] + sum_t sum_i X[v + d_t][i] W[t][o][i],   W: BF16 [27][cout][cin]
 *     X is the channel concatenation of src1 (c1 channels; on the grid lg1 =
 *     lg, or lg - 1 read by nearest-neighbour upsampling) and src2 (c2
 *     channels on grid lg, or absent with c2 = 0).  cin = c1 + c2.
 *   - err: device int, OR-ed with 1 if a bounded wait inside a kernel gave up.
 *   - Every call is stream ordered and returns ISIS_EINVAL for bad sizes or
 *     pointers, ISIS_ECUDA for a failed launch.
 */
#ifndef ISIS_UNET_H
#define ISIS_UNET_H
#include <stdint.h>

#include "isis.h"

#ifdef __cplusplus
extern "C" {
#endif

/* out (BF16, cout channels) = optional ReLU of the convolution plus bias (FP32 [cout]),
 * any grid; the A operand is gathered per voxel and tap.
 * 16 <= c1, 0 <= c2, c1 + c2 <= 128, 16 <= cout <= 64, all multiples of 16. */
isis_status isis_unet_conv3_fwd(const void* src1, int c1, int lg1, const void* src2, int c2, int lg, const void* w,
                                const float* bias, int cout, int relu, void* out, int* err, void* stream);

/* Weights packed for isis_unet_line_fwd: for stage s (16-channel slice s / 9 of
 * the cin input channels, line s % 9 = (di + 1) * 3 + (dj + 1)),
 *   wl[s][c][dk * cout + o][e] = W[3 (s % 9) + dk][o][16 (s / 9) + 8 c + e],
 * c in {0, 1}, dk in {0, 1, 2}, e < 8; wl has the size of w. */
isis_status isis_unet_pack_w(const void* w, int cout, int cin, void* wl, void* stream);

/* 1 if isis_unet_line_fwd takes these sizes: grids of 32..512 cells per side and
 * the accumulators and shared-memory stages fit one SM. */
int isis_unet_line_ok(int c1, int lg1, int c2, int lg, int cout);

/* The same convolution as isis_unet_conv3_fwd with weights wl packed by
 * isis_unet_pack_w (cin = c1 + c2).  One CTA per SM computes whole grid rows:
 * for each (di, dj) and 16-channel slice, the source rows are bulk-copied once
 * (no per-voxel gather) and one tcgen05 MMA with N = 3 cout applies the three
 * k taps at once; the k shift is applied in the epilogue.  An upsampled src1 is
 * staged at its own resolution.  ISIS_EINVAL where isis_unet_line_ok is 0. */
isis_status isis_unet_line_fwd(const void* src1, int c1, int lg1, const void* src2, int c2, int lg, const void* wl,
                               const float* bias, int cout, int relu, void* out, int* err, void* stream);

/* Input gradient: din (FP32 [V][cin]) = sum_t sum_o dz[v - d_t][o] W[t][o][i],
 * with wt = W transposed per tap (BF16 [27][cin][cout], isis_unet_transpose_w),
 * dz BF16 [V][cout]; cin <= 128. */
isis_status isis_unet_conv3_dgrad(const void* dz, int cout, int lg, const void* wt, int cin, float* din, int* err,
                                  void* stream);

/* Weight gradient: dw[t][o][i] += sum_v dz[v][o] X[v + d_t][i] (FP32, accumulated with
 * atomics, so the summation order is not fixed).  Same src1/src2 convention as the forward. */
isis_status isis_unet_conv3_wgrad(const void* src1, int c1, int lg1, const void* src2, int c2, int lg,
                                  const void* dz, int cout, float* dw, int* err, void* stream);

/* Input features of the net: f0 = (ln eta - mu) * isd and f1 = afeat (a
 * normalised expansion factor), written as x16 (BF16 [V][16]: f0, f1, then 14
 * zero channels) and/or f2 (BF16 [V][2]: f0, f1); either may be NULL, not both. */
isis_status isis_unet_input(const double* eta, int lg, float mu, float isd, float afeat, void* x16, void* f2,
                            void* stream);

/* First layer from the two features f2 (BF16 [V][2]): out (BF16 [V][16]) =
 * ReLU(bias + sum_t f0(v + d_t) W[t][o][0] + f1(v + d_t) W[t][o][1]), with
 * W BF16 [27][16][wcin] (wcin >= 2, a multiple of 8; channels >= 2 unused).
 * Equal to isis_unet_conv3_fwd of x16 (relu = 1) up to the FP32 summation order. */
isis_status isis_unet_stem_fwd(const void* f2, int lg, const void* w, int wcin, const float* bias, void* out,
                               int* err, void* stream);

/* y (grid lgc) = mean of the 8 children of x (grid lgc + 1), BF16, C channels. */
isis_status isis_unet_pool_fwd(const void* x, int C, int lgc, void* y, void* stream);
/* dx (grid lgc + 1, FP32) += dy (grid lgc) / 8, broadcast to the 8 children. */
isis_status isis_unet_pool_bwd(const float* dy, int C, int lgc, float* dx, void* stream);
/* dz (BF16) = dy where y > 0, else 0 (gradient through a ReLU whose output is y). */
isis_status isis_unet_relu_bwd(const float* dy, const void* y, int64_t n, void* dz, void* stream);
/* Split the FP32 gradient dx [V][c1+c2] of a concatenated input on grid lg:
 * d1 = channels [0, c1) (summed over the 8 fine voxels of each half-resolution
 * cell when up != 0), d2 += channels [c1, c1+c2). */
isis_status isis_unet_split_bwd(const float* dx, int c1, int c2, int lg, int up, float* d1, float* d2,
                                void* stream);
/* Output head and loss: p[v] = hb[C] + sum_c hb[c] y[v][c] (into pred if not NULL);
 * if target is not NULL: loss += mean (p - tscale target)^2, dy = d loss / d y,
 * dhb += d loss / d hb.  hb: FP32 [C + 1] (weights, then bias). */
isis_status isis_unet_head(const void* y, int C, int lg, const float* hb, const float* target, float tscale,
                           float* pred, float* dy, float* dhb, double* loss, void* stream);
/* db[o] += sum_v dz[v][o]. */
isis_status isis_unet_bias_grad(const void* dz, int C, int lg, float* db, void* stream);
/* Adam (Kingma & Ba) on FP32 parameters p with gradient g and moments m1, m2,
 * step number step >= 1; writes the BF16 copy pbf16 if not NULL. */
isis_status isis_unet_adam(float* p, const float* g, float* m1, float* m2, int64_t n, float lr, float b1, float b2,
                           float eps, int step, void* pbf16, void* stream);
/* wt[t][i][o] = w[t][o][i] (BF16). */
isis_status isis_unet_transpose_w(const void* w, int cout, int cin, void* wt, void* stream);
/* b = BF16(a). */
isis_status isis_unet_to_bf16(const float* a, int64_t n, void* b, void* stream);
/* Features of a grid twice as fine as the net's (eta on grid lg + 1): f2 (BF16 [V][2]) on
 * grid lg from the mean density of each 8-cell block: f0 = (ln mean - mu) * isd, f1 = afeat.
 * The net then runs at its training cell size; 2 <= lg <= 9. */
isis_status isis_unet_input_pooled(const double* eta, int lg, float mu, float isd, float afeat, void* f2,
                                   void* stream);
/* phi (FP64, grid lg + 1) = bg + scale * P(pred), with pred on grid lg and P the cell-centred
 * trilinear prolongation (per axis: 3/4 of the parent, 1/4 of the neighbour on the fine cell's
 * side, periodic). */
isis_status isis_unet_guess_fine(const float* pred, int lg, double bg, double scale, double* phi, void* stream);
/* phi[v] = bg + scale * pred[v] (FP64 initial guess for isis_scalar_solve). */
isis_status isis_unet_guess(const float* pred, int lg, double bg, double scale, double* phi, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* ISIS_UNET_H */
