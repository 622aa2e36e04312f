// isis_patch.cuh -- refinement patches: the solve of one refinement level over
// a box of its parent grid, with the mask function and ghost values of
// Sect. 3.3.1 (canonical operators) and Sect. 3.4.1 (non-canonical).
//
// A patch is a box of n[0] x n[1] x n[2] parent cells at `origin` in the
// parent grid, refined by two.  Its finest level holds 2n cells per axis (all
// of them: the box is dense), of which the children of flagged parent cells
// are unknowns (mask +1) and the rest do not exist in the paper's sense
// (mask -1): they hold the parent field interpolated to them.  The patch's own
// multigrid levels halve the box and restrict the mask, so coarse cells get
// fractional masks.  Readings of the paper:
//   - mask: m = +1 / -1 on the finest level, m = mean of the 8 children below
//     except on the outer layer of each level, which stays -1; cells with
//     m > 0 are unknowns, the others keep their values;
//   - ghost of a neighbour with m_nb <= 0 of an unknown c (Eq. (ueq)):
//     u_nb + (m_nb/m_c)(u_c - u_c^Pre), u_c^Pre = u_c when the smoothing phase
//     began; residuals take u^Pre = u; f(R) takes b and db/du of the ghost value;
//   - dL/du_c gains the terms through the ghost values (Sect. 3.4.1), with the
//     factor 1/2 of the face mean's derivative;
//   - FAS between the patch levels as on the domain grid (full-approximation
//     restriction of u, residual restricted with zeros off the unknowns,
//     correction added at unknowns only, none from outside the box);
//   - mixed precision (ISIS_F32_REFINE64): the FP64 residual r = -L(u) at
//     the unknowns, then FP32 V-cycles of the same patch FAS on the correction
//     e about B = fp32(u), L(B + e) - L(B) = r (masked neighbours enter as
//     B_nb + e_nb + (m_nb/m_c)(e_c - e_c^Pre)), then u += e, as on the domain;
//   - levels halve while every dimension is even and the smallest is >= 8;
//     the coarsest level gets 16 red/black sweeps in one block;
//   - flags on the box's outer layer of parent cells are rejected, so on every
//     level the unknowns lie inside the outer layer and stencils stay in the box
//     (the kernels also skip the outer layer whatever the mask says).
#pragma once
#include <stdint.h>

#include "isis.h"
#include "isis_model.cuh"

namespace isis {

struct PatchArgs {
  int model;               // POI, SYM, FOFR
  Coef coef;               // model constants (FIELD form, fscale = 1)
  double ref_scale;        // reference residual = ref_scale * RMS over unknowns of (eta - eref)
  double eref;             // 1, or the domain mean for Poisson
  int n[3], origin[3], pn[3], periodic;
  double h;                // finest patch cell size
  const double* parent;    // parent field, pn dims
  const uint8_t* flags;    // n dims
  const double* eta;       // finest patch density, 2n dims
  double* phi;             // finest patch field, 2n dims
  int64_t unknowns;        // 8 * number of flagged cells
  double tol;
  int nu1, nu2, max_cycles;
  int prec;                // ISIS_F64, or ISIS_F32_REFINE64: FP32 correction cycles in FP64 defect correction
  int inner;               // FP32 V-cycles per FP64 outer iteration (ISIS_F32_REFINE64)
  int init_parent;         // 1: unknowns start from the interpolated parent
  isis_solve_info* info;
  cudaStream_t st;
};

isis_status run_patch_poi(const PatchArgs& A);
isis_status run_patch_sym(const PatchArgs& A);
isis_status run_patch_fofr(const PatchArgs& A);

}  // namespace isis
