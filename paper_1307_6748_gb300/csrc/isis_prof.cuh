// isis_prof.cuh -- launch counting and optional per-launch CUDA-event timing.
// Every kernel launch of the library goes through ISIS_LAUNCH, which counts
// it and, when profiling is enabled, brackets it with events on its stream
// and records its algorithmic bytes under a kernel kind.
#pragma once
#include <cuda_runtime.h>

namespace isis {

enum KernelKind : int {
  KK_SMOOTH_FINE = 0,   // smoother on the finest grid
  KK_SMOOTH_COARSE,     // smoother on the coarser grids
  KK_RESTRICT_FINE,     // residual + restriction from the finest grid
  KK_RESTRICT_COARSE,
  KK_SIGMA,             // coarse FAS source
  KK_PROLONG_FINE,      // prolongation onto the finest grid
  KK_PROLONG_COARSE,
  KK_COARSE_NEWTON,
  KK_NORM,              // residual norm of the finest grid
  KK_OUTER_RESID,       // FP64 residual of the defect-correction loop
  KK_UPDATE,            // FP64 solution update
  KK_SETUP,             // density / base restriction, conversions, e^B
  KK_REDUCE,            // final reductions, moments, mean removal
  KK_INIT,              // initial guess
  KK_CIC_SCATTER,
  KK_CIC_FINISH,
  KK_FORCE_GRID,
  KK_FORCE,
  KK_UNET_CONV,         // tcgen05 convolutions of the learned guess (bytes field: FLOPs)
  KK_UNET_ELEM,         // its element-wise kernels
  KK_PATCH_SMOOTH,      // smoother on a refinement patch
  KK_PATCH_OTHER,       // the patch's residual, transfers, interpolation and norms
  KK_PATCH_COARSEST,    // the relaxation of a patch's coarsest level (one block)
  KK_COARSE_CYCLE,      // the levels of a V-cycle from 16^3 down, in one block
  KK_COUNT
};

// A launch of the multigrid kernels also records the instantiation it runs: the recorded kind is
// kind + KK_COUNT * tag with tag = 1 + 2 * model + form (model 0 Poisson, 1 symmetron, 2 f(R) and the
// chameleon; form 0 field, 1 correction), tag 0 for the other kernels.
constexpr int kKindTags = 7;
constexpr int kind_tag(int kind, int model, int form) { return kind + KK_COUNT * (1 + 2 * model + form); }

void prof_pre(cudaStream_t st);
void prof_post(int kind, double bytes, cudaStream_t st);
// Whether per-launch events are on; the launches counted so far; count n launches run through a CUDA graph
// (n < 0 takes back the count of launches recorded into one while it was captured).
bool prof_enabled();
long long prof_launches();
void prof_add_launches(long long n);

}  // namespace isis

// Launch a kernel through the profiler; returns ISIS_ECUDA from the
// enclosing function if the launch fails.
#define ISIS_LAUNCH(kind, bytes, st, ...)        \
  do {                                           \
    ::isis::prof_pre(st);                        \
    __VA_ARGS__;                                 \
    cudaError_t le_ = cudaGetLastError();        \
    ::isis::prof_post((kind), (bytes), (st));    \
    if (le_ != cudaSuccess) return ISIS_ECUDA;   \
  } while (0)
