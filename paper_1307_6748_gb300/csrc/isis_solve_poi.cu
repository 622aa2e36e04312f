// isis_solve_poi.cu -- instantiation of the multigrid drivers for one model
// (one translation unit per model so the three compile in parallel).
#include "isis_solver.cuh"

namespace isis {
isis_status run_poi(const SolveArgs& A) {
  switch (A.prec) {
    case ISIS_F64: return solve_field<POI, double>(A);
    case ISIS_F32: return solve_field<POI, float>(A);
    case ISIS_F32_REFINE64: return solve_refine<POI>(A);
  }
  return ISIS_EINVAL;
}
}  // namespace isis
