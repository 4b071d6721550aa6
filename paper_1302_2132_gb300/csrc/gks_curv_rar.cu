// Body-fitted step and steady residual with the rarefaction option (gks_turb.rarefaction =
// GKS_RAR_TAUHAT: the degree of rarefaction tau/tauhat, Eqs. tautautilde, tautilde, epsilonkomega, in
// place of tau over the step or the face window inside the time coefficients): MUSCL-2, FP64 and the
// FP32 float-pair form, both expansions; the time step on the 16 x 11 tile, the residual on the 32 x 15
// tile for large grids and the 16 x 11 tile otherwise (as launch_curv_residual chooses).
#include "gks_curv.h"
#include "gks_curv_step.cuh"

namespace gks {

cudaError_t prepare_curv_rar() {
  const cudaError_t r[12] = {
      prepare_one<PREC_F64, 2, 0, false, 0, false, true>(), prepare_one<PREC_F64, 2, 0, true, 0, false, true>(),
      prepare_one<PREC_F32, 2, 0, false, 0, false, true>(), prepare_one<PREC_F32, 2, 0, true, 0, false, true>(),
      prepare_one<PREC_F64, 0, 1, false, 0, false, true>(), prepare_one<PREC_F64, 0, 1, true, 0, false, true>(),
      prepare_one<PREC_F32, 0, 1, false, 0, false, true>(), prepare_one<PREC_F32, 0, 1, true, 0, false, true>(),
      prepare_one<PREC_F64, 2, 1, false, 0, false, true>(), prepare_one<PREC_F64, 2, 1, true, 0, false, true>(),
      prepare_one<PREC_F32, 2, 1, false, 0, false, true>(), prepare_one<PREC_F32, 2, 1, true, 0, false, true>()};
  for (cudaError_t x : r)
    if (x != cudaSuccess) return x;
  return cudaSuccess;
}

void launch_curv_step_rar(int prec, const StepArgs& A, const CurvGeom& G, bool multid, cudaStream_t s) {
  if (prec == PREC_F64) {
    if (multid) launch_fused<PREC_F64, 2, 0, true, 0, false, true>(A, G, s);
    else launch_fused<PREC_F64, 2, 0, false, 0, false, true>(A, G, s);
  } else {
    if (multid) launch_fused<PREC_F32, 2, 0, true, 0, false, true>(A, G, s);
    else launch_fused<PREC_F32, 2, 0, false, 0, false, true>(A, G, s);
  }
}

void launch_curv_residual_rar(int prec, const StepArgs& A, const CurvGeom& G, const SteadyArgs& SA, cudaStream_t s) {
  const bool big = A.g.ncell >= 300000;
  if (SA.multid) {
    if (prec == PREC_F64)
      big ? launch_fused<PREC_F64, 0, 1, true, 0, false, true>(A, G, s, SA)
          : launch_fused<PREC_F64, 2, 1, true, 0, false, true>(A, G, s, SA);
    else
      big ? launch_fused<PREC_F32, 0, 1, true, 0, false, true>(A, G, s, SA)
          : launch_fused<PREC_F32, 2, 1, true, 0, false, true>(A, G, s, SA);
  } else {
    if (prec == PREC_F64)
      big ? launch_fused<PREC_F64, 0, 1, false, 0, false, true>(A, G, s, SA)
          : launch_fused<PREC_F64, 2, 1, false, 0, false, true>(A, G, s, SA);
    else
      big ? launch_fused<PREC_F32, 0, 1, false, 0, false, true>(A, G, s, SA)
          : launch_fused<PREC_F32, 2, 1, false, 0, false, true>(A, G, s, SA);
  }
}

}  // namespace gks
