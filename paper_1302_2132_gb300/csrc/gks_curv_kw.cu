// k-omega transport fused into the body-fitted time step (GKS_TURB_KOMEGA_TRANSPORT on a grid set by
// gks_set_nodes): the fused curvilinear tile step (gks_curv_step.cuh) with the transport of rho k
// and rho omega evaluated on the tile's faces and cells, so that one kernel per time step replaces
// the step and transport kernels.  Instantiated for FP64 and the FP32 float-pair form with MUSCL-2,
// both expansions, on the 32 x 15 (variant 0) and 16 x 11 (variant 2) tiles.
#include "gks_curv.h"
#include "gks_curv_step.cuh"

namespace gks {

namespace {

template <int PREC, bool MD>
void launch_tr(const StepArgs& A, const CurvGeom& G, int variant, cudaStream_t s) {
  if (variant == 0)
    launch_fused<PREC, 0, 0, MD, 0, true>(A, G, s);
  else
    launch_fused<PREC, 2, 0, MD, 0, true>(A, G, s);
}

template <int PREC>
cudaError_t prepare_tr() {
  const cudaError_t r[4] = {prepare_one<PREC, 0, 0, false, 0, true>(), prepare_one<PREC, 0, 0, true, 0, true>(),
                            prepare_one<PREC, 2, 0, false, 0, true>(), prepare_one<PREC, 2, 0, true, 0, true>()};
  for (cudaError_t x : r)
    if (x != cudaSuccess) return x;
  return cudaSuccess;
}

}  // namespace

cudaError_t prepare_curv_transport() {
  const cudaError_t a = prepare_tr<PREC_F64>(), b = prepare_tr<PREC_F32>();
  return a != cudaSuccess ? a : b;
}

void launch_curv_step_transport(int prec, const StepArgs& A, const CurvGeom& G, int variant, bool multid,
                                cudaStream_t s) {
  if (prec == PREC_F64) {
    if (multid)
      launch_tr<PREC_F64, true>(A, G, variant, s);
    else
      launch_tr<PREC_F64, false>(A, G, variant, s);
  } else {
    if (multid)
      launch_tr<PREC_F32, true>(A, G, variant, s);
    else
      launch_tr<PREC_F32, false>(A, G, variant, s);
  }
}

}  // namespace gks
