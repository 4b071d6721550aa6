// MUSCL-3 and WENO-5 on body-fitted 2D grids (Section 4 lists both beside the second-order MUSCL):
// the fused curvilinear tile step (gks_curv_step.cuh) with the face reconstruction in index space
// along each grid line on the states rotated into the face frame, three halo layers for WENO-5's
// six-cell stencil.  Instantiated for FP64 and the FP32 float-pair form, both expansions, on the
// 32 x 15 tile (variant 0) and the 16 x 11 tile (variant 2), for the time step and for the steady
// solver's fine-level residual.
#include "gks_curv.h"
#include "gks_curv_step.cuh"

namespace gks {

namespace {

template <int PREC, int RC, bool MD>
void launch_rc(const StepArgs& A, const CurvGeom& G, int variant, cudaStream_t s) {
  if (variant == 0)
    launch_fused<PREC, 0, 0, MD, RC>(A, G, s);
  else
    launch_fused<PREC, 2, 0, MD, RC>(A, G, s);
}

template <int PREC, int RC>
void launch_md(const StepArgs& A, const CurvGeom& G, int variant, bool md, cudaStream_t s) {
  if (md)
    launch_rc<PREC, RC, true>(A, G, variant, s);
  else
    launch_rc<PREC, RC, false>(A, G, variant, s);
}

// the steady residual (MODE 1): 32 x 15 tiles on grids of two or more waves of them, 16 x 11 tiles
// below (as the MUSCL-2 residual)
template <int PREC, int RC, bool MD>
void residual_rc(const StepArgs& A, const CurvGeom& G, const SteadyArgs& SA, cudaStream_t s) {
  if (A.g.ncell >= 300000)
    launch_fused<PREC, 0, 1, MD, RC>(A, G, s, SA);
  else
    launch_fused<PREC, 2, 1, MD, RC>(A, G, s, SA);
}

template <int PREC, int RC>
void residual_md(const StepArgs& A, const CurvGeom& G, const SteadyArgs& SA, cudaStream_t s) {
  if (SA.multid)
    residual_rc<PREC, RC, true>(A, G, SA, s);
  else
    residual_rc<PREC, RC, false>(A, G, SA, s);
}

template <int PREC, int RC>
cudaError_t prepare_rc() {
  const cudaError_t r[8] = {prepare_one<PREC, 0, 0, false, RC>(), prepare_one<PREC, 0, 0, true, RC>(),
                            prepare_one<PREC, 2, 0, false, RC>(), prepare_one<PREC, 2, 0, true, RC>(),
                            prepare_one<PREC, 0, 1, false, RC>(), prepare_one<PREC, 0, 1, true, RC>(),
                            prepare_one<PREC, 2, 1, false, RC>(), prepare_one<PREC, 2, 1, true, RC>()};
  for (cudaError_t x : r)
    if (x != cudaSuccess) return x;
  return cudaSuccess;
}

}  // namespace

cudaError_t prepare_curv_recon() {
  const cudaError_t r[4] = {prepare_rc<PREC_F64, 1>(), prepare_rc<PREC_F64, 2>(), prepare_rc<PREC_F32, 1>(),
                            prepare_rc<PREC_F32, 2>()};
  for (cudaError_t x : r)
    if (x != cudaSuccess) return x;
  return cudaSuccess;
}

void launch_curv_residual_recon(int prec, const StepArgs& A, const CurvGeom& G, const SteadyArgs& SA, cudaStream_t s) {
  if (prec == PREC_F64) {
    if (SA.recon == 2)
      residual_md<PREC_F64, 2>(A, G, SA, s);
    else
      residual_md<PREC_F64, 1>(A, G, SA, s);
  } else {
    if (SA.recon == 2)
      residual_md<PREC_F32, 2>(A, G, SA, s);
    else
      residual_md<PREC_F32, 1>(A, G, SA, s);
  }
}

void launch_curv_step_recon(int prec, int recon, const StepArgs& A, const CurvGeom& G, int variant, bool multid,
                            cudaStream_t s) {
  if (prec == PREC_F64) {
    if (recon == 2)
      launch_md<PREC_F64, 2>(A, G, variant, multid, s);
    else
      launch_md<PREC_F64, 1>(A, G, variant, multid, s);
  } else {
    if (recon == 2)
      launch_md<PREC_F32, 2>(A, G, variant, multid, s);
    else
      launch_md<PREC_F32, 1>(A, G, variant, multid, s);
  }
}

}  // namespace gks
