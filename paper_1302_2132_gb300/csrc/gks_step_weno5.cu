// The step kernel with fifth-order WENO face reconstruction (default tile of each dimension and the 32 x 27
// tile in 2D; FP64 and the FP32 float-pair form).
#include "gks_dispatch.h"
#include "gks_step.cuh"

namespace gks {

cudaError_t prepare_step_weno5() {
  cudaError_t e = cudaSuccess, r;
#define GKS_PREP(D, P, M) if ((r = prepare_step<D, P, M, 0, RECON_WENO5>()) != cudaSuccess) e = r;
  GKS_PREP(1, PREC_F64, false)
  GKS_PREP(1, PREC_F32, false)
  GKS_PREP(2, PREC_F64, false)
  GKS_PREP(2, PREC_F32, false)
  GKS_PREP(2, PREC_F64, true)
  GKS_PREP(2, PREC_F32, true)
  GKS_PREP(3, PREC_F64, true)
  GKS_PREP(3, PREC_F32, true)
#undef GKS_PREP
  if ((r = prepare_step<2, PREC_F32, true, 3, RECON_WENO5>()) != cudaSuccess) e = r;
  return e;
}

bool launch_step_weno5(int D, int prec, bool multid, int variant, const StepArgs& A, int nblocks, cudaStream_t s) {
  if (prec == PREC_F32D || (D == 3 && !multid) || (D == 1 && multid)) return false;
  if (variant == 3) {  // 32 x 27 tile, 2D FP32 multi-D
    if (D != 2 || prec != PREC_F32 || !multid) return false;
    launch_step<2, PREC_F32, true, 3, RECON_WENO5>(A, nblocks, s);
    return true;
  }
  const bool f64 = prec == PREC_F64;
  if (D == 1) {
    if (f64) launch_step<1, PREC_F64, false, 0, RECON_WENO5>(A, nblocks, s);
    else launch_step<1, PREC_F32, false, 0, RECON_WENO5>(A, nblocks, s);
  } else if (D == 2) {
    if (multid) {
      if (f64) launch_step<2, PREC_F64, true, 0, RECON_WENO5>(A, nblocks, s);
      else launch_step<2, PREC_F32, true, 0, RECON_WENO5>(A, nblocks, s);
    } else {
      if (f64) launch_step<2, PREC_F64, false, 0, RECON_WENO5>(A, nblocks, s);
      else launch_step<2, PREC_F32, false, 0, RECON_WENO5>(A, nblocks, s);
    }
  } else {
    if (f64) launch_step<3, PREC_F64, true, 0, RECON_WENO5>(A, nblocks, s);
    else launch_step<3, PREC_F32, true, 0, RECON_WENO5>(A, nblocks, s);
  }
  return true;
}

}  // namespace gks
