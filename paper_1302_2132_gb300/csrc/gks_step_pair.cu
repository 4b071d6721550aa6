// Paired tiles of the step kernel (2D variants 6: 32x27 on 128 threads, 7: 64x27 on 256 threads; 3D
// variant 3: 16x8x2 on 128 threads) in the FP32 forms (float-pair and double state): each thread
// evaluates two faces at once with the paired FP32 instructions.  Chosen at run time by the
// autotuner.
#include "gks_dispatch.h"
#include "gks_step.cuh"

namespace gks {

cudaError_t prepare_step_pair() {
  cudaError_t e = cudaSuccess, r;
#define GKS_PREP(P, M, V) if ((r = prepare_step<2, P, M, V>()) != cudaSuccess) e = r;
  GKS_PREP(PREC_F32, false, 6) GKS_PREP(PREC_F32, true, 6) GKS_PREP(PREC_F32, false, 7) GKS_PREP(PREC_F32, true, 7)
  GKS_PREP(PREC_F32D, false, 6) GKS_PREP(PREC_F32D, true, 6) GKS_PREP(PREC_F32D, false, 7)
  GKS_PREP(PREC_F32D, true, 7)
#undef GKS_PREP
  if ((r = prepare_step<3, PREC_F32, true, 3>()) != cudaSuccess) e = r;
  if ((r = prepare_step<3, PREC_F32, false, 3>()) != cudaSuccess) e = r;
  if ((r = prepare_step<3, PREC_F32D, true, 3>()) != cudaSuccess) e = r;
  if ((r = prepare_step<3, PREC_F32D, false, 3>()) != cudaSuccess) e = r;
  return e;
}

template <int P, int V>
void launch_pair(bool multid, const StepArgs& A, int nblocks, cudaStream_t s) {
  if (multid) launch_step<2, P, true, V>(A, nblocks, s);
  else launch_step<2, P, false, V>(A, nblocks, s);
}

void launch_step_pair(int D, int prec, int variant, bool multid, const StepArgs& A, int nblocks, cudaStream_t s) {
  if (D == 3) {
    if (prec == PREC_F32D) {
      if (multid) launch_step<3, PREC_F32D, true, 3>(A, nblocks, s);
      else launch_step<3, PREC_F32D, false, 3>(A, nblocks, s);
    } else {
      if (multid) launch_step<3, PREC_F32, true, 3>(A, nblocks, s);
      else launch_step<3, PREC_F32, false, 3>(A, nblocks, s);
    }
    return;
  }
  if (prec == PREC_F32D) {
    if (variant == 6) launch_pair<PREC_F32D, 6>(multid, A, nblocks, s);
    else launch_pair<PREC_F32D, 7>(multid, A, nblocks, s);
  } else {
    if (variant == 6) launch_pair<PREC_F32, 6>(multid, A, nblocks, s);
    else launch_pair<PREC_F32, 7>(multid, A, nblocks, s);
  }
}

}  // namespace gks
