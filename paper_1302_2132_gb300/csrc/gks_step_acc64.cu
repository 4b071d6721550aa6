// Tile shapes of the step kernel in the double-state form (FP32 flux, IEEE double state): 2D variants
// 1 to 5 and 8 and 3D variants 1 and 2, the same shapes as the float-pair form, chosen at run time by the
// autotuner (variant 0 is instantiated with the other precisions).
#include "gks_dispatch.h"
#include "gks_step.cuh"

namespace gks {

cudaError_t prepare_step_acc64() {
  cudaError_t e = cudaSuccess, r;
#define GKS_PREP(D, M, V) if ((r = prepare_step<D, PREC_F32D, M, V>()) != cudaSuccess) e = r;
  GKS_PREP(2, false, 1) GKS_PREP(2, true, 1)
  GKS_PREP(2, false, 2) GKS_PREP(2, true, 2)
  GKS_PREP(2, false, 3) GKS_PREP(2, true, 3)
  GKS_PREP(2, false, 4) GKS_PREP(2, true, 4)
  GKS_PREP(2, false, 5) GKS_PREP(2, true, 5)
  GKS_PREP(2, false, 8) GKS_PREP(2, true, 8)
  GKS_PREP(3, false, 1) GKS_PREP(3, true, 1)
  GKS_PREP(3, false, 2) GKS_PREP(3, true, 2)
#undef GKS_PREP
  return e;
}

template <int D, int V>
void launch_acc64(bool multid, const StepArgs& A, int nblocks, cudaStream_t s) {
  if (multid) launch_step<D, PREC_F32D, true, V>(A, nblocks, s);
  else launch_step<D, PREC_F32D, false, V>(A, nblocks, s);
}

void launch_step_acc64_variant(int D, int variant, bool multid, const StepArgs& A, int nblocks, cudaStream_t s) {
  if (D == 3) {
    if (variant == 3) launch_step_pair(3, PREC_F32D, 3, multid, A, nblocks, s);
    else if (variant == 1) launch_acc64<3, 1>(multid, A, nblocks, s);
    else launch_acc64<3, 2>(multid, A, nblocks, s);
    return;
  }
  if (variant == 8) {
    launch_acc64<2, 8>(multid, A, nblocks, s);
    return;
  }
  if (variant >= 6) {
    launch_step_pair(2, PREC_F32D, variant, multid, A, nblocks, s);
    return;
  }
  switch (variant) {
    case 1: launch_acc64<2, 1>(multid, A, nblocks, s); break;
    case 2: launch_acc64<2, 2>(multid, A, nblocks, s); break;
    case 3: launch_acc64<2, 3>(multid, A, nblocks, s); break;
    case 4: launch_acc64<2, 4>(multid, A, nblocks, s); break;
    default: launch_acc64<2, 5>(multid, A, nblocks, s); break;
  }
}

}  // namespace gks
