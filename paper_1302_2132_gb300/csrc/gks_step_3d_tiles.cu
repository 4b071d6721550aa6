// 3D tile shapes 1 (16x8x2) and 2 (8x8x4) of the FP32 step kernel, with the per-cell slope table,
// chosen at run time by the autotuner.
#include "gks_dispatch.h"
#include "gks_step.cuh"

namespace gks {

cudaError_t prepare_step_d3_variants() {
  cudaError_t e = cudaSuccess, r;
  if ((r = prepare_step<3, PREC_F32, false, 1>()) != cudaSuccess) e = r;
  if ((r = prepare_step<3, PREC_F32, true, 1>()) != cudaSuccess) e = r;
  if ((r = prepare_step<3, PREC_F32, false, 2>()) != cudaSuccess) e = r;
  if ((r = prepare_step<3, PREC_F32, true, 2>()) != cudaSuccess) e = r;
  return e;
}

void launch_step_d3_variant(int variant, bool multid, const StepArgs& A, int nblocks, cudaStream_t s) {
  if (variant == 3) {
    launch_step_pair(3, PREC_F32, 3, multid, A, nblocks, s);
  } else if (variant == 1) {
    if (multid) launch_step<3, PREC_F32, true, 1>(A, nblocks, s);
    else launch_step<3, PREC_F32, false, 1>(A, nblocks, s);
  } else {
    if (multid) launch_step<3, PREC_F32, true, 2>(A, nblocks, s);
    else launch_step<3, PREC_F32, false, 2>(A, nblocks, s);
  }
}

}  // namespace gks
