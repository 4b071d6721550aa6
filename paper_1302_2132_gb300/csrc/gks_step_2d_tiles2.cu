// 2D tile shapes 3 (32x27), 4 (32x18) and 5 (64x27, 512 threads) of the FP32 step kernel, chosen at run time by the
// autotuner (a translation unit of their own so that the library builds in parallel).
#include "gks_dispatch.h"
#include "gks_step.cuh"

namespace gks {

cudaError_t prepare_step_d2_variants2() {
  cudaError_t e = cudaSuccess, r;
  if ((r = prepare_step<2, PREC_F32, false, 3>()) != cudaSuccess) e = r;
  if ((r = prepare_step<2, PREC_F32, true, 3>()) != cudaSuccess) e = r;
  if ((r = prepare_step<2, PREC_F32, false, 4>()) != cudaSuccess) e = r;
  if ((r = prepare_step<2, PREC_F32, true, 4>()) != cudaSuccess) e = r;
  if ((r = prepare_step<2, PREC_F32, false, 5>()) != cudaSuccess) e = r;
  if ((r = prepare_step<2, PREC_F32, true, 5>()) != cudaSuccess) e = r;
  return e;
}

void launch_step_d2_variant2(int variant, bool multid, const StepArgs& A, int nblocks, cudaStream_t s) {
  if (variant == 3) {
    if (multid) launch_step<2, PREC_F32, true, 3>(A, nblocks, s);
    else launch_step<2, PREC_F32, false, 3>(A, nblocks, s);
  } else if (variant == 4) {
    if (multid) launch_step<2, PREC_F32, true, 4>(A, nblocks, s);
    else launch_step<2, PREC_F32, false, 4>(A, nblocks, s);
  } else {
    if (multid) launch_step<2, PREC_F32, true, 5>(A, nblocks, s);
    else launch_step<2, PREC_F32, false, 5>(A, nblocks, s);
  }
}

}  // namespace gks
