// Alternative 2D tile shapes of the FP32 step kernel (variants 1, 2 and 8 here; 3 to 5 in
// gks_step_2d_tiles2.cu; 6 and 7, two faces per thread, in gks_step_pair.cu), chosen at run time by
// the autotuner.
#include "gks_dispatch.h"
#include "gks_step.cuh"

namespace gks {

cudaError_t prepare_step_d2_variants() {
  cudaError_t e = prepare_step_d2_variants2(), r;
  if ((r = prepare_step<2, PREC_F32, false, 1>()) != cudaSuccess) e = r;
  if ((r = prepare_step<2, PREC_F32, true, 1>()) != cudaSuccess) e = r;
  if ((r = prepare_step<2, PREC_F32, false, 2>()) != cudaSuccess) e = r;
  if ((r = prepare_step<2, PREC_F32, true, 2>()) != cudaSuccess) e = r;
  if ((r = prepare_step<2, PREC_F32, false, 8>()) != cudaSuccess) e = r;
  if ((r = prepare_step<2, PREC_F32, true, 8>()) != cudaSuccess) e = r;
  return e;
}

void launch_step_d2_variant(int variant, bool multid, const StepArgs& A, int nblocks, cudaStream_t s) {
  if (variant == 8) {
    if (multid) launch_step<2, PREC_F32, true, 8>(A, nblocks, s);
    else launch_step<2, PREC_F32, false, 8>(A, nblocks, s);
  } else if (variant >= 6) {
    launch_step_pair(2, PREC_F32, variant, multid, A, nblocks, s);
  } else if (variant >= 3) {
    launch_step_d2_variant2(variant, multid, A, nblocks, s);
  } else if (variant == 1) {
    if (multid) launch_step<2, PREC_F32, true, 1>(A, nblocks, s);
    else launch_step<2, PREC_F32, false, 1>(A, nblocks, s);
  } else {
    if (multid) launch_step<2, PREC_F32, true, 2>(A, nblocks, s);
    else launch_step<2, PREC_F32, false, 2>(A, nblocks, s);
  }
}

void tile_shape(int D, int variant, int* x, int* y, int* z) {
  if (D == 1) {
    *x = variant == 1 ? Tile<1, 1>::X : (variant == 2 ? Tile<1, 2>::X : Tile<1, 0>::X);
    *y = 1;
    *z = 1;
    return;
  }
  if (D == 3) {
    if (variant == 3) { *x = Tile<3, 3>::X; *y = Tile<3, 3>::Y; *z = Tile<3, 3>::Z; }
    else if (variant == 1) { *x = Tile<3, 1>::X; *y = Tile<3, 1>::Y; *z = Tile<3, 1>::Z; }
    else if (variant == 2) { *x = Tile<3, 2>::X; *y = Tile<3, 2>::Y; *z = Tile<3, 2>::Z; }
    else { *x = Tile<3, 0>::X; *y = Tile<3, 0>::Y; *z = Tile<3, 0>::Z; }
    return;
  }
  if (variant == 1) { *x = Tile<2, 1>::X; *y = Tile<2, 1>::Y; }
  else if (variant == 2) { *x = Tile<2, 2>::X; *y = Tile<2, 2>::Y; }
  else if (variant == 3) { *x = Tile<2, 3>::X; *y = Tile<2, 3>::Y; }
  else if (variant == 4) { *x = Tile<2, 4>::X; *y = Tile<2, 4>::Y; }
  else if (variant == 5) { *x = Tile<2, 5>::X; *y = Tile<2, 5>::Y; }
  else if (variant == 6) { *x = Tile<2, 6>::X; *y = Tile<2, 6>::Y; }
  else if (variant == 7) { *x = Tile<2, 7>::X; *y = Tile<2, 7>::Y; }
  else if (variant == 8) { *x = Tile<2, 8>::X; *y = Tile<2, 8>::Y; }
  else { *x = Tile<2, 0>::X; *y = Tile<2, 0>::Y; }
  *z = 1;
}

}  // namespace gks
