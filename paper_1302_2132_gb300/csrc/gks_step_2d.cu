// Instantiations of the fused step kernel for dimension 2.
#include "gks_dispatch.h"
#include "gks_step.cuh"

namespace gks {

cudaError_t prepare_step_d2() {
  cudaError_t e = cudaSuccess;
  cudaError_t r;
#define GKS_PREP(P, M) if ((r = prepare_step<2, P, M>()) != cudaSuccess) e = r;
  GKS_PREP(PREC_F64, false)
  GKS_PREP(PREC_F32, false)
  GKS_PREP(PREC_F32D, false)
  GKS_PREP(PREC_F64, true)
  GKS_PREP(PREC_F32, true)
  GKS_PREP(PREC_F32D, true)
#undef GKS_PREP
  return e;
}

void launch_step_d2(int prec, bool multid, const StepArgs& A, int nblocks, cudaStream_t s) {
  if (multid) {
    if (prec == PREC_F64) launch_step<2, PREC_F64, true>(A, nblocks, s);
    else if (prec == PREC_F32) launch_step<2, PREC_F32, true>(A, nblocks, s);
    else launch_step<2, PREC_F32D, true>(A, nblocks, s);
    return;
  }
  if (prec == PREC_F64) launch_step<2, PREC_F64, false>(A, nblocks, s);
  else if (prec == PREC_F32) launch_step<2, PREC_F32, false>(A, nblocks, s);
  else launch_step<2, PREC_F32D, false>(A, nblocks, s);
}


// Batch kernels of 2D solves: in FP32 the tile variants 0 (32x15), 1 (64x7), 3 (32x27), 4 (32x18) of
// both expansions, in FP64 variant 0.  resident[2 v + multid]: CTAs per SM.
template <int V>
cudaError_t prep_b2(int* resident) {
  cudaError_t e = prepare_batch<2, PREC_F32, false, V>(&resident[2 * V]);
  const cudaError_t f = prepare_batch<2, PREC_F32, true, V>(&resident[2 * V + 1]);
  return e != cudaSuccess ? e : f;
}

cudaError_t prepare_batch_d2(int prec, int* resident) {
  if (prec == PREC_F64) {
    const cudaError_t e = prepare_batch<2, PREC_F64, false, 0>(&resident[0]);
    const cudaError_t f = prepare_batch<2, PREC_F64, true, 0>(&resident[1]);
    return e != cudaSuccess ? e : f;
  }
  cudaError_t e = cudaSuccess, r;
  if ((r = prep_b2<0>(resident)) != cudaSuccess) e = r;
  if ((r = prep_b2<1>(resident)) != cudaSuccess) e = r;
  if ((r = prep_b2<3>(resident)) != cudaSuccess) e = r;
  if ((r = prep_b2<4>(resident)) != cudaSuccess) e = r;
  return e;
}

template <int V>
void launch_b2(bool multid, const BatchArgs& B, int nblocks, cudaStream_t s) {
  if (multid) launch_batch<2, PREC_F32, true, V>(B, nblocks, s);
  else launch_batch<2, PREC_F32, false, V>(B, nblocks, s);
}

void launch_batch_d2(int prec, int variant, bool multid, const BatchArgs& B, int nblocks, cudaStream_t s) {
  if (prec == PREC_F64) {
    if (multid) launch_batch<2, PREC_F64, true, 0>(B, nblocks, s);
    else launch_batch<2, PREC_F64, false, 0>(B, nblocks, s);
    return;
  }
  switch (variant) {
    case 1: launch_b2<1>(multid, B, nblocks, s); break;
    case 3: launch_b2<3>(multid, B, nblocks, s); break;
    case 4: launch_b2<4>(multid, B, nblocks, s); break;
    default: launch_b2<0>(multid, B, nblocks, s); break;
  }
}

}  // namespace gks
