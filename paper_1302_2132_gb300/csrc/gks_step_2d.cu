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


cudaError_t prepare_batch_d2() {
  cudaError_t e = cudaSuccess, r;
  if ((r = prepare_batch<2, PREC_F64, false>()) != cudaSuccess) e = r;
  if ((r = prepare_batch<2, PREC_F32, false>()) != cudaSuccess) e = r;
  if ((r = prepare_batch<2, PREC_F64, true>()) != cudaSuccess) e = r;
  if ((r = prepare_batch<2, PREC_F32, true>()) != cudaSuccess) e = r;
  return e;
}

void launch_batch_d2(int prec, bool multid, const BatchArgs& B, int nblocks, cudaStream_t s) {
  if (multid) {
    if (prec == PREC_F64) launch_batch<2, PREC_F64, true>(B, nblocks, s);
    else launch_batch<2, PREC_F32, true>(B, nblocks, s);
    return;
  }
  if (prec == PREC_F64) launch_batch<2, PREC_F64, false>(B, nblocks, s);
  else launch_batch<2, PREC_F32, false>(B, nblocks, s);
}

}  // namespace gks
