// Instantiations of the fused step kernel for dimension 1.
#include "gks_dispatch.h"
#include "gks_step.cuh"

namespace gks {

cudaError_t prepare_step_d1() {
  cudaError_t e = cudaSuccess;
  cudaError_t r;
#define GKS_PREP(P, M) if ((r = prepare_step<1, P, M>()) != cudaSuccess) e = r;
  GKS_PREP(PREC_F64, false)
  GKS_PREP(PREC_F32, false)
  GKS_PREP(PREC_F32D, false)

#undef GKS_PREP
  return e;
}

void launch_step_d1(int prec, bool multid, const StepArgs& A, int nblocks, cudaStream_t s) {

  if (prec == PREC_F64) launch_step<1, PREC_F64, false>(A, nblocks, s);
  else if (prec == PREC_F32) launch_step<1, PREC_F32, false>(A, nblocks, s);
  else launch_step<1, PREC_F32D, false>(A, nblocks, s);
}


// Batch kernels of 1D solves: tile variants 0 (256 cells), 1 (31), 2 (63) in FP32, variant 0 in FP64.
// resident[v]: CTAs per SM of variant v (FP32), or of variant 0 (FP64, resident[0]).
cudaError_t prepare_batch_d1(int prec, int* resident) {
  cudaError_t e = cudaSuccess, r;
  if (prec == PREC_F64) return prepare_batch<1, PREC_F64, false, 0>(&resident[0]);
  if ((r = prepare_batch<1, PREC_F32, false, 0>(&resident[0])) != cudaSuccess) e = r;
  if ((r = prepare_batch<1, PREC_F32, false, 1>(&resident[1])) != cudaSuccess) e = r;
  if ((r = prepare_batch<1, PREC_F32, false, 2>(&resident[2])) != cudaSuccess) e = r;
  return e;
}

void launch_batch_d1(int prec, int variant, const BatchArgs& B, int nblocks, cudaStream_t s) {
  if (prec == PREC_F64) launch_batch<1, PREC_F64, false, 0>(B, nblocks, s);
  else if (variant == 1) launch_batch<1, PREC_F32, false, 1>(B, nblocks, s);
  else if (variant == 2) launch_batch<1, PREC_F32, false, 2>(B, nblocks, s);
  else launch_batch<1, PREC_F32, false, 0>(B, nblocks, s);
}


cudaError_t prepare_step_d1_variants() {
  cudaError_t e = cudaSuccess, r;
  if ((r = prepare_step<1, PREC_F64, false, 1>()) != cudaSuccess) e = r;
  if ((r = prepare_step<1, PREC_F32, false, 1>()) != cudaSuccess) e = r;
  if ((r = prepare_step<1, PREC_F32D, false, 1>()) != cudaSuccess) e = r;
  if ((r = prepare_step<1, PREC_F64, false, 2>()) != cudaSuccess) e = r;
  if ((r = prepare_step<1, PREC_F32, false, 2>()) != cudaSuccess) e = r;
  if ((r = prepare_step<1, PREC_F32D, false, 2>()) != cudaSuccess) e = r;
  return e;
}

void launch_step_d1_variant(int variant, int prec, const StepArgs& A, int nblocks, cudaStream_t s) {
  if (variant == 1) {
    if (prec == PREC_F64) launch_step<1, PREC_F64, false, 1>(A, nblocks, s);
    else if (prec == PREC_F32) launch_step<1, PREC_F32, false, 1>(A, nblocks, s);
    else launch_step<1, PREC_F32D, false, 1>(A, nblocks, s);
  } else {
    if (prec == PREC_F64) launch_step<1, PREC_F64, false, 2>(A, nblocks, s);
    else if (prec == PREC_F32) launch_step<1, PREC_F32, false, 2>(A, nblocks, s);
    else launch_step<1, PREC_F32D, false, 2>(A, nblocks, s);
  }
}

}  // namespace gks
