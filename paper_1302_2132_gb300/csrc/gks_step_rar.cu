// The step kernel with the rarefaction option (gks_turb.rarefaction = GKS_RAR_TAUHAT: the degree of
// rarefaction tau/tauhat in place of tau/dt in the time coefficients, Eqs. tautautilde, tautilde,
// epsilonkomega): MUSCL-2, the default tile of each dimension, every precision and expansion.
#include "gks_dispatch.h"
#include "gks_step.cuh"

namespace gks {

cudaError_t prepare_step_rar() {
  cudaError_t e = cudaSuccess, r;
#define GKS_PREP(D, P, M) if ((r = prepare_step<D, P, M, 0, RECON_MUSCL2, true>()) != cudaSuccess) e = r;
  GKS_PREP(1, PREC_F64, false) GKS_PREP(1, PREC_F32, false) GKS_PREP(1, PREC_F32D, false)
  GKS_PREP(2, PREC_F64, false) GKS_PREP(2, PREC_F32, false) GKS_PREP(2, PREC_F32D, false)
  GKS_PREP(2, PREC_F64, true) GKS_PREP(2, PREC_F32, true) GKS_PREP(2, PREC_F32D, true)
  GKS_PREP(3, PREC_F64, false) GKS_PREP(3, PREC_F32, false) GKS_PREP(3, PREC_F32D, false)
  GKS_PREP(3, PREC_F64, true) GKS_PREP(3, PREC_F32, true) GKS_PREP(3, PREC_F32D, true)
#undef GKS_PREP
  return e;
}

template <int D, bool M>
void launch_rar_d(int prec, const StepArgs& A, int nblocks, cudaStream_t s) {
  if (prec == PREC_F64) launch_step<D, PREC_F64, M, 0, RECON_MUSCL2, true>(A, nblocks, s);
  else if (prec == PREC_F32) launch_step<D, PREC_F32, M, 0, RECON_MUSCL2, true>(A, nblocks, s);
  else launch_step<D, PREC_F32D, M, 0, RECON_MUSCL2, true>(A, nblocks, s);
}

void launch_step_rar(int D, int prec, bool multid, const StepArgs& A, int nblocks, cudaStream_t s) {
  if (D == 1) launch_rar_d<1, false>(prec, A, nblocks, s);
  else if (D == 2 && multid) launch_rar_d<2, true>(prec, A, nblocks, s);
  else if (D == 2) launch_rar_d<2, false>(prec, A, nblocks, s);
  else if (multid) launch_rar_d<3, true>(prec, A, nblocks, s);
  else launch_rar_d<3, false>(prec, A, nblocks, s);
}

}  // namespace gks
