// Entry points of the separately compiled kernel units.
#pragma once
#include <cuda_runtime.h>

namespace gks {

struct StepArgs;

cudaError_t prepare_step_d1();
cudaError_t prepare_step_d2();
cudaError_t prepare_step_d3();
void launch_step_d1(int prec, bool multid, const StepArgs& A, int nblocks, cudaStream_t s);
void launch_step_d2(int prec, bool multid, const StepArgs& A, int nblocks, cudaStream_t s);
void launch_step_d3(int prec, bool multid, const StepArgs& A, int nblocks, cudaStream_t s);

void launch_face_flux(int D, int prec, bool multid, int abar_t0, double gamma, double mu, double C_a,
                      double dt, const double* faces, long nfaces, double* F, double* tau, cudaStream_t s);

}  // namespace gks
