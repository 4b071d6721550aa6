// Entry points of the separately compiled kernel units.
#pragma once
#include <cuda_runtime.h>

namespace gks {

struct StepArgs;
struct BatchArgs;
struct KOmegaArgs;

cudaError_t prepare_step_d1();
cudaError_t prepare_step_d2();
cudaError_t prepare_step_d3();
void launch_step_d1(int prec, bool multid, const StepArgs& A, int nblocks, cudaStream_t s);
void launch_step_d2(int prec, bool multid, const StepArgs& A, int nblocks, cudaStream_t s);
void launch_step_d3(int prec, bool multid, const StepArgs& A, int nblocks, cudaStream_t s);

// 2D FP32 tile variants 1 to 4 (variant 0 is launch_step_d2) and the tile shape of a variant
cudaError_t prepare_step_d2_variants();
void launch_step_d2_variant(int variant, bool multid, const StepArgs& A, int nblocks, cudaStream_t s);
void tile_shape(int D, int variant, int* x, int* y, int* z);
constexpr int kTileVariants2D = 9;
// the paired tiles (two faces per thread) of the FP32 forms: 2D variants 6 and 7, 3D variant 3
cudaError_t prepare_step_pair();
void launch_step_pair(int D, int prec, int variant, bool multid, const StepArgs& A, int nblocks, cudaStream_t s);
// variants 3 to 5 (their own translation unit)
cudaError_t prepare_step_d2_variants2();
void launch_step_d2_variant2(int variant, bool multid, const StepArgs& A, int nblocks, cudaStream_t s);
// 3D FP32 tile variants 1 and 2 (256-cell tiles with the slope table)
cudaError_t prepare_step_d3_variants();
void launch_step_d3_variant(int variant, bool multid, const StepArgs& A, int nblocks, cudaStream_t s);
constexpr int kTileVariants3D = 4;
// double-state form (FP32 flux, IEEE double state): 2D variants 1 to 5, 3D variants 1 and 2
cudaError_t prepare_step_acc64();
void launch_step_acc64_variant(int D, int variant, bool multid, const StepArgs& A, int nblocks, cudaStream_t s);
// the rarefaction option (MUSCL-2, default tile of each dimension, every precision)
cudaError_t prepare_step_rar();
void launch_step_rar(int D, int prec, bool multid, const StepArgs& A, int nblocks, cudaStream_t s);
// 1D tile variants 1 and 2 (narrow tiles for small grids)
cudaError_t prepare_step_d1_variants();
void launch_step_d1_variant(int variant, int prec, const StepArgs& A, int nblocks, cudaStream_t s);
constexpr int kTileVariants1D = 3;

// batches of independent solves (FP64 or FP32 float-pair arithmetic) with a tile variant per group;
// prepare_* fill the resident CTAs per SM of each variant (1D: [v]; 2D: [2 v + multid])
cudaError_t prepare_batch_d1(int prec, int* resident);
cudaError_t prepare_batch_d2(int prec, int* resident);
void launch_batch_d1(int prec, int variant, const BatchArgs& B, int nblocks, cudaStream_t s);
void launch_batch_d2(int prec, int variant, bool multid, const BatchArgs& B, int nblocks, cudaStream_t s);

// higher-order reconstructions (default tiles, and the 32 x 27 tile for 2D FP32 multi-D; FP64 and
// FP32; 3D multi-dimensional only): false if the combination is not built
cudaError_t prepare_step_muscl3();
cudaError_t prepare_step_weno5();
bool launch_step_muscl3(int D, int prec, bool multid, int variant, const StepArgs& A, int nblocks, cudaStream_t s);
bool launch_step_weno5(int D, int prec, bool multid, int variant, const StepArgs& A, int nblocks, cudaStream_t s);

// k-omega transport step after a flow step (gks_komega.cu)
cudaError_t prepare_komega();
void launch_komega(int D, int prec, const KOmegaArgs& K, cudaStream_t s);

void launch_face_flux(int D, int prec, bool multid, int abar_t0, int rar, double gamma, double mu, double C_a,
                      double dt, const double* faces, long nfaces, double* F, double* tau, cudaStream_t s);

}  // namespace gks
