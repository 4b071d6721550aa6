// Body-fitted 2D grids (gks_curv.cu): device metrics and the step kernels of the directional
// expansion in each face's (normal, tangent) frame.
#pragma once
#include <cuda_runtime.h>

namespace gks {

struct StepArgs;
struct KOmegaArgs;

// Device buffers of a curvilinear grid, owned by the handle.
struct CurvGeom {
  long nf[2];     // faces per axis: (n0 + 1) n1 i-faces (x fastest), n0 (n1 + 1) j-faces
  void* face[2];  // per axis [8][nf], arithmetic type: n_x, n_y, L, 1/d01, 1/d12, 1/d23, d_l, d_r
                  // (d01, d12, d23 the centroid distances of the four-cell stencil along the grid
                  // line, d_l, d_r the distances from the two adjacent centroids to the face midpoint)
  void* tang[2];  // per axis [4][nf], arithmetic type: 1/hm, 1/hp of the left and of the right cell,
                  // hm, hp the centroid steps to the transverse neighbours projected on the tangent
  void* iarea;    // 1 / area per cell, arithmetic type
  double* area;   // area per cell
  void* tau;      // per-cell turbulent relaxation time of the current step, arithmetic type
  void* flux[2];  // per axis [4][nf]: time-integrated face flux times face length, arithmetic type
};

// Steady-residual mode of the fused tile kernel (arithmetic-type arrays of the level).
struct SteadyArgs {
  const void* s_loc;      // local explicit steps (CFL 1) per cell
  double cfl_flux;        // face window = cfl_flux min(s_l, s_r)
  int first_order;        // no slopes
  void* R;                // out: [4][ncell] sum over faces of the flux rate times L, outward (+ forcing)
  const void* forcing;    // [4][ncell] or null
  void* tau;              // out: tau_t per cell
  double* res_acc;        // if set: += sum over cells of (R_rho / A)^2
  int multid;             // multi-dimensional expansion (second-order levels only)
  int recon;              // GKS_RECON_* of the second-order level (MUSCL-3, WENO-5: launch_curv_residual_recon)
};

// Metrics from nodes[(n1 + 1)][(n0 + 1)][2] (device, double); *bad (device) is or-ed with 1 if a
// cell is not a convex counter-clockwise quadrilateral.  cut: cells of a C-grid wake cut at each end
// of the j-lo side (their ghost centroids are the centroids of the cells across the cut).
cudaError_t curv_metrics(const double* nodes, int n0, int n1, const bool periodic[2], int cut, int prec,
                         CurvGeom& G, int* bad, cudaStream_t s);
// The fused tile step (variant 0: 32 x 15 cells, 256 threads; variant 1: 16 x 7, 128 threads;
// variant 2: 16 x 11, 128 threads).
cudaError_t prepare_curv();
void launch_curv_step(int prec, const StepArgs& A, const CurvGeom& G, int variant, bool multid, cudaStream_t s);
// The same step with MUSCL-3 (recon 1) or WENO-5 (recon 2) along the grid lines: PREC_F64 or PREC_F32,
// tile variants 0 and 2 (any other variant runs as 2); prepare_curv_recon sets their shared memory.
cudaError_t prepare_curv_recon();
// The body-fitted MUSCL-2 time step with k-omega transport fused in (A.f1, A.f2: rho k, rho omega in;
// A.RKout, A.RWout and the kw_* coefficients of StepArgs): PREC_F64 or PREC_F32, tile variants 0 and 2.
cudaError_t prepare_curv_transport();
void launch_curv_step_transport(int prec, const StepArgs& A, const CurvGeom& G, int variant, bool multid,
                                cudaStream_t s);
// The steady residual (SteadyArgs, second-order level) with MUSCL-3 or WENO-5.
void launch_curv_residual_recon(int prec, const StepArgs& A, const CurvGeom& G, const SteadyArgs& SA, cudaStream_t s);
void launch_curv_step_recon(int prec, int recon, const StepArgs& A, const CurvGeom& G, int variant, bool multid,
                            cudaStream_t s);
// The rarefaction option (gks_turb.rarefaction = GKS_RAR_TAUHAT), MUSCL-2, FP64 or FP32: the time step on
// the 16 x 11 tile and the steady residual.
cudaError_t prepare_curv_rar();
void launch_curv_step_rar(int prec, const StepArgs& A, const CurvGeom& G, bool multid, cudaStream_t s);
void launch_curv_residual_rar(int prec, const StepArgs& A, const CurvGeom& G, const SteadyArgs& SA, cudaStream_t s);
void curv_tile_shape(int variant, int* x, int* y);
constexpr int kCurvVariants = 3;
void launch_curv_rate(int prec, const StepArgs& A, const CurvGeom& G, cudaStream_t s);
void launch_curv_tau(int prec, const StepArgs& A, const CurvGeom& G, void* out, cudaStream_t s, int what = 0);
// steady solver pieces (FP64 and FP32 state): the residual of A.Win, the local explicit steps
void launch_curv_residual(int prec, const StepArgs& A, const CurvGeom& G, const SteadyArgs& SA, cudaStream_t s);
void launch_curv_lts(int prec, const StepArgs& A, const CurvGeom& G, void* s_out, cudaStream_t s);
// k-omega transport after a flow step on the grid (K.mflux: the step's face mass fluxes times length)
void launch_curv_komega(int prec, const KOmegaArgs& K, const CurvGeom& G, cudaStream_t s);
// Steady k-omega update on the finest grid of the steady solver, in place (K.mflux: the residual's
// face mass flux rates times length; k, om: the fields of the cycle's start; pseudo-time steps
// cfl s_loc; PREC_F64 or PREC_F32)
void launch_steady_komega(int prec, const KOmegaArgs& K, const CurvGeom& G, const void* k, const void* om, void* RK,
                          void* RW, const void* s_loc, double cfl, cudaStream_t s);

}  // namespace gks
