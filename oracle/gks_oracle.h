/*
 * ORACLE — TEST INFRASTRUCTURE, NOT PART OF THE LIBRARY.
 *
 * Plain, slow, double-precision CPU statement of the gas-kinetic BGK-Navier-Stokes scheme with a
 * turbulent relaxation time (Righi 2013, Sections 2-4, after Xu's 2001 scheme).  Only the tests,
 * __graft_entry__.smoke() and bench.py's cpu_baseline leg may load it.  It shares no source, header,
 * table or helper with the CUDA library (paper_1302_2132_gb300/csrc, include/gks.h).
 *
 * Conventions (all quantities double precision):
 *   D      spatial dimension 1..3, nv = D + 2 conservative variables (rho, rho*u_1..u_D, rho*E)
 *   K      internal degrees of freedom, K = 2/(gamma-1) - D (Section 2, Maxwellian)
 *   lambda = rho / (2 p)
 *   Moments <.> are normalised by rho.
 */
#ifndef GKS_ORACLE_H
#define GKS_ORACLE_H
#ifdef __cplusplus
extern "C" {
#endif

enum { ORC_FULL = 0, ORC_POS = 1, ORC_NEG = 2 };
enum { ORC_BC_PERIODIC = 0, ORC_BC_TRANSMISSIVE = 1, ORC_BC_WALL = 2, ORC_BC_DIRICHLET = 3, ORC_BC_OUTFLOW = 4 };
enum { ORC_TURB_NONE = 0, ORC_TURB_MUT = 1, ORC_TURB_KEPS = 2, ORC_TURB_KOMEGA = 3 };
enum { ORC_LIM_MINMOD = 0, ORC_LIM_VANLEER = 1 };
enum { ORC_ABAR_TIMEINT = 0, ORC_ABAR_T0 = 1 };
/* face reconstruction (Section 4 lists second- and third-order MUSCL and fifth-order WENO) */
enum { ORC_RECON_MUSCL2 = 0, ORC_RECON_MUSCL3 = 1, ORC_RECON_WENO5 = 2 };

typedef struct {
  int dim;
  int n[3];
  const double* dx[3];          /* per-cell widths along each axis, n[d] entries */
  int bc[3][2];                 /* ORC_BC_* per axis, [lo, hi] */
  const double* bc_prim[3][2];  /* Dirichlet data: primitive (rho, u_1..u_D, p) per boundary cell */
  double gamma, mu, T_wall;     /* T_wall in units of p/rho */
  int turb_model;
  double C_mu, beta_star, C_a;
  int limiter, multid, abar_mode;
  int recon;                    /* ORC_RECON_*; MUSCL2 uses `limiter` */
  int wake_cut;                 /* 2D C-grids: the first and last wake_cut cells of the j-lo side are a
                                   wake cut, ghost (i, -k) = cell (n0 - 1 - i, k - 1); 0: none */
  int rarefaction;              /* 0: x = dt/tau in the time coefficients; 1: the degree of rarefaction
                                   eps = tau/tauhat of Eqs. tautautilde, epsilonkomega in their place */
  int no_fallback;              /* tests only: the rectilinear step skips the first-order fallback of a face side whose
                                   reconstructed rho or p is not positive (a planted mistake) */
} orc_problem;

/* Per-face record, normal frame (velocity index 0 is the face normal):
 *   wl, wr   reconstructed conservative states left/right of the face        (nv each)
 *   cl, cr   cell averages of the two adjacent cells                          (nv each)
 *   sl, sr   normal slopes dW/dn of the left and right cells                  (nv each)
 *   tl, tr   tangential slopes, D-1 blocks of nv each                         (3*nv each slot)
 *   dxl, dxr distance from the left/right cell centre to the face
 *   tau_t    turbulent relaxation time at the face
 */
typedef struct {
  double wl[5], wr[5], cl[5], cr[5], sl[5], sr[5];
  double tl[2][5], tr[2][5];
  double dxl, dxr, tau_t;
} orc_face;

typedef struct {
  double w0[5];                 /* interface equilibrium state */
  double al[5], ar[5];          /* normal slope coefficients */
  double bl[2][5], br[2][5];    /* tangential slope coefficients */
  double Al[5], Ar[5];          /* time coefficients of the initial state */
  double abl[5], abr[5];        /* equilibrium normal slopes */
  double bb[2][5];              /* equilibrium tangential slopes */
  double Ab[5];                 /* equilibrium time coefficient */
  double tau;                   /* total relaxation time */
  double T[6];                  /* T0..T5 */
  double tauhat;                /* rarefaction option: rho / |D rho| at the face (0 otherwise) */
} orc_face_diag;

int orc_umoments(double U, double lam, int region, int nmax, double* out);
int orc_ximoments(double K, double lam, int lmax, double* out);
int orc_time_coeffs(double dt, double tau, double* T /* T0..T5, then dt^2/2 - T2 */);
int orc_slope(int D, double K, const double* w, const double* rhs, double* a_out);
int orc_time_coeffs_hat(double dt, double tau, double eps, double* T /* as orc_time_coeffs */);
int orc_face_flux(int D, double gamma, double mu, double C_a, double dt, int multid, int abar_mode,
                  int rarefaction, const orc_face* f, double* F, orc_face_diag* diag);
int orc_face_flux_compact(int D, double gamma, double mu, double C_a, double dt, int multid, int abar_mode,
                          int rarefaction, int printed_beta, const orc_face* f, double* F);
int orc_euler_flux(int D, double gamma, const double* w, double* F);
/* Number of face sides (over every face of every axis) whose reconstructed density or pressure is
 * not positive, i.e. that the step evaluates at first order. */
int orc_fallback_count(const orc_problem* P, const double* W, const double* f1, const double* f2, long* count);
/* Face values of a 1D row of cell averages v[0..n) with widths h (the ends take the nearest
 * cell): wl[i] = value at the right face of cell i (its own reconstruction), wr[i] = value at the
 * left face of cell i, for the faces with a full stencil; other entries are left untouched. */
int orc_reconstruct(int recon, int limiter, const double* v, const double* h, int n, double* wl, double* wr);

int orc_prim_to_cons(const orc_problem* P, const double* prim, double* W, long ncell);
int orc_cons_to_prim(const orc_problem* P, const double* W, double* prim, long ncell);
int orc_compute_dt(const orc_problem* P, const double* W, double cfl, double* dt);
int orc_tau_turb(const orc_problem* P, const double* W, const double* f1, const double* f2, double* tau_t);
int orc_rarefaction(const orc_problem* P, const double* W, const double* f1, const double* f2, double* eps);
int orc_step(const orc_problem* P, double* W, const double* f1, const double* f2, double dt,
             double* resid /* 3*nv: L2, Linf, total */, int nthreads);
int orc_run(const orc_problem* P, double* W, const double* f1, const double* f2, double dt_fixed,
            double cfl, int nsteps, double t_end, double* t_inout, int* steps_done, int nthreads);

/* k-omega transport solved together with the flow equations (Section 4 evolves k and omega this
 * way with Wilcox's 2006 k-omega model, which it cites without printing the equations).  Closure
 * coefficients; orc_komega_defaults fills Wilcox's 2006 values.  sources = 0 and diffusion = 0
 * switch those parts off (tests only). */
typedef struct {
  double alpha, beta0, beta_star, sigma, sigma_star, sigma_do, C_lim;
  double omega_floor;   /* smallest omega kept after an update */
  int sources, diffusion;
} orc_komega;
int orc_komega_defaults(orc_komega* c);
/* One flow step (as orc_step, with the turbulent relaxation time of the k-omega model from
 * k = RK/rho and omega = RW/rho) followed by the transport step of RK = rho k and RW = rho omega
 * with the same dt and the face mass fluxes of that flow step.  P->turb_model must be
 * ORC_TURB_KOMEGA.  Returns 4 if a cell ends with rho <= 0 or p <= 0. */
int orc_step_komega(const orc_problem* P, const orc_komega* c, double* W, double* RK, double* RW, double dt,
                    int nthreads);

/* Curvilinear (body-fitted) 2D grids with the directional expansion: the cells are the
 * quadrilaterals of a structured node lattice nodes[(j (n0+1) + i) * 2 + {0, 1}] = (x, y),
 * i = 0..n0, j = 0..n1 (P->dx is not used; P->dim must be 2, P->recon MUSCL2).  Per face: unit
 * normal pointing to increasing index, length, midpoint; per cell: area (diagonal cross product)
 * and the vertex-average centroid.  A face rotates its four-cell stencil along the grid line into
 * its (normal, tangent) frame, reconstructs with limited slopes over the centroid distances,
 * evaluates the face flux with the centroid-to-midpoint distances, rotates the momentum flux back
 * and weights it by the face length; a cell's update divides by its area.  Ghost cells follow
 * the boundary rules of the index lattice; ghost centroids are interior centroids reflected
 * through the boundary face midpoints (translated by the period on periodic axes; corners by the
 * parallelogram rule); the turbulent relaxation time uses Green-Gauss gradients (face velocity =
 * mean of the two cells) and a ghost cell takes its source cell's value.  With P->multid the face
 * also takes tangential slopes of its two cells: limited differences along the transverse grid
 * line over the centroid steps projected on the face tangent. */
/* Status 2 (nothing updated): a cell that is not a convex counter-clockwise quadrilateral. */
int orc_step_curv(const orc_problem* P, const double* nodes, double* W, const double* f1, const double* f2,
                  double dt, int nthreads);
/* Rarefaction diagnostic on a curvilinear grid: eps = (mu / p + tau_t) |div U| per cell, div U by
 * Green-Gauss with face values the means of the two cells. */
int orc_rarefaction_curv(const orc_problem* P, const double* nodes, const double* W, const double* f1,
                         const double* f2, double* eps);
/* CFL step on a curvilinear grid: dt = cfl / max_cells sum_faces (|U.n| + c) L / (2 A). */
int orc_compute_dt_curv(const orc_problem* P, const double* nodes, const double* W, double cfl, double* dt);

/* k-omega transport on a curvilinear grid (orc_step_komega in each face's frame; P->turb_model must be
 * ORC_TURB_KOMEGA): the flow step with tau_t from RK / rho, RW / rho, then RK, RW advanced with the
 * face mass fluxes, half-time upwind face values along the grid lines, normal diffusion over the
 * centroid distance, Wilcox's sources with Green-Gauss gradients, point-implicit destruction. */
int orc_step_komega_curv(const orc_problem* P, const double* nodes, const orc_komega* K, double* W, double* RK,
                         double* RW, double dt, int nthreads);

/* Steady-state solver on curvilinear grids (Section 4: local time stepping, LU-SGS, multigrid).
 * orc_steady_residual: local explicit steps dt_cell[i] = 2 A_i / sum_faces (|U.n| + c) L and the
 * residual R[v][i] = sum over faces of (flux over the face window cfl_flux min(dt_l, dt_r)) / window
 * * L, outward (first_order: no slopes).  orc_lusgs: the LU-SGS increment dW for residual R and
 * pseudo-time steps dt_cell,
 * sweeping tiles of tile0 x tile1 cells independently (neighbours outside the tile enter neither
 * sweep).  orc_steady_cycle: one FAS multigrid cycle over `levels` grids (every coarse grid takes
 * every second node; n divisible by 2^(levels-1)): LU-SGS smoothing with pseudo-time steps cfl times
 * the local explicit steps on the way down (fine level
 * second order, coarse levels first order with the FAS forcing), corrections injected on the way
 * up; *res = RMS over cells of R_rho / A before the cycle. */
int orc_steady_residual(const orc_problem* P, const double* nodes, const double* W, const double* f1,
                        const double* f2, double cfl, int first_order, double* dt_cell, double* R, int nthreads);
int orc_lusgs(const orc_problem* P, const double* nodes, const double* W, const double* f1, const double* f2,
              const double* dt_cell, const double* R, int tile0, int tile1, double* dW);
int orc_steady_cycle(const orc_problem* P, const double* nodes, double* W, const double* f1, const double* f2,
                     double cfl, double cfl_flux, int levels, int tile0, int tile1, int nthreads, double* res);

/* Steady k-omega update (P->turb_model ORC_TURB_KOMEGA): with k = RK / rho, omega = RW / rho and the
 * flow residual of W (face mass flux rates m over the windows cfl_flux min(dt_l, dt_r), local explicit
 * steps dt_loc), one diagonal-implicit step of the steady k-omega equations on the finest grid:
 * per face G = m phi_upwind - (mu + sigma rho k / omega |face) (phi_r - phi_l) / d12 L (phi the
 * cell value plus its limited slope times the centroid-to-face distance); per cell R = sum G
 * (outward) - A (S - beta omega RK), RK -= R / D with D = A / (cfl dt_loc) + sum (max(m_out, 0) +
 * conductance) / rho + A beta omega; floors RK >= 0, RW >= rho omega_floor.  W is not changed.  A
 * steady cycle with k-omega transport is this update followed by orc_steady_cycle with the fields
 * k, omega of the cycle's start. */
int orc_steady_komega(const orc_problem* P, const double* nodes, const orc_komega* K, const double* W, double* RK,
                      double* RW, double cfl, double cfl_flux, int nthreads);

#ifdef __cplusplus
}
#endif
#endif
