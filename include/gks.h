/*
 * gks.h -- C ABI of the GB300 gas-kinetic flux library (libgks.so).
 *
 * The library advances the compressible Navier-Stokes equations with the gas-kinetic BGK-NS
 * interface flux (Righi 2013 Section 2; Xu's scheme) whose relaxation time carries a turbulent
 * part built from prescribed turbulence fields (Section 3, Eqs. tauttrivial, tautchen; Section 4,
 * Eqs. relaxation time, taua, tautchenadjusted).  One call of gks_step performs, per time step:
 * boundary cells, the CFL time step, the turbulent relaxation-time field, MUSCL reconstruction,
 * the interface equilibrium state from half-space Maxwellian moments, the slope coefficients
 * a, A, b, the time-integration coefficients, flux assembly (Eq. fluxesf) and the conservative
 * update, all in CUDA kernels on the handle's device.
 *
 * Conventions shared by every call:
 *   - Every call returns a gks_status; nothing throws across the ABI.  gks_last_error() gives a
 *     message for the last failing call on a handle.
 *   - Caller buffers are never retained: state and fields are copied in and out.
 *   - Device pointers must be on the handle's device.  Host buffers may be pageable or pinned
 *     (pinned buffers make the copies asynchronous up to the synchronising calls).
 *   - Work is ordered on the handle's CUDA stream.  gks_compute_dt, gks_residual, gks_get_time,
 *     gks_status_word and the host-memory variants of the copy calls synchronise that stream.
 *   - State layout: conservative variables W = (rho, rho u_1..rho u_D, rho E), nv = D + 2.
 *     SOA means [v][z][y][x] (x fastest), AOS means [z][y][x][v].  Primitive layout is
 *     (rho, u_1..u_D, p) in SOA order.
 *   - GKS_ENONPHYS (a cell reached rho <= 0 or p <= 0) is sticky until the next gks_set_state;
 *     it is reported by the synchronising calls.
 */
#ifndef GKS_H
#define GKS_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct gks_handle gks_handle;

typedef enum {
  GKS_OK = 0,
  GKS_EINVAL = 1,       /* invalid argument */
  GKS_ENOMEM = 2,       /* device or host allocation failed */
  GKS_ECUDA = 3,        /* a CUDA runtime call failed */
  GKS_ENONPHYS = 4,     /* non-physical state (rho <= 0 or p <= 0) produced */
  GKS_ETIMEOUT = 5,     /* a bounded device wait gave up */
  GKS_EUNSUPPORTED = 6  /* option not built */
} gks_status;

/* boundary conditions per axis side (Section 4: walls are treated as in conventional CFD) */
enum { GKS_BC_PERIODIC = 0, GKS_BC_TRANSMISSIVE = 1, GKS_BC_WALL = 2, GKS_BC_DIRICHLET = 3, GKS_BC_OUTFLOW = 4 };
/* turbulent relaxation time: none, tau_t = mu_t/p (Eq. tauttrivial), k-epsilon (Eq. tautchen),
 * k-omega (Eq. tautchenadjusted) from prescribed fields, or k-omega with k and omega transported
 * alongside the flow (Section 4; Wilcox's 2006 k-omega equations, see gks_komega) */
enum { GKS_TURB_NONE = 0, GKS_TURB_MUT = 1, GKS_TURB_KEPS = 2, GKS_TURB_KOMEGA = 3, GKS_TURB_KOMEGA_TRANSPORT = 4 };
enum { GKS_LIM_MINMOD = 0, GKS_LIM_VANLEER = 1 };
/* expansion of the distribution along the face normal only, or along every axis (Section 4) */
enum { GKS_EXPAND_DIRECTIONAL = 0, GKS_EXPAND_MULTID = 1 };
/* arithmetic: FP64 throughout; FP32 flux with the state accumulated as an unevaluated pair of
 * floats (about 48 significant bits); FP32 flux with an IEEE double state */
enum { GKS_FP64 = 0, GKS_FP32 = 1, GKS_FP32_ACC64 = 2 };
/* equilibrium time slope Abar: time-integrated compatibility (default) or the t = 0 one */
enum { GKS_ABAR_TIMEINT = 0, GKS_ABAR_T0 = 1 };
/* face reconstruction (Section 4 lists second- and third-order MUSCL and fifth-order WENO):
 * MUSCL2 = limited slopes over the centre distances (the default, `limiter` chooses minmod or van
 * Leer); MUSCL3 = the kappa = 1/3 scheme with minmod compression 4; WENO5 = Jiang and Shu's
 * fifth-order weighted reconstruction.  MUSCL3 and WENO5 work in index space on the conservative
 * variables, take the GKS normal slopes as the one-sided differences to the face values, keep the
 * MUSCL2 tangential slopes, and are built for GKS_FP64 and GKS_FP32 (in 3D for multi-dimensional
 * expansion only). */
enum { GKS_RECON_MUSCL2 = 0, GKS_RECON_MUSCL3 = 1, GKS_RECON_WENO5 = 2 };
enum { GKS_LAYOUT_SOA_CONS = 0, GKS_LAYOUT_AOS_CONS = 1, GKS_LAYOUT_SOA_PRIM = 2 };
enum { GKS_MEM_HOST = 0, GKS_MEM_DEVICE = 1 };
enum { GKS_F64 = 0, GKS_F32 = 1 };

typedef struct {
  int dim;                       /* 1, 2 or 3 */
  int n[3];                      /* cells per axis (>= 2 on active axes) */
  double lo[3], hi[3];           /* extent; used when dx[d] is NULL (uniform cells) */
  const double* dx[3];           /* host array of n[d] cell widths, or NULL */
  int bc[3][2];                  /* GKS_BC_* for [axis][lo, hi]; periodic must be set on both sides */
  const double* bc_data[3][2];   /* host, GKS_BC_DIRICHLET only: primitive (rho, u.., p) per boundary
                                    cell, cells ordered by the other axes in increasing order, [cell][nv] */
  int wake_cut;                  /* body-fitted 2D C-grids (gks_set_nodes, gks_steady_create): the first
                                    and last wake_cut cells of the j-lo side form a wake cut, the ghost
                                    cell (i, -k) being the cell (n0 - 1 - i, k - 1) across it (state,
                                    fields, centroid); the rest of that side keeps bc[1][0].  0: none */
} gks_grid;

typedef struct {
  double gamma;    /* ratio of specific heats; K = 2/(gamma-1) - dim internal degrees of freedom >= 0 */
  double mu;       /* molecular viscosity, tau_mol = mu / p (Section 2, Chapman-Enskog) */
  double prandtl;  /* only 1 (the BGK value) is built */
  double T_wall;   /* wall temperature in units of p/rho, GKS_BC_WALL */
} gks_gas;

/* degree of rarefaction in the time coefficients (Section 3): x = dt/tau, the exact time integral of
 * Eq. resultingf (the default; Eq. epsilonkepsilon), or eps = tau/tauhat with tauhat = rho/|D rho| the
 * resolved time scale of the mean flow (Eqs. tautautilde, tautilde, rarefactionkepsilon; Section 4,
 * Eq. epsilonkomega) in place of tau/dt inside alpha and beta of Eq. fkepsilon.  The library's reading:
 * D rho = d_t rho + U_n d_n rho at the face, d_t rho from the t = 0 compatibility condition of the
 * equilibrium part (-rho0 <(abar u + bbar v) psi_rho>_0), d_n rho the mean of (w0 - W_l)/dxl and
 * (W_r - w0)/dxr; tauhat at most 1e30 (uniform flow: eps -> 0); alpha = eps (1 - e^{-1/eps}),
 * beta = e^{-1/eps}; T0 = dt (1 - alpha), T1 = dt tau (2 alpha - 1 - beta), T2 = dt (dt/2 - tau
 * (1 - alpha)), T3 = dt alpha, T4 = dt tau (beta - 2 alpha), T5 = -dt tau alpha, and Abar from the
 * compatibility condition integrated with these. */
enum { GKS_RAR_DT = 0, GKS_RAR_TAUHAT = 1 };

/* Turbulence inputs (Section 3: tau_t from an eddy viscosity, Eq. tauttrivial, or from k and epsilon,
 * Eq. tautchen; Section 4: k and omega, Eq. tautchenadjusted; tau_a of Eq. taua). */
typedef struct {
  int model;        /* GKS_TURB_* */
  double C_mu;      /* k-epsilon constant (Eq. tautchen), usually 0.09 */
  double beta_star; /* k-omega: eta = S / (beta* omega) */
  double C_a;       /* artificial dissipation coefficient in [0, 1] (Eq. taua) */
  int rarefaction;  /* GKS_RAR_DT (default, zero) or GKS_RAR_TAUHAT.  GKS_RAR_TAUHAT is built for
                       MUSCL2 in every precision on rectilinear grids (the default tile shape), and
                       for GKS_FP64 and GKS_FP32 on body-fitted grids and in the steady solver;
                       GKS_EUNSUPPORTED otherwise */
} gks_turb;

typedef struct {
  int limiter;    /* GKS_LIM_* */
  int expand;     /* GKS_EXPAND_* */
  int precision;  /* GKS_FP64 | GKS_FP32 | GKS_FP32_ACC64 */
  int abar_mode;  /* GKS_ABAR_* */
  int reconstruction;  /* GKS_RECON_*; zero (the default) is MUSCL2 */
} gks_numerics;

/* Largest grid gks_create accepts, in cells: over a terabyte of state, beyond any device's memory. */
#define GKS_MAX_CELLS (1LL << 34)

/* Create a solver on the current CUDA device for the problem the paper states: a state on a grid
 * (Section 2, Eq. moment1), a gas with gamma and mu = tau p (Section 2, Eqs. maxwellian,
 * chapman-enskog-ns; Pr = 1), the turbulence inputs of Sections 3 and 4 (Eqs. tauttrivial, tautchen,
 * tautchenadjusted, taua) and the numerics of Section 4.  cuda_stream is a cudaStream_t or NULL (the
 * library then creates its own non-blocking stream).  All device buffers are allocated here and owned
 * by the handle.  Errors: GKS_EINVAL for bad sizes (fewer than two cells on an active axis, more than
 * GKS_MAX_CELLS cells in all), codes or Dirichlet data, GKS_EUNSUPPORTED for an option that is not
 * built (prandtl != 1, see also gks_turb.rarefaction), GKS_ENOMEM, GKS_ECUDA.  Arguments are checked
 * before any CUDA call.  On an error after the handle itself is allocated (every error but a null
 * argument or a failed host allocation), *out receives a handle that holds the message
 * (gks_last_error) and must be passed to gks_destroy. */
gks_status gks_create(const gks_grid* grid, const gks_gas* gas, const gks_turb* turb,
                      const gks_numerics* num, void* cuda_stream, gks_handle** out);

/* Copy a state in: the conservative variables W = (rho, rho U, rho E), the moments of the distribution
 * (Section 2, Eq. moment1), in any layout, float or double, host or device; reset time to 0, the step
 * counter and the sticky status.  The CFL rate of the new state is computed on the device; a cell with
 * rho <= 0 or p <= 0 sets the sticky GKS_ENONPHYS status. */
gks_status gks_set_state(gks_handle* h, const void* W, int layout, int memspace, int dtype);

/* Body-fitted 2D grid (the C-type and channel grids of the paper's cases, Section 5, Table 2):
 * nodes[(n1 + 1)][(n0 + 1)][2] = (x, y) of the structured node lattice (host or device, double;
 * copied, not retained); cell (i, j) is the quadrilateral of nodes (i, j), (i+1, j), (i+1, j+1),
 * (i, j+1), which must be convex and counter-clockwise.  The grid's widths and extents are then
 * unused; boundary conditions keep their meaning on the index lattice (GKS_BC_WALL: no-slip image;
 * a periodic axis repeats by translation).  Each face works in its own frame: unit normal n
 * towards increasing index, states rotated to (rho, rho u_n, rho u_t, rho E), MUSCL slopes along
 * the grid line over centroid distances (vertex-average centroids; ghost centroids mirrored
 * through the boundary face midpoint, or translated by the period), the flux weighted by the face
 * length and the update divided by the cell area; tau_t from Green-Gauss velocity gradients (a
 * ghost cell takes its source cell's value); CFL rate sum_faces (|U.n| + c) L / (2 A).  With
 * GKS_EXPAND_MULTID each face also takes tangential slopes of its two cells in the face frame: limited
 * differences along the transverse grid line over the centroid steps projected on the face tangent
 * (corner ghost centroids by the parallelogram of the i ghost, the j ghost and their source cell).
 * With GKS_TURB_KOMEGA_TRANSPORT, rho k and rho omega are advanced after each flow step as on
 * rectilinear grids, in each face's frame: convection by the face mass flux times L with half-time
 * upwind values along the grid line (the swept length F_rho / (rho L)), normal diffusion over the
 * centroid distance, sources with Green-Gauss gradients, each divergence over the cell area.
 * With GKS_RECON_MUSCL3 or GKS_RECON_WENO5 the face values come from the index-space formulas on
 * the four or six rotated cells along the grid line, the normal slopes being the one-sided
 * differences to the face values over the centroid-to-face distances (tangential slopes as for
 * MUSCL2).  Built for dim 2 (GKS_EUNSUPPORTED otherwise), both expansions, every reconstruction and
 * precision the handle allows.  May be called before or after gks_set_state; a second call
 * replaces the grid.  GKS_EINVAL for a folded or clockwise cell (the handle's grid is then the
 * rectilinear one again).
 * gks_get_tau_turb and gks_get_rarefaction work on such grids (Green-Gauss gradients and divergence,
 * face values the means of the two cells). */
gks_status gks_set_nodes(gks_handle* h, const double* nodes, int memspace);

/* Steady-state solver on a body-fitted 2D grid (Section 4: the paper's solver is steady, with local
 * time stepping, LU-SGS smoothing in the form of Yoon and Jameson and 4-level multigrid).  The
 * readings of this library:
 *   - local explicit step s_i = 2 A_i / sum_faces (|U.n| + c) L; the steady residual R_i = sum over
 *     the faces of (the face flux integrated over the window cfl_flux min(s_l, s_r)) / window times
 *     L, outward (a ghost cell has its source cell's step);
 *   - LU-SGS with pseudo-time steps cfl s_i on tiles of lusgs_tile x lusgs_tile cells (16, the
 *     default when 0, or 32; neighbours outside a tile enter neither sweep; on the 528 x 136 corner
 *     grid 16 x 16 tiles need 4% more cycles than 32 x 32 and take 25% less time per cycle): D dW*_i = -R_i - sum_{(i-1,j),(i,j-1)} 1/2 (dF_j - lambda dW*_j) L,
 *     dW_i = dW*_i - D^-1 sum_{(i+1,j),(i,j+1)} 1/2 (dF_j - lambda dW_j) L, D = A/dt + 1/2 sum lambda L,
 *     dF_j the change of the Euler flux of cell j through the face (normal away from cell i),
 *     lambda = max over the two cells of |U.n| + c, plus 2 (mu + p tau_t)/(rho d) (face means, d the
 *     centroid distance);
 *   - FAS multigrid over `levels` grids (each coarse grid takes every second node; n divisible by
 *     2^(levels-1)): state restricted by area weights, residuals by sums, prescribed turbulence
 *     fields and Dirichlet data by means; coarse residuals first order with the forcing
 *     sum R_f - R_c(W_c^0); one LU-SGS smoothing per level on the way down, the corrections
 *     W_c - W_c^0 injected on the way up.
 *   - GKS_TURB_KOMEGA_TRANSPORT: each cycle first takes k = rho k / rho, omega = rho omega / rho of
 *     its starting state on the finest grid (four-cell means below), evaluates the fine residual
 *     with them, and from the same residual (its face mass flux rates m, times L, and local steps)
 *     makes one diagonal-implicit step of the steady k-omega equations (the model of gks_komega):
 *     per face G = m phi_upwind - (mu + sigma rho k / omega |face) L / d12 (phi_r - phi_l), phi the
 *     cell value plus its limited slope along the grid line times the centroid-to-face distance;
 *     per cell R = sum G (outward) - A (S - beta omega rho k) with Wilcox's production terms S,
 *     rho k -= R / D, D = A / (cfl s) + sum_faces (max(m_out, 0) + conductance) / rho + A beta omega
 *     (beta* for k, beta0 for omega), then the floors; the flow cycle keeps the fields of the
 *     cycle's start.
 *   - gks_turb.rarefaction = GKS_RAR_TAUHAT (the paper's steady solver): the faces of every level's
 *     residual take the degree of rarefaction eps = tau/tauhat in place of tau over the face window
 *     inside the time coefficients (MUSCL2 only); the window itself is unchanged.
 * Built for GKS_FP64 and GKS_FP32 (state stored in the arithmetic type), both expansions and the
 * three reconstructions (MUSCL2, MUSCL3, WENO5 as for gks_set_nodes) on the finest level (coarse
 * levels are first order), turbulence models NONE, MUT, KEPS, KOMEGA (prescribed fields) and
 * KOMEGA_TRANSPORT.  nodes: host,
 * [(n1 + 1)][(n0 + 1)][2] as gks_set_nodes.  Errors: GKS_EUNSUPPORTED for other options, GKS_EINVAL
 * for bad sizes, levels or a folded cell on any level. */
typedef struct gks_steady gks_steady;
gks_status gks_steady_create(const gks_grid* grid, const gks_gas* gas, const gks_turb* turb,
                             const gks_numerics* num, const double* nodes, int levels, int lusgs_tile,
                             void* cuda_stream, gks_steady** out);
/* Copy the fine-grid state in (as gks_set_state; Section 2, Eq. moment1); the prescribed turbulence fields (as
 * gks_set_turbulence; coarse levels take four-cell means).  With GKS_TURB_KOMEGA_TRANSPORT the fields
 * are the initial k and omega, stored as rho k and rho omega with the density of the current state:
 * set the state first (gks_steady_set_state clears them); GKS_EINVAL otherwise. */
gks_status gks_steady_set_state(gks_steady* s, const void* W, int layout, int memspace, int dtype);
gks_status gks_steady_set_turbulence(gks_steady* s, const void* f1, const void* f2, int memspace, int dtype);
/* Run ncycles multigrid cycles of the steady solver of Section 4 (one CUDA graph per cycle, captured
 * once per (cfl, cfl_flux)); res_out
 * (host, ncycles entries, or NULL) receives the RMS over fine cells of R_rho / A before each cycle.
 * Synchronises the stream; GKS_ENONPHYS if the fine state is non-physical afterwards. */
gks_status gks_steady_cycles(gks_steady* s, int ncycles, double cfl, double cfl_flux, double* res_out);
/* The fine-level local steps (host, ncell) and steady residual (Section 4; host, [4][ncell]) of the
 * current state, second order unless first_order; either output may be NULL.  Synchronises. */
gks_status gks_steady_residual(gks_steady* s, double cfl_flux, int first_order, double* dt_out, double* R_out);
/* Copy out the fine-grid state (Section 2, Eq. moment1). */
gks_status gks_steady_get_state(gks_steady* s, void* W_out, int layout, int memspace, int dtype);
/* Free the steady solver; the message of its last failing call (no paper counterpart). */
gks_status gks_steady_destroy(gks_steady* s);
const char* gks_steady_last_error(const gks_steady* s);

/* Copy out the current state W (Section 2, Eq. moment1) in the requested layout and type. */
gks_status gks_get_state(gks_handle* h, void* W_out, int layout, int memspace, int dtype);

/* Copy in the turbulence fields (Section 3, Eqs. tauttrivial and tautchen; Section 4,
 * Eq. tautchenadjusted), one value per cell in [z][y][x] order: f1 = k (or mu_t),
 * f2 = epsilon or omega (NULL for GKS_TURB_MUT).  With GKS_TURB_KOMEGA_TRANSPORT these are the
 * initial k and omega, stored as rho k and rho omega with the density of the current state: call
 * it after gks_set_state (which clears transported fields); GKS_EINVAL otherwise. */
gks_status gks_set_turbulence(gks_handle* h, const void* f1, const void* f2, int memspace, int dtype);

/* k-omega transport (GKS_TURB_KOMEGA_TRANSPORT).  Each gks_step step advances the flow and then
 * rho k, rho omega with the same dt:
 *   d(rho k)/dt + div(rho U k) = P - beta* rho k omega + div((mu + sigma* rho k/omega) grad k)
 *   d(rho w)/dt + div(rho U w) = alpha (omega/k) P - beta rho omega^2
 *                                + sigma_d (rho/omega) grad k . grad omega + div((mu + sigma rho k/omega) grad omega)
 *   P = mu_T (2 S:S - 2/3 (div U)^2) - 2/3 rho k div U, mu_T = rho k / max(omega, C_lim sqrt(2 Sbar:Sbar/beta*)),
 *   beta = beta0 (1 + 85 chi)/(1 + 100 chi) (chi the vortex-stretching invariant, zero in 1D and 2D),
 *   sigma_d = sigma_do where grad k . grad omega > 0, else 0;
 * convection by the flow step's face mass fluxes with half-time MUSCL face values of the upwind
 * cell, normal diffusion with the mean coefficient of the two cells, destruction point-implicit,
 * then k >= 0 and omega >= omega_floor.  The turbulent relaxation time of the flow step uses
 * k and omega of the step's start (Eq. tautchenadjusted).  beta* is gks_turb.beta_star.  Ghost
 * values of k and omega: periodic axes wrap, other boundaries take the nearest interior cell. */
typedef struct {
  double alpha, beta0, sigma, sigma_star, sigma_do, C_lim;
  double omega_floor;  /* smallest omega kept after an update */
  int sources;         /* 0: convection and diffusion only (tests) */
  int diffusion;       /* 0: no diffusion (tests) */
} gks_komega;

/* The closure coefficients of the k-omega model the paper uses (Section 4: Wilcox 2006), Wilcox's
 * values: alpha 13/25, beta0 0.0708, sigma 1/2, sigma* 3/5, sigma_do 1/8, C_lim 7/8;
 * omega_floor 1e-12, sources and diffusion on.  Errors: GKS_EINVAL for a null pointer. */
gks_status gks_komega_defaults(gks_komega* c);

/* Replace the closure coefficients (Section 4, the k-omega model) of a GKS_TURB_KOMEGA_TRANSPORT handle (the defaults are set at
 * gks_create).  Takes effect from the next gks_step.  Errors: GKS_EINVAL (null, other model). */
gks_status gks_set_komega(gks_handle* h, const gks_komega* c);

/* Copy out the transported k and omega (Section 4; GKS_TURB_KOMEGA_TRANSPORT), one value per cell. */
gks_status gks_get_turbulence(gks_handle* h, void* k_out, void* omega_out, int memspace, int dtype);

/* Steady solver handles with GKS_TURB_KOMEGA_TRANSPORT (Section 4): replace the closure coefficients (defaults gks_komega_defaults;
 * effective from the next cycle), and copy out k = rho k / rho, omega = rho omega / rho of the
 * current state (either output may be NULL; synchronises).  GKS_EINVAL for other handles. */
gks_status gks_steady_set_komega(gks_steady* s, const gks_komega* c);
gks_status gks_steady_get_turbulence(gks_steady* s, void* k_out, void* omega_out, int memspace, int dtype);

/* CFL time step of the current state: dt = cfl / max_cells sum_d (|U_d| + c) / dx_d (no paper
 * counterpart: the paper's solver is steady and gives no time-step rule; this is the library's
 * reading).  Synchronises;
 * GKS_ENONPHYS if the sticky status is set. */
gks_status gks_compute_dt(gks_handle* h, double cfl, double* dt_out);

/* Advance nsteps steps of the finite-volume scheme with the time-integrated interface fluxes of
 * Eq. fluxesf (Section 2: Eqs. intermediatestate, initialf0, eqlgform, resultingf; relaxation time of
 * Eqs. relaxation time, taua and the turbulent part of Sections 3 and 4), W <- W - sum_d dF_d/dx_d.
 * dt > 0: fixed step; dt <= 0: the CFL step of the current state each step.
 * t_end > 0: the step that would pass t_end is clamped to reach it and later steps do nothing.
 * Asynchronous; the last step also accumulates the residual norms read by gks_residual. */
gks_status gks_step(gks_handle* h, double dt, double cfl, int nsteps, double t_end);

/* Time and number of steps taken since the last gks_set_state (or gks_set_time); no paper
 * counterpart.  Synchronises. */
gks_status gks_get_time(gks_handle* h, double* t, long long* steps);

/* Set the solution time (restart from a checkpoint: gks_set_state then gks_set_time); no paper
 * counterpart. */
gks_status gks_set_time(gks_handle* h, double t);

/* Residual of the last step (the rate of change that the steady solver of Section 4 drives to zero):
 * norms of (W^{n+1} - W^n)/dt of the last step of the last gks_step call, per variable (nv each):
 * L2 = sqrt(mean of squares), L-infinity, and total = sum of W times cell volume.  Synchronises. */
gks_status gks_residual(gks_handle* h, double* l2, double* linf, double* total);

/* Sticky status bits (bit 0: non-physical state) and the last time step used (no paper
 * counterpart).  Synchronises. */
gks_status gks_status_word(gks_handle* h, unsigned int* bits, double* last_dt);

/* Rarefaction diagnostic per cell (Eqs. tautautilde, tautilde): eps = (mu/p + tau_t) |div U|,
 * tauhat = rho / |D rho| with D rho = -rho div U. */
gks_status gks_get_rarefaction(gks_handle* h, void* eps_out, int memspace, int dtype);

/* Turbulent relaxation time per cell (Eqs. tauttrivial, tautchen, tautchenadjusted, T = p/rho). */
gks_status gks_get_tau_turb(gks_handle* h, void* tau_out, int memspace, int dtype);

/* Device time of the step kernels launched by gks_step while timing is enabled (CUDA events on
 * the handle's stream around each launch; graphs are not used while timing); no paper counterpart. */
gks_status gks_enable_timing(gks_handle* h, int enable);
gks_status gks_kernel_time(gks_handle* h, double* ms_total, long long* launches);

/* Tile shape of the handle's step kernel (no paper counterpart).  2D GKS_FP32 and GKS_FP32_ACC64 handles choose among nine
 * shapes (variants 0..5 and 8: 32x15, 64x7, 32x31, 32x27, 32x18, 64x27 and 32x21 cells, one face per thread
 * per round, 512 threads per CTA for 32x31 and 64x27, 256 otherwise; variants 6 and 7: 32x27 on 128 and
 * 64x27 on 256 threads, each thread evaluating two faces at once with the paired FP32 instructions), 3D ones
 * among four (16x8x4, 16x8x2, 8x8x4, and 16x8x2 with two faces per thread on 128 threads), 1D handles among 256, 31 and
 * 63 cells per CTA (the rarefaction option runs the first shape of each), on their first gks_step: each is timed
 * on the step about to be taken and the fastest kept (and reused by later handles of the same grid);
 * the environment variable GKS_TILE_VARIANT forces one (0..8 in 2D, 0..3 in 3D, 0..2 in 1D).  The result does
 * not depend on it beyond rounding. */
gks_status gks_tile_shape(gks_handle* h, int* variant, int* tx, int* ty, int* tz);

/* Free the handle and everything it owns (no paper counterpart: resource management). */
gks_status gks_destroy(gks_handle* h);
/* Message of the last failing call on a handle (no paper counterpart). */
const char* gks_last_error(const gks_handle* h);

/* Stateless evaluation of nfaces interface fluxes (Eq. fluxesf; Eqs. intermediatestate, initialf0,
 * eqlgform, resultingf, relaxation time, taua) on the device, for testing and for callers with their
 * own reconstruction.  rarefaction: GKS_RAR_DT or GKS_RAR_TAUHAT (see gks_turb).  faces: device array of nfaces records of
 * gks_face_record_len(dim) doubles, in the frame of the face (velocity 0 = normal):
 *   wl[nv] wr[nv] cl[nv] cr[nv] sl[nv] sr[nv] tl[dim-1][nv] tr[dim-1][nv] dxl dxr tau_t
 * (reconstructed states, adjacent cell averages, normal slopes, tangential slopes, centre-to-face
 * distances, turbulent relaxation time).  F_out: device, nfaces * nv time-integrated fluxes;
 * tau_out: device, nfaces total relaxation times, or NULL.  precision GKS_FP64 or GKS_FP32.
 * Asynchronous on cuda_stream. */
int gks_face_record_len(int dim);
gks_status gks_face_flux(int dim, int precision, int expand, int abar_mode, int rarefaction, double gamma,
                         double mu, double C_a, double dt, const double* faces, long nfaces, double* F_out,
                         double* tau_out, void* cuda_stream);

/* Operation count of one interface flux (Eq. fluxesf) as the device code is written (no GPU needed): counts[0..5]
 * = additions/subtractions, multiplications, divisions, square roots, exponentials, erfc.
 * with_recon adds the face values of the MUSCL reconstruction from the cell slopes.  Operations on
 * literal 0 or 1 are not counted.  Used to state the algorithmic FLOPs behind the roofline figures. */
int gks_face_op_count(int dim, int expand, int with_recon, long long* counts);
/* The same count for the per-cell part of the reconstruction (Section 4): the limited (van Leer) slope of every
 * variable along every axis, computed once per cell and step. */
int gks_cell_op_count(int dim, long long* counts);
/* The same count for the face values of a higher-order reconstruction (Section 4; recon = GKS_RECON_MUSCL3 or
 * GKS_RECON_WENO5): both sides, every variable, and the two one-sided normal slopes of a face.
 * Returns nonzero for other values. */
int gks_recon_op_count(int dim, int recon, long long* counts);

/* CFL time step, as gks_compute_dt computes it, of a caller-held FP64 state on a uniform grid, for
 * callers that cannot allocate device memory (for example while another allocator holds all of
 * the device's free memory, or on a path where the implicit synchronisation of cudaMalloc is not
 * acceptable).  The paper has no counterpart: this is an allocation-free variant of the library's
 * CFL reduction.
 *   dim, n[dim], h[dim]  grid dimension, cells and (uniform) cell width per axis
 *   W        device, SoA conservative state [nv][cells] in double (caller-owned, read only)
 *   dt_out   host: cfl / max_cells sum_d (|U_d| + c) / h_d; not written unless GKS_OK
 * Errors: GKS_EINVAL for bad sizes or arguments, more than GKS_NOALLOC_MAX_CELLS cells, or a stream
 * that is being captured into a CUDA graph (the call copies to the host and synchronises, which a
 * capture cannot hold: never make it on a capturing stream); GKS_ENONPHYS if a cell has rho <= 0,
 * p <= 0 or NaN (as gks_compute_dt reports such a state); GKS_ECUDA.
 * No device memory is allocated: the scratch is a static device array inside the library (about
 * 8 KB, 1024 partial maxima, held on every device that loads the library until the process exits).
 * The first call on a device looks up the array's device address (cudaGetSymbolAddress) and the SM
 * count with that device current.  Every call shares the array and the last call's contents stay in
 * it, so calls that overlap on the GPU (concurrent streams or threads) race and must be serialised by
 * the caller.  Synchronises cuda_stream (NULL: the legacy default stream). */
#define GKS_NOALLOC_MAX_CELLS (16384L * 1024L)
gks_status gks_cfl_dt_noalloc(int dim, const int* n, const double* h, double gamma, const double* W,
                              double cfl, double* dt_out, void* cuda_stream);

/* ---- Serving: continuous batching of independent solves on one GPU (no paper counterpart: each
 * solve is the time-accurate scheme of gks_step, Eq. fluxesf) ----------------------------------
 * A server owns a device arena.  Submitted requests wait in arrival order until the arena has room
 * for their state (footprint admission); admitted solves stay resident and advance together, one
 * persistent batch launch per step per group (1D, 2D directional, 2D multi-dimensional), in chunks
 * of chunk_steps steps replayed as captured CUDA graphs.  Between chunks a worker thread retires
 * finished solves (final state copied to the host, memory freed) and admits waiting ones.  Each
 * solve computes exactly what the single-solve path computes (same tile kernel, its own CFL time
 * step), so its result does not depend on the rest of the batch.  Uniform grids without turbulence
 * model; boundaries periodic, transmissive, outflow or wall. */
typedef struct gks_server gks_server;

typedef struct {
  int dim;               /* 1 or 2 */
  int n[3];              /* cells per axis */
  double lo[3], hi[3];   /* extent (uniform cells) */
  int bc[3][2];          /* GKS_BC_PERIODIC | TRANSMISSIVE | OUTFLOW | WALL */
  double gamma, mu, C_a, T_wall;
  double cfl;            /* CFL number of the time step */
  int limiter, expand;   /* GKS_LIM_*, GKS_EXPAND_* */
  int nsteps;            /* steps to run */
} gks_request;

/* Serving (no paper counterpart).  precision GKS_FP32 (float-pair state) or GKS_FP64; arena_bytes of device memory for resident
 * solves; max_cells per request; chunk_steps a multiple of 6.  Starts the worker thread. */
gks_status gks_server_create(int precision, size_t arena_bytes, long max_cells, int chunk_steps, void* cuda_stream,
                             gks_server** out);
/* Serving (no paper counterpart): queue a request with its initial primitive state (host, SoA (rho, u.., p), copied).  GKS_ENOMEM if
 * the request can never fit in the arena. */
gks_status gks_server_submit(gks_server* s, const gks_request* q, const double* prim, long long* id_out);
/* Serving (no paper counterpart): done = 1 once finished; then W_out (host, SoA conservative, or NULL) receives the final state and
 * latency_s the time from submission to completion. */
gks_status gks_server_poll(gks_server* s, long long id, int* done, double* W_out, double* latency_s);
/* Serving (no paper counterpart): block until every submitted request has finished (GKS_ETIMEOUT
 * after timeout_s seconds). */
gks_status gks_server_wait_all(gks_server* s, double timeout_s);
/* Serving (no paper counterpart): completed requests, latency percentiles (seconds), completions per
 * second since the first submission, and seconds the GPU spent in batch steps; destroy a server. */
gks_status gks_server_stats(gks_server* s, long long* completed, double* p50_s, double* p99_s, double* solves_per_s,
                            double* busy_s);
/* Serving (no paper counterpart): the tile shape of each group's batch kernel (variants of
 * gks_tile_shape: [0] 1D, [1] 2D directional, [2] 2D multi-dimensional).  A GKS_FP32 server times the
 * candidate shapes (1D: 0, 1, 2; 2D: 0, 1, 3, 4) on a synthetic batch of periodic solves once per
 * process and device, at the first gks_server_create, and keeps the fastest per group for every server
 * of the process (so a solve's result does not depend on the server or mix it runs in); the
 * environment variable GKS_BATCH_TILES="v1d,v2d,v2dm" forces them.  GKS_FP64 servers use shape 0. */
gks_status gks_server_tile_variants(gks_server* s, int* variants);
gks_status gks_server_destroy(gks_server* s);

/* Measured FMA throughput of the current device for FP32 and FP64 (independent FMA chains on every
 * SM, CUDA events), in TFLOP/s: context for the arithmetic roofline (no paper counterpart).
 * Synchronises the device. */
gks_status gks_probe_alu(double* fp32_tflops, double* fp64_tflops);
/* No paper counterpart: the FP32 chains of gks_probe_alu with the paired single-precision FMA (two FMAs per thread
 * instruction, sm_100 and later), in TFLOP/s: whether pairing raises the FP32 rate or only halves the
 * issue slots it takes.  Same conditions and errors as gks_probe_alu. */
gks_status gks_probe_alu_packed(double* fp32x2_tflops);
/* No paper counterpart: conversion throughput of the current device, double -> float and float -> double, in units of 1e9
 * conversions per second (independent chains on every SM, CUDA events): context for the
 * double-state form (GKS_FP32_ACC64), which converts the staged state and the increments.  Same
 * conditions and errors as gks_probe_alu. */
gks_status gks_probe_cvt(double* d2f_gops, double* f2d_gops);

#ifdef __cplusplus
}
#endif
#endif /* GKS_H */
