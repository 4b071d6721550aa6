/*
 * ORACLE — TEST INFRASTRUCTURE, NOT PART OF THE LIBRARY.
 *
 * A plain double-precision CPU statement of the gas-kinetic BGK-Navier-Stokes scheme with a
 * turbulent relaxation time, written from Righi 2013 (Sections 2-4; the scheme is Xu's of 2001).
 * Only the tests, __graft_entry__.smoke() and bench.py's cpu_baseline leg may load it.  It shares
 * no code with the CUDA library: moments are taken of explicit polynomials in (u, v, w, xi^2)
 * term by term, and every slope coefficient is found by an LU solve of the moment matrix
 * <psi_m psi_n>, where the CUDA path uses hand-expanded closed forms.
 *
 * Readings of the paper that this file takes (the paper is silent, ambiguous or garbled there):
 *   - Maxwellian normalisation: g = rho (lambda/pi)^((K+D)/2) exp(-lambda(|u-U|^2 + xi^2)),
 *     K = 2/(gamma-1) - D internal degrees of freedom; the normalisation never enters the
 *     rho-normalised moments (Eq. maxwellian prints a garbled exponent).
 *   - Interface state (Eq. intermediatestate): the left Maxwellian contributes u > 0, the right
 *     one u < 0.
 *   - Equilibrium part (Eq. eqlgform): g0 (1 + abar x + bbar y + Abar t), with +Abar t as in
 *     Eq. resultingf; abar_l from (w0 - W_j)/(x_{j+1/2} - x_j), abar_r from
 *     (W_{j+1} - w0)/(x_{j+1} - x_{j+1/2}).
 *   - Each side uses its own coefficients (index typos in Eqs. resultingf and fupwind).
 *   - The flux is Xu's exact time integral (T0..T5 below) of Eq. resultingf; the compact form of
 *     Eq. resultingf4 agrees with it only when beta = exp(-1/eps) (the printed eps*exp(-1/eps) does
 *     not), which orc_face_flux_compact exhibits.
 *   - tau = mu/p0 + tau_t + tau_a (Eqs. relaxation time, taua) is one sum used everywhere.
 *   - Turbulent relaxation time (Eqs. tautchen, tautchenadjusted, tauttrivial): T = p/rho,
 *     S = sqrt(2 S_ij S_ij) by central differences, nu_t = C_mu k^2/eps with eta = S k/eps, or
 *     nu_t = k/omega with eta = S/(beta* omega); tau_t = rho nu_t / (p sqrt(1 + eta^2)); the face
 *     value is the mean of the two cells.
 *   - Rarefaction diagnostic (Eqs. tautautilde, tautilde): tauhat = rho/|D rho| with
 *     D rho = -rho div U (continuity), so eps = (mu/p + tau_t) |div U| per cell.
 *   - Reconstruction: MUSCL on conservative variables with minmod or van Leer, applied also to the
 *     tangential slopes; a side whose reconstructed rho or p is not positive falls back to first
 *     order at that face.
 *   - Body-fitted 2D grids (the paper's C-type and channel grids, Table 2) with the directional
 *     expansion: each face works in its own (normal, tangent) frame; MUSCL runs along the grid
 *     line with centroid distances (vertex-average centroids, ghosts mirrored through the boundary
 *     face or translated by the period); the face flux is weighted by the face length and the
 *     update divided by the cell area; tau_t takes Green-Gauss velocity gradients (face value the
 *     mean of the two cells) and a ghost cell the value of its source cell.  The multi-dimensional
 *     expansion takes tangential slopes in the face frame: limited differences along the transverse
 *     grid line, each over the centroid step projected on the face tangent.
 *     MUSCL-3 and WENO-5 on such grids reconstruct the rotated states along the grid line in index
 *     space; their normal slopes are the one-sided differences to the face values over the
 *     centroid-to-face distances.  C-grids: the first and last wake_cut cells of the j-lo side see
 *     the cells across the wake cut as their ghosts.
 *   - k-omega transport (Wilcox 2006; the paper cites the model without its equations): after each
 *     flow step with the same dt, convection by the face mass fluxes with half-time upwind values,
 *     normal diffusion with the mean coefficient of the two cells, sources from central (Green-Gauss
 *     on body-fitted grids) gradients, point-implicit destruction.
 *   - Steady-state solver (Section 4 names local time stepping, LU-SGS after Yoon and Jameson and
 *     4-level multigrid without formulas): see the block before curv_lts; with k-omega transport one
 *     diagonal-implicit steady k-omega step per cycle (orc_steady_komega).
 */
#include "gks_oracle.h"

#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>
#ifdef _OPENMP
#include <omp.h>
#endif

namespace {

const int MAXP = 10;  // highest power of u, v, w tabulated; (xi^2) up to 4

// ---------------------------------------------------------------------------------------------
// Polynomials in (u, v, w, xi^2): a list of monomials c * u^e0 v^e1 w^e2 (xi^2)^e3.
// ---------------------------------------------------------------------------------------------
struct Mono {
  int e[4];
  double c;
};
struct Poly {
  std::vector<Mono> t;
};

Poly pconst(double c) {
  Poly p;
  p.t.push_back({{0, 0, 0, 0}, c});
  return p;
}
// var 0,1,2 = velocity component in the normal frame (u, v, w); var 3 = xi^2
Poly pvar(int var, double c = 1.0) {
  Poly p;
  Mono m = {{0, 0, 0, 0}, c};
  m.e[var] = 1;
  p.t.push_back(m);
  return p;
}
void pmerge(Poly& p) {
  std::vector<Mono> out;
  for (const Mono& m : p.t) {
    bool found = false;
    for (Mono& o : out) {
      if (o.e[0] == m.e[0] && o.e[1] == m.e[1] && o.e[2] == m.e[2] && o.e[3] == m.e[3]) {
        o.c += m.c;
        found = true;
        break;
      }
    }
    if (!found) out.push_back(m);
  }
  p.t.swap(out);
}
Poly operator+(const Poly& a, const Poly& b) {
  Poly p = a;
  p.t.insert(p.t.end(), b.t.begin(), b.t.end());
  pmerge(p);
  return p;
}
Poly operator*(double s, const Poly& a) {
  Poly p = a;
  for (Mono& m : p.t) m.c *= s;
  return p;
}
Poly operator*(const Poly& a, const Poly& b) {
  Poly p;
  for (const Mono& x : a.t)
    for (const Mono& y : b.t) {
      Mono m;
      for (int i = 0; i < 4; ++i) m.e[i] = x.e[i] + y.e[i];
      m.c = x.c * y.c;
      p.t.push_back(m);
    }
  pmerge(p);
  return p;
}

// psi = (1, u_1..u_D, 1/2 (|u|^2 + xi^2)), Section 2 (moment map)
Poly psi(int D, int m) {
  if (m == 0) return pconst(1.0);
  if (m <= D) return pvar(m - 1);
  Poly e = pvar(3, 0.5);
  for (int i = 0; i < D; ++i) e = e + 0.5 * (pvar(i) * pvar(i));
  return e;
}
// a . psi, the polynomial expansion coefficient of Eq. initialf0
Poly expansion(int D, const double* a) {
  Poly p = a[0] * psi(D, 0);
  for (int m = 1; m < D + 2; ++m) p = p + a[m] * psi(D, m);
  return p;
}

// ---------------------------------------------------------------------------------------------
// Moments of a Maxwellian (Eq. maxwellian).  <u^n> over the full line or a half line, from the
// textbook Gaussian integrals: <1>_{u>0} = erfc(-sqrt(lam) U)/2,
// <u>_{u>0} = U <1>_{u>0} + exp(-lam U^2)/(2 sqrt(pi lam)), and integration by parts
// <u^{n+2}> = U <u^{n+1}> + (n+1)/(2 lam) <u^n> (valid on u>0, u<0 and the full line).
// Internal degrees of freedom: <(xi^2)^l> = prod_{i<l} (K + 2 i)/(2 lam).
// ---------------------------------------------------------------------------------------------
void umom(double U, double lam, int region, int nmax, double* out) {
  const double pi = 3.14159265358979323846;
  if (region == ORC_FULL) {
    out[0] = 1.0;
    out[1] = U;
  } else {
    double s = (region == ORC_POS) ? 1.0 : -1.0;
    out[0] = 0.5 * std::erfc(-s * std::sqrt(lam) * U);
    out[1] = U * out[0] + s * 0.5 * std::exp(-lam * U * U) / std::sqrt(pi * lam);
  }
  for (int n = 0; n + 2 <= nmax; ++n) out[n + 2] = U * out[n + 1] + (n + 1) / (2.0 * lam) * out[n];
}
void ximom(double K, double lam, int lmax, double* out) {
  out[0] = 1.0;
  for (int l = 1; l <= lmax; ++l) out[l] = out[l - 1] * (K + 2.0 * (l - 1)) / (2.0 * lam);
}

struct Maxw {
  int D;
  double K, rho, U[3], lam;
  double mu[3][MAXP + 1];   // normal velocity: full, u>0, u<0
  double mt[2][MAXP + 1];   // tangential velocities: full line
  double mx[5];
};

Maxw make_maxw(int D, double K, const double* w) {
  Maxw g;
  g.D = D;
  g.K = K;
  g.rho = w[0];
  double q = 0.0;
  for (int i = 0; i < 3; ++i) g.U[i] = 0.0;
  for (int i = 0; i < D; ++i) {
    g.U[i] = w[1 + i] / w[0];
    q += g.U[i] * g.U[i];
  }
  // rho E = 1/2 rho |U|^2 + (K + D) rho / (4 lambda)
  g.lam = (K + D) * g.rho / (4.0 * (w[D + 1] - 0.5 * g.rho * q));
  for (int r = 0; r < 3; ++r) umom(g.U[0], g.lam, r, MAXP, g.mu[r]);
  for (int k = 0; k < 2; ++k) umom(g.U[1 + k], g.lam, ORC_FULL, MAXP, g.mt[k]);
  ximom(K, g.lam, 4, g.mx);
  return g;
}

double moment(const Maxw& g, int region, const Poly& p) {
  double s = 0.0;
  for (const Mono& m : p.t) {
    if (m.e[0] > MAXP || m.e[1] > MAXP || m.e[2] > MAXP || m.e[3] > 4) return NAN;
    if (g.D < 2 && m.e[1] > 0) return NAN;
    if (g.D < 3 && m.e[2] > 0) return NAN;
    double v = m.c * g.mu[region][m.e[0]] * g.mx[m.e[3]];
    if (g.D >= 2) v *= g.mt[0][m.e[1]];
    if (g.D >= 3) v *= g.mt[1][m.e[2]];
    s += v;
  }
  return s;
}

// Dense LU with partial pivoting; solves M x = b in place (n <= 5).
bool lu_solve(int n, double M[5][5], double* b) {
  for (int c = 0; c < n; ++c) {
    int piv = c;
    for (int r = c + 1; r < n; ++r)
      if (std::fabs(M[r][c]) > std::fabs(M[piv][c])) piv = r;
    if (M[piv][c] == 0.0) return false;
    if (piv != c) {
      for (int k = 0; k < n; ++k) std::swap(M[c][k], M[piv][k]);
      std::swap(b[c], b[piv]);
    }
    for (int r = c + 1; r < n; ++r) {
      double f = M[r][c] / M[c][c];
      for (int k = c; k < n; ++k) M[r][k] -= f * M[c][k];
      b[r] -= f * b[c];
    }
  }
  for (int r = n - 1; r >= 0; --r) {
    double s = b[r];
    for (int k = r + 1; k < n; ++k) s -= M[r][k] * b[k];
    b[r] = s / M[r][r];
  }
  return true;
}

// Coefficients a of a . psi with <(a . psi) psi_m>_g = rhs_m (moments normalised by rho).
void slope(const Maxw& g, const double* rhs, double* a) {
  int nv = g.D + 2;
  double M[5][5];
  for (int m = 0; m < nv; ++m)
    for (int n = 0; n < nv; ++n) M[m][n] = moment(g, ORC_FULL, psi(g.D, m) * psi(g.D, n));
  for (int m = 0; m < nv; ++m) a[m] = rhs[m];
  if (!lu_solve(nv, M, a))
    for (int m = 0; m < nv; ++m) a[m] = NAN;
}

// ---------------------------------------------------------------------------------------------
// Time integrals over [0, dt] of the kernels of Eq. resultingf (from Kogan's Eq. integralbgk):
//   T0 = int (1 - e^{-t/tau})              T3 = int e^{-t/tau}
//   T1 = int ((tau + t) e^{-t/tau} - tau)  T4 = -int (tau + t) e^{-t/tau}
//   T2 = int (t - tau + tau e^{-t/tau})    T5 = -tau int e^{-t/tau}
// and Dn = dt^2/2 - T2.  For x = dt/tau < 1 each integral is summed from the exponential series
// term by term; otherwise the closed forms are used.
// ---------------------------------------------------------------------------------------------
void time_coeffs(double dt, double tau, double* T) {
  double x = dt / tau;
  if (tau > 0.0 && x < 1.0) {
    double t0 = 0, t1 = 0, t2 = 0, t3 = 0, t4 = 0, dn = 0;
    double xp = x, fact = 1.0;  // xp = x^(m+1), fact = (m+1)!
    for (int m = 0; m < 40; ++m) {
      double term = xp / fact;  // x^(m+1)/(m+1)!
      double sg = (m % 2 == 0) ? 1.0 : -1.0;  // (-1)^m
      t3 += sg * term;
      if (m >= 1) t0 += -sg * term;  // (-1)^(m+1)
      if (m >= 1) dn += -sg * term;
      if (m >= 2) t1 += sg * (1.0 - m) * term;
      if (m >= 2) t2 += sg * term;
      t4 += -sg * (1.0 - m) * term;
      xp *= x;
      fact *= (m + 2);
    }
    T[0] = tau * t0;
    T[1] = tau * tau * t1;
    T[2] = tau * tau * t2;
    T[3] = tau * t3;
    T[4] = tau * tau * t4;
    T[5] = -tau * T[3];
    T[6] = tau * tau * dn;
  } else {
    double E = std::exp(-x), q = 1.0 - E;
    T[0] = dt - tau * q;
    T[1] = -tau * dt * (1.0 + E) + 2.0 * tau * tau * q;
    T[2] = 0.5 * dt * dt - tau * dt + tau * tau * q;
    T[3] = tau * q;
    T[4] = tau * dt * E - 2.0 * tau * tau * q;
    T[5] = -tau * tau * q;
    T[6] = tau * dt - tau * tau * q;
  }
}

// The time coefficients with the degree of rarefaction eps in place of tau/dt (Eqs. tautautilde,
// rarefactionkepsilon, epsilonkomega; reading G9): Eq. fkepsilon with alpha = eps (1 - e^{-1/eps}) and
// beta = e^{-1/eps} (Eq. alphabetakepsilon with the corrected beta of reading G7), written as the
// T0..T5 of Eq. fluxesf (the compact form equals the time integral with these alpha, beta):
//   T0 = dt (1 - alpha)            T3 = dt alpha
//   T1 = dt tau (2 alpha - 1 - beta)  T4 = dt tau (beta - 2 alpha)
//   T2 = dt (dt/2 - tau (1 - alpha))  T5 = -dt tau alpha,   T[6] = dt^2/2 - T2 = dt tau (1 - alpha).
// With eps = tau/dt these are the coefficients of time_coeffs.  For eps > 1, 1 - alpha and
// 2 alpha - 1 - beta cancel to O(1/eps) and O(1/eps^2): they are summed from the exponential series
// in x = 1/eps term by term.
void time_coeffs_hat(double dt, double tau, double eps, double* T) {
  double a, one_a, c1, c4;
  if (eps > 1.0) {
    const double x = 1.0 / eps;
    a = 0.0;
    one_a = 0.0;
    c1 = 0.0;
    double xp = 1.0, fact = 1.0;  // xp = x^m, fact = (m+1)!
    for (int m = 0; m < 40; ++m) {
      const double term = xp / fact;  // x^m/(m+1)!
      const double sg = (m % 2 == 0) ? 1.0 : -1.0;
      a += sg * term;                          // alpha = sum (-x)^m/(m+1)!
      if (m >= 1) one_a -= sg * term;          // 1 - alpha
      if (m >= 2) c1 += sg * (1.0 - m) * term;  // 2 alpha - 1 - beta
      xp *= x;
      fact *= (m + 2);
    }
    c4 = std::exp(-x) - 2.0 * a;
  } else {
    const double beta = eps > 0.0 ? std::exp(-1.0 / eps) : 0.0;
    a = eps * (1.0 - beta);
    one_a = 1.0 - a;
    c1 = 2.0 * a - 1.0 - beta;
    c4 = beta - 2.0 * a;
  }
  T[0] = dt * one_a;
  T[1] = dt * tau * c1;
  T[2] = dt * (0.5 * dt - tau * one_a);
  T[3] = dt * a;
  T[4] = dt * tau * c4;
  T[5] = -dt * tau * a;
  T[6] = dt * tau * one_a;
}

double pressure(int D, double gamma, const double* w) {
  double q = 0.0;
  for (int i = 0; i < D; ++i) q += w[1 + i] * w[1 + i];
  return (gamma - 1.0) * (w[D + 1] - 0.5 * q / w[0]);
}

// Everything one face needs, Sections 2 and 4.
struct FaceWork {
  int D, nv;
  Maxw gl, gr, g0;
  double w0[5], al[5], ar[5], bl[2][5], br[2][5], Al[5], Ar[5], abl[5], abr[5], bb[2][5], Ab[5];
  double tau, T[7];
  double tauhat;  // rarefaction option: the resolved time scale rho / |D rho| at the face
  Poly Ql, Qr, Q0l, Q0r, Qt0, PAl, PAr, PAb;
};

bool face_setup(int D, double gamma, double mu, double C_a, double dt, int multid, int abar_mode,
                const orc_face& f, FaceWork& W, int rarefaction = 0) {
  const int nv = D + 2;
  const double K = 2.0 / (gamma - 1.0) - D;
  W.D = D;
  W.nv = nv;
  W.gl = make_maxw(D, K, f.wl);
  W.gr = make_maxw(D, K, f.wr);
  // Eq. intermediatestate: w0 = int_{u>0} psi g_l + int_{u<0} psi g_r
  for (int m = 0; m < nv; ++m)
    W.w0[m] = W.gl.rho * moment(W.gl, ORC_POS, psi(D, m)) + W.gr.rho * moment(W.gr, ORC_NEG, psi(D, m));
  W.g0 = make_maxw(D, K, W.w0);
  const double rl = W.gl.rho, rr = W.gr.rho, r0 = W.g0.rho;

  // Eq. initialf0: spatial coefficients from the conservative gradients, <a psi> = (1/rho) dW/dn
  double rhs[5];
  for (int m = 0; m < nv; ++m) rhs[m] = f.sl[m] / rl;
  slope(W.gl, rhs, W.al);
  for (int m = 0; m < nv; ++m) rhs[m] = f.sr[m] / rr;
  slope(W.gr, rhs, W.ar);
  for (int k = 0; k < 2; ++k)
    for (int m = 0; m < 5; ++m) W.bl[k][m] = W.br[k][m] = W.bb[k][m] = 0.0;
  if (multid) {
    for (int k = 0; k < D - 1; ++k) {
      for (int m = 0; m < nv; ++m) rhs[m] = f.tl[k][m] / rl;
      slope(W.gl, rhs, W.bl[k]);
      for (int m = 0; m < nv; ++m) rhs[m] = f.tr[k][m] / rr;
      slope(W.gr, rhs, W.br[k]);
    }
  }
  // Polynomials a u + sum_k b_k v_k of the initial state (f0 = g (1 + a x + b y - tau(a u + b v + A)))
  W.Ql = expansion(D, W.al) * pvar(0);
  W.Qr = expansion(D, W.ar) * pvar(0);
  for (int k = 0; k < D - 1; ++k) {
    W.Ql = W.Ql + expansion(D, W.bl[k]) * pvar(1 + k);
    W.Qr = W.Qr + expansion(D, W.br[k]) * pvar(1 + k);
  }
  // A from the compatibility condition at t = 0: <(a u + b v + A) psi> = 0
  for (int m = 0; m < nv; ++m) rhs[m] = -moment(W.gl, ORC_FULL, W.Ql * psi(D, m));
  slope(W.gl, rhs, W.Al);
  for (int m = 0; m < nv; ++m) rhs[m] = -moment(W.gr, ORC_FULL, W.Qr * psi(D, m));
  slope(W.gr, rhs, W.Ar);
  W.PAl = expansion(D, W.Al);
  W.PAr = expansion(D, W.Ar);

  // Eq. eqlgform: equilibrium slopes from the linear interpolation through W_j, w0, W_{j+1}
  for (int m = 0; m < nv; ++m) rhs[m] = (W.w0[m] - f.cl[m]) / (f.dxl * r0);
  slope(W.g0, rhs, W.abl);
  for (int m = 0; m < nv; ++m) rhs[m] = (f.cr[m] - W.w0[m]) / (f.dxr * r0);
  slope(W.g0, rhs, W.abr);
  if (multid) {
    for (int k = 0; k < D - 1; ++k) {
      for (int m = 0; m < nv; ++m) rhs[m] = 0.5 * (f.tl[k][m] + f.tr[k][m]) / r0;
      slope(W.g0, rhs, W.bb[k]);
    }
  }
  W.Q0l = expansion(D, W.abl) * pvar(0);
  W.Q0r = expansion(D, W.abr) * pvar(0);
  W.Qt0 = pconst(0.0);
  for (int k = 0; k < D - 1; ++k) W.Qt0 = W.Qt0 + expansion(D, W.bb[k]) * pvar(1 + k);

  // Eqs. relaxation time and taua: tau = mu/p + tau_t + C_a |p_r - p_l| / |p_r + p_l| dt
  double p0 = r0 / (2.0 * W.g0.lam);
  double pl = rl / (2.0 * W.gl.lam), pr = rr / (2.0 * W.gr.lam);
  W.tau = mu / p0 + f.tau_t + C_a * std::fabs(pr - pl) / std::fabs(pr + pl) * dt;
  W.tauhat = 0.0;
  if (rarefaction) {
    // Eqs. tautautilde, tautilde, epsilonkomega: the degree of rarefaction eps = tau / tauhat with
    // tauhat = rho / |D rho| at the face, D rho = d_t rho + U_n d_n rho (reading G9).  d_t rho is the
    // density row of the equilibrium time slope of the t = 0 compatibility condition
    // <(abar u + bbar v + A0) psi>_0 = 0; d_n rho that of the mean of the two normal slopes abar.
    double rhs0[5], A0[5], ab[5];
    for (int m = 0; m < nv; ++m) {
      Poly p = psi(D, m);
      rhs0[m] = -(moment(W.g0, ORC_POS, W.Q0l * p) + moment(W.g0, ORC_NEG, W.Q0r * p) +
                  moment(W.g0, ORC_FULL, W.Qt0 * p));
      ab[m] = 0.5 * (W.abl[m] + W.abr[m]);
    }
    slope(W.g0, rhs0, A0);
    const double dt_rho = r0 * moment(W.g0, ORC_FULL, expansion(D, A0) * psi(D, 0));
    const double dn_rho = r0 * moment(W.g0, ORC_FULL, expansion(D, ab) * psi(D, 0));
    const double Drho = std::fabs(dt_rho + W.g0.U[0] * dn_rho);
    W.tauhat = Drho > 1e-30 * r0 ? r0 / Drho : 1e30;  // uniform flow: tauhat -> infinity, eps -> 0
    time_coeffs_hat(dt, W.tau, W.tau / W.tauhat, W.T);
  } else {
    time_coeffs(dt, W.tau, W.T);
  }

  // Abar from the compatibility condition integrated over [0, dt] at the face:
  //   Dn <Abar psi>_0 = T1 <(abar u + bbar v) psi>_0 + T4 (rho_l <(a_l u + b_l v) psi>_{l,u>0}
  //                     + rho_r <...>_{r,u<0}) / rho0 + T5 (rho_l <A_l psi>_{l,u>0} + rho_r <...>) / rho0
  double X1[5], X4[5], X5[5];
  for (int m = 0; m < nv; ++m) {
    Poly p = psi(D, m);
    X1[m] = moment(W.g0, ORC_POS, W.Q0l * p) + moment(W.g0, ORC_NEG, W.Q0r * p) + moment(W.g0, ORC_FULL, W.Qt0 * p);
    X4[m] = (rl * moment(W.gl, ORC_POS, W.Ql * p) + rr * moment(W.gr, ORC_NEG, W.Qr * p)) / r0;
    X5[m] = (rl * moment(W.gl, ORC_POS, W.PAl * p) + rr * moment(W.gr, ORC_NEG, W.PAr * p)) / r0;
  }
  for (int m = 0; m < nv; ++m) {
    if (abar_mode == ORC_ABAR_T0 || W.tau == 0.0)
      rhs[m] = -X1[m];  // t = 0 compatibility, also the tau -> 0 limit of the integrated one
    else
      rhs[m] = (W.T[1] * X1[m] + W.T[4] * X4[m] + W.T[5] * X5[m]) / W.T[6];
  }
  slope(W.g0, rhs, W.Ab);
  W.PAb = expansion(D, W.Ab);
  return true;
}

void fill_diag(const FaceWork& W, orc_face_diag* dg) {
  if (!dg) return;
  std::memset(dg, 0, sizeof(*dg));
  for (int m = 0; m < W.nv; ++m) {
    dg->w0[m] = W.w0[m];
    dg->al[m] = W.al[m];
    dg->ar[m] = W.ar[m];
    dg->Al[m] = W.Al[m];
    dg->Ar[m] = W.Ar[m];
    dg->abl[m] = W.abl[m];
    dg->abr[m] = W.abr[m];
    dg->Ab[m] = W.Ab[m];
    for (int k = 0; k < 2; ++k) {
      dg->bl[k][m] = W.bl[k][m];
      dg->br[k][m] = W.br[k][m];
      dg->bb[k][m] = W.bb[k][m];
    }
  }
  dg->tau = W.tau;
  for (int i = 0; i < 6; ++i) dg->T[i] = W.T[i];
  dg->tauhat = W.tauhat;
}

// Eq. fluxesf: F = int_0^dt int u psi f dXi dt, with f from Eq. resultingf.
void face_flux(const FaceWork& W, double* F) {
  const int D = W.D;
  const Poly u = pvar(0);
  const double r0 = W.g0.rho, rl = W.gl.rho, rr = W.gr.rho;
  for (int m = 0; m < W.nv; ++m) {
    Poly up = u * psi(D, m);
    double eq = W.T[0] * moment(W.g0, ORC_FULL, up) +
                W.T[1] * (moment(W.g0, ORC_POS, W.Q0l * up) + moment(W.g0, ORC_NEG, W.Q0r * up) +
                          moment(W.g0, ORC_FULL, W.Qt0 * up)) +
                W.T[2] * moment(W.g0, ORC_FULL, W.PAb * up);
    double left = W.T[3] * moment(W.gl, ORC_POS, up) + W.T[4] * moment(W.gl, ORC_POS, W.Ql * up) +
                  W.T[5] * moment(W.gl, ORC_POS, W.PAl * up);
    double right = W.T[3] * moment(W.gr, ORC_NEG, up) + W.T[4] * moment(W.gr, ORC_NEG, W.Qr * up) +
                   W.T[5] * moment(W.gr, ORC_NEG, W.PAr * up);
    F[m] = r0 * eq + rl * left + rr * right;
  }
}

// ---------------------------------------------------------------------------------------------
// Grid machinery: SoA state [nv][nz][ny][nx]; a padded copy with two ghost layers per active axis.
// ---------------------------------------------------------------------------------------------
const int NGH = 3;  // ghost layers per side (the WENO-5 stencil reaches three cells)

struct Grid {
  int D, nv, n[3], N[3], g[3];
  long ncell, npad;
  std::vector<double> w[3];  // widths with ghosts, index i + 2
  long idx(int i, int j, int k) const {
    return ((long)(k + g[2]) * N[1] + (j + g[1])) * N[0] + (i + g[0]);
  }
};

Grid make_grid(const orc_problem* P) {
  Grid G;
  G.D = P->dim;
  G.nv = P->dim + 2;
  G.ncell = 1;
  G.npad = 1;
  for (int d = 0; d < 3; ++d) {
    bool act = d < P->dim;
    G.n[d] = act ? P->n[d] : 1;
    G.g[d] = act ? NGH : 0;
    G.N[d] = G.n[d] + 2 * G.g[d];
    G.ncell *= G.n[d];
    G.npad *= G.N[d];
    G.w[d].assign(G.n[d] + 2 * NGH, 1.0);
    if (act) {
      int n = G.n[d];
      for (int i = 0; i < n; ++i) G.w[d][i + NGH] = P->dx[d][i];
      bool per = P->bc[d][0] == ORC_BC_PERIODIC;
      for (int gi = 1; gi <= NGH; ++gi) {
        G.w[d][NGH - gi] = per ? P->dx[d][n - gi] : P->dx[d][std::min(gi - 1, n - 1)];
        G.w[d][n + NGH - 1 + gi] = per ? P->dx[d][gi - 1] : P->dx[d][std::max(n - gi, 0)];
      }
    }
  }
  return G;
}
double width(const Grid& G, int d, int i) { return G.w[d][i + NGH]; }

void cons_from_prim(int D, double gamma, const double* pr, double* w) {
  double q = 0.0;
  w[0] = pr[0];
  for (int i = 0; i < D; ++i) {
    w[1 + i] = pr[0] * pr[1 + i];
    q += pr[1 + i] * pr[1 + i];
  }
  w[D + 1] = pr[D + 1] / (gamma - 1.0) + 0.5 * pr[0] * q;
}
void prim_from_cons(int D, double gamma, const double* w, double* pr) {
  pr[0] = w[0];
  for (int i = 0; i < D; ++i) pr[1 + i] = w[1 + i] / w[0];
  pr[D + 1] = pressure(D, gamma, w);
}

// Ghost cells.  Axes are filled from the last to the first; when axis a is filled, lower axes
// range over interior cells and higher axes over the padded range, so corners take the lower
// axis' rule.  Wall: no-slip mirror with p_g = p_i and T_g = T_w^2 / T_i (T = p/rho), so that the
// geometric mean of the two temperatures is the wall temperature.
// Cell i of the j-lo side lies on the wake cut of a C-grid.
bool in_cut(const orc_problem* P, int i) {
  return P->wake_cut > 0 && i >= 0 && i < P->n[0] && (i < P->wake_cut || i >= P->n[0] - P->wake_cut);
}

void fill_ghosts(const orc_problem* P, const Grid& G, std::vector<double>& Wp) {
  const int D = G.D, nv = G.nv;
  for (int a = D - 1; a >= 0; --a) {
    int lo[3], hi[3];
    for (int b = 0; b < 3; ++b) {
      if (b < a) {
        lo[b] = 0;
        hi[b] = G.n[b];
      } else {
        lo[b] = -G.g[b];
        hi[b] = G.n[b] + G.g[b];
      }
    }
    const int n = G.n[a];
    for (int side = 0; side < 2; ++side) {
      int bc = P->bc[a][side];
      for (int gi = 1; gi <= NGH; ++gi) {
        int gidx = side == 0 ? -gi : n - 1 + gi;
        int c[3];
        for (c[2] = lo[2]; c[2] < hi[2]; ++c[2])
          for (c[1] = lo[1]; c[1] < hi[1]; ++c[1])
            for (c[0] = lo[0]; c[0] < hi[0]; ++c[0]) {
              if (c[a] != lo[a]) continue;  // iterate the transverse set once
              int dst[3] = {c[0], c[1], c[2]};
              dst[a] = gidx;
              int src[3] = {c[0], c[1], c[2]};
              double wv[5];
              if (D == 2 && a == 1 && side == 0 && in_cut(P, c[0])) {  // C-grid wake cut
                src[0] = P->n[0] - 1 - c[0];
                src[1] = gi - 1;
                for (int v = 0; v < nv; ++v) wv[v] = Wp[v * G.npad + G.idx(src[0], src[1], src[2])];
              } else if (bc == ORC_BC_PERIODIC) {
                src[a] = side == 0 ? n - gi : gi - 1;
                for (int v = 0; v < nv; ++v) wv[v] = Wp[v * G.npad + G.idx(src[0], src[1], src[2])];
              } else if (bc == ORC_BC_TRANSMISSIVE || bc == ORC_BC_OUTFLOW) {
                src[a] = side == 0 ? 0 : n - 1;
                for (int v = 0; v < nv; ++v) wv[v] = Wp[v * G.npad + G.idx(src[0], src[1], src[2])];
              } else if (bc == ORC_BC_WALL) {
                src[a] = side == 0 ? gi - 1 : n - gi;
                double wi[5], pri[5], prg[5];
                for (int v = 0; v < nv; ++v) wi[v] = Wp[v * G.npad + G.idx(src[0], src[1], src[2])];
                prim_from_cons(D, P->gamma, wi, pri);
                double Ti = pri[D + 1] / pri[0];
                double Tg = P->T_wall * P->T_wall / Ti;
                prg[D + 1] = pri[D + 1];
                prg[0] = pri[D + 1] / Tg;
                for (int i = 0; i < D; ++i) prg[1 + i] = -pri[1 + i];
                cons_from_prim(D, P->gamma, prg, wv);
              } else {  // Dirichlet: primitive state per boundary cell, transverse index clamped
                long off = 0, stride = 1;
                for (int b = 0; b < D; ++b) {
                  if (b == a) continue;
                  int cb = std::min(std::max(c[b], 0), G.n[b] - 1);
                  off += cb * stride;
                  stride *= G.n[b];
                }
                cons_from_prim(D, P->gamma, P->bc_prim[a][side] + off * nv, wv);
              }
              for (int v = 0; v < nv; ++v) Wp[v * G.npad + G.idx(dst[0], dst[1], dst[2])] = wv[v];
            }
      }
    }
  }
}

void pad_state(const Grid& G, const double* W, std::vector<double>& Wp) {
  Wp.assign((size_t)G.nv * G.npad, 0.0);
  for (int v = 0; v < G.nv; ++v)
    for (int k = 0; k < G.n[2]; ++k)
      for (int j = 0; j < G.n[1]; ++j)
        for (int i = 0; i < G.n[0]; ++i)
          Wp[v * G.npad + G.idx(i, j, k)] = W[v * G.ncell + ((long)k * G.n[1] + j) * G.n[0] + i];
}

// Turbulence fields with ghosts: periodic axes wrap, other axes repeat the nearest interior cell (a
// C-grid wake cut takes the cell across the cut).
std::vector<double> pad_scalar(const orc_problem* P, const Grid& G, const double* f) {
  std::vector<double> out(G.npad, 0.0);
  if (!f) return out;
  for (int k = -G.g[2]; k < G.n[2] + G.g[2]; ++k)
    for (int j = -G.g[1]; j < G.n[1] + G.g[1]; ++j)
      for (int i = -G.g[0]; i < G.n[0] + G.g[0]; ++i) {
        int c[3] = {i, j, k};
        if (G.D == 2 && j < 0 && in_cut(P, i)) {  // C-grid wake cut: the cell across the cut
          c[0] = G.n[0] - 1 - i;
          c[1] = -j - 1;
        } else {
          for (int d = 0; d < G.D; ++d) {
            int n = G.n[d];
            if (P->bc[d][0] == ORC_BC_PERIODIC)
              c[d] = (c[d] + n) % n;
            else
              c[d] = std::min(std::max(c[d], 0), n - 1);
          }
        }
        out[G.idx(i, j, k)] = f[((long)c[2] * G.n[1] + c[1]) * G.n[0] + c[0]];
      }
  return out;
}

void get_cell(const Grid& G, const std::vector<double>& Wp, int i, int j, int k, double* w) {
  long id = G.idx(i, j, k);
  for (int v = 0; v < G.nv; ++v) w[v] = Wp[v * G.npad + id];
}

// Velocity gradient by central differences; grad[a][b] = d U_b / d x_a
void vel_grad(const Grid& G, const std::vector<double>& Wp, int i, int j, int k, double grad[3][3]) {
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) grad[a][b] = 0.0;
  int c[3] = {i, j, k};
  for (int a = 0; a < G.D; ++a) {
    int cm[3] = {i, j, k}, cp[3] = {i, j, k};
    cm[a] -= 1;
    cp[a] += 1;
    double wm[5], wp[5];
    get_cell(G, Wp, cm[0], cm[1], cm[2], wm);
    get_cell(G, Wp, cp[0], cp[1], cp[2], wp);
    double dist = 0.5 * width(G, a, c[a] - 1) + width(G, a, c[a]) + 0.5 * width(G, a, c[a] + 1);
    for (int b = 0; b < G.D; ++b) grad[a][b] = (wp[1 + b] / wp[0] - wm[1 + b] / wm[0]) / dist;
  }
}

double strain_rate(const Grid& G, const std::vector<double>& Wp, int i, int j, int k) {
  double g[3][3];
  vel_grad(G, Wp, i, j, k, g);
  double s2 = 0.0;
  for (int a = 0; a < G.D; ++a)
    for (int b = 0; b < G.D; ++b) {
      double sab = 0.5 * (g[a][b] + g[b][a]);
      s2 += sab * sab;
    }
  return std::sqrt(2.0 * s2);
}

// Eqs. tauttrivial, tautchen and tautchenadjusted with T = p/rho (the turbulent part only).
double tau_turb_cell(const orc_problem* P, const Grid& G, const std::vector<double>& Wp,
                     const std::vector<double>& f1, const std::vector<double>& f2, int i, int j, int k) {
  if (P->turb_model == ORC_TURB_NONE) return 0.0;
  double w[5];
  get_cell(G, Wp, i, j, k, w);
  double rho = w[0], p = pressure(G.D, P->gamma, w);
  long id = G.idx(i, j, k);
  if (P->turb_model == ORC_TURB_MUT) return f1[id] / p;
  double S = strain_rate(G, Wp, i, j, k);
  double kk = f1[id], e2 = f2[id];
  if (!(kk > 0.0) || !(e2 > 0.0)) return 0.0;
  double nu_t, eta;
  if (P->turb_model == ORC_TURB_KEPS) {
    nu_t = P->C_mu * kk * kk / e2;
    eta = S * kk / e2;
  } else {
    nu_t = kk / e2;
    eta = S / (P->beta_star * e2);
  }
  return rho * nu_t / (p * std::sqrt(1.0 + eta * eta));
}

double limiter(int lim, double a, double b) {
  if (lim == ORC_LIM_MINMOD) {
    double sa = (a > 0) - (a < 0), sb = (b > 0) - (b < 0);
    return 0.5 * (sa + sb) * std::min(std::fabs(a), std::fabs(b));
  }
  // van Leer: (a b + |a b|) / (a + b), zero when a b <= 0
  return (a * b > 0.0) ? 2.0 * a * b / (a + b) : 0.0;
}

// Face values at the face between cells 0 and 1 of a stencil v[0..5] = cells -2 .. 3 (widths wd):
// wl is cell 0's value at that face, wr cell 1's.
//   MUSCL2: limited slopes over the centre distances, w = W +- h/2 s (the scheme's default).
//   MUSCL3: the kappa = 1/3 scheme in index space, each one-sided difference limited by minmod
//           against 4 times the other (the compression (3 - kappa)/(1 - kappa) of kappa = 1/3):
//           w_{j+1/2} = W_j + (1/6) minmod(D-, 4 D+) + (1/3) minmod(D+, 4 D-), mirrored for w_{j-1/2}.
//   WENO5:  Jiang and Shu's fifth-order weighted reconstruction in index space (linear weights
//           1/10, 6/10, 3/10; smoothness indicators with 13/12 and 1/4; epsilon 1e-6).
double weno5(double a, double b, double c, double d, double e) {  // value at the face right of c
  double q0 = (2.0 * a - 7.0 * b + 11.0 * c) / 6.0;
  double q1 = (-b + 5.0 * c + 2.0 * d) / 6.0;
  double q2 = (2.0 * c + 5.0 * d - e) / 6.0;
  double b0 = 13.0 / 12.0 * (a - 2.0 * b + c) * (a - 2.0 * b + c) + 0.25 * (a - 4.0 * b + 3.0 * c) * (a - 4.0 * b + 3.0 * c);
  double b1 = 13.0 / 12.0 * (b - 2.0 * c + d) * (b - 2.0 * c + d) + 0.25 * (b - d) * (b - d);
  double b2 = 13.0 / 12.0 * (c - 2.0 * d + e) * (c - 2.0 * d + e) + 0.25 * (3.0 * c - 4.0 * d + e) * (3.0 * c - 4.0 * d + e);
  const double eps = 1e-6;
  double a0 = 0.1 / ((eps + b0) * (eps + b0));
  double a1 = 0.6 / ((eps + b1) * (eps + b1));
  double a2 = 0.3 / ((eps + b2) * (eps + b2));
  return (a0 * q0 + a1 * q1 + a2 * q2) / (a0 + a1 + a2);
}

void recon_face(int recon, int lim, const double* v, const double* wd, double& wl, double& wr) {
  if (recon == ORC_RECON_WENO5) {
    wl = weno5(v[0], v[1], v[2], v[3], v[4]);
    wr = weno5(v[5], v[4], v[3], v[2], v[1]);
  } else if (recon == ORC_RECON_MUSCL3) {
    double dm = v[2] - v[1], dp = v[3] - v[2];  // cell 0
    wl = v[2] + limiter(ORC_LIM_MINMOD, dm, 4.0 * dp) / 6.0 + limiter(ORC_LIM_MINMOD, dp, 4.0 * dm) / 3.0;
    dm = v[3] - v[2];  // cell 1
    dp = v[4] - v[3];
    wr = v[3] - limiter(ORC_LIM_MINMOD, dp, 4.0 * dm) / 6.0 - limiter(ORC_LIM_MINMOD, dm, 4.0 * dp) / 3.0;
  } else {
    double dm = (v[2] - v[1]) / (0.5 * (wd[1] + wd[2]));
    double dc = (v[3] - v[2]) / (0.5 * (wd[2] + wd[3]));
    double dp = (v[4] - v[3]) / (0.5 * (wd[3] + wd[4]));
    wl = v[2] + 0.5 * wd[2] * limiter(lim, dm, dc);
    wr = v[3] - 0.5 * wd[3] * limiter(lim, dc, dp);
  }
}

void perm_for(int D, int d, int* perm) {
  if (D == 1) {
    perm[0] = 0;
  } else if (D == 2) {
    perm[0] = d;
    perm[1] = 1 - d;
  } else {
    perm[0] = d;
    perm[1] = d == 0 ? 1 : 0;
    perm[2] = d == 2 ? 1 : 2;
  }
}
void rotate(int D, const int* perm, const double* w, double* r) {
  r[0] = w[0];
  for (int k = 0; k < D; ++k) r[1 + k] = w[1 + perm[k]];
  r[D + 1] = w[D + 1];
}

struct StepCtx {
  const orc_problem* P;
  Grid G;
  std::vector<double> Wp, f1p, f2p, taut;  // taut on the padded index
};

void prepare(const orc_problem* P, const double* W, const double* f1, const double* f2, StepCtx& C) {
  C.P = P;
  C.G = make_grid(P);
  pad_state(C.G, W, C.Wp);
  fill_ghosts(P, C.G, C.Wp);
  C.f1p = pad_scalar(P, C.G, f1);
  C.f2p = pad_scalar(P, C.G, f2);
  C.taut.assign(C.G.npad, 0.0);
  const Grid& G = C.G;
  for (int k = -(G.g[2] / 2); k < G.n[2] + G.g[2] / 2; ++k)
    for (int j = -(G.g[1] / 2); j < G.n[1] + G.g[1] / 2; ++j)
      for (int i = -(G.g[0] / 2); i < G.n[0] + G.g[0] / 2; ++i)
        C.taut[G.idx(i, j, k)] = tau_turb_cell(P, G, C.Wp, C.f1p, C.f2p, i, j, k);
}

// Face record for the face between cell c (index j along axis d) and its + neighbour; *nfb (if
// given) receives the number of sides that fell back to first order.
void build_face(const StepCtx& C, int d, const int* c, orc_face& f, int* nfb = nullptr) {
  const Grid& G = C.G;
  const orc_problem* P = C.P;
  const int D = G.D, nv = G.nv;
  int perm[3];
  perm_for(D, d, perm);
  double S[6][5];  // cells j-2 .. j+3 along d (rotated)
  double wd[6];
  for (int s = 0; s < 6; ++s) {
    int cc[3] = {c[0], c[1], c[2]};
    cc[d] += s - 2;
    double w[5];
    get_cell(G, C.Wp, cc[0], cc[1], cc[2], w);
    rotate(D, perm, w, S[s]);
    wd[s] = width(G, d, cc[d]);
  }
  std::memset(&f, 0, sizeof(f));
  for (int v = 0; v < nv; ++v) {
    double st[6];
    for (int s = 0; s < 6; ++s) st[s] = S[s][v];
    recon_face(P->recon, P->limiter, st, wd, f.wl[v], f.wr[v]);
    // normal slopes of the two cells: the one-sided difference to the face value (for MUSCL2 this
    // is the limited slope itself)
    if (P->recon == ORC_RECON_MUSCL2) {
      double dm = (S[2][v] - S[1][v]) / (0.5 * (wd[1] + wd[2]));
      double dc = (S[3][v] - S[2][v]) / (0.5 * (wd[2] + wd[3]));
      double dp = (S[4][v] - S[3][v]) / (0.5 * (wd[3] + wd[4]));
      f.sl[v] = limiter(P->limiter, dm, dc);
      f.sr[v] = limiter(P->limiter, dc, dp);
    } else {
      f.sl[v] = (f.wl[v] - S[2][v]) / (0.5 * wd[2]);
      f.sr[v] = (S[3][v] - f.wr[v]) / (0.5 * wd[3]);
    }
    f.cl[v] = S[2][v];
    f.cr[v] = S[3][v];
  }
  // first order on a side whose reconstructed density or pressure is not positive
  const bool bad_l = !(f.wl[0] > 0.0) || !(pressure(D, P->gamma, f.wl) > 0.0);
  const bool bad_r = !(f.wr[0] > 0.0) || !(pressure(D, P->gamma, f.wr) > 0.0);
  if (nfb) *nfb = (int)bad_l + (int)bad_r;
  if (bad_l && !P->no_fallback)
    for (int v = 0; v < nv; ++v) {
      f.wl[v] = S[2][v];
      f.sl[v] = 0.0;
    }
  if (bad_r && !P->no_fallback)
    for (int v = 0; v < nv; ++v) {
      f.wr[v] = S[3][v];
      f.sr[v] = 0.0;
    }
  if (P->multid) {
    for (int t = 0; t < D - 1; ++t) {
      int ax = perm[1 + t];
      for (int side = 0; side < 2; ++side) {
        int cc[3] = {c[0], c[1], c[2]};
        cc[d] += side;
        double wm[5], w0[5], wp[5], rm[5], r0[5], rp[5];
        int cm[3] = {cc[0], cc[1], cc[2]}, cp[3] = {cc[0], cc[1], cc[2]};
        cm[ax] -= 1;
        cp[ax] += 1;
        get_cell(G, C.Wp, cm[0], cm[1], cm[2], wm);
        get_cell(G, C.Wp, cc[0], cc[1], cc[2], w0);
        get_cell(G, C.Wp, cp[0], cp[1], cp[2], wp);
        rotate(D, perm, wm, rm);
        rotate(D, perm, w0, r0);
        rotate(D, perm, wp, rp);
        double hm = 0.5 * (width(G, ax, cc[ax] - 1) + width(G, ax, cc[ax]));
        double hp = 0.5 * (width(G, ax, cc[ax]) + width(G, ax, cc[ax] + 1));
        for (int v = 0; v < nv; ++v) {
          double s = limiter(P->limiter, (r0[v] - rm[v]) / hm, (rp[v] - r0[v]) / hp);
          if (side == 0)
            f.tl[t][v] = s;
          else
            f.tr[t][v] = s;
        }
      }
    }
  }
  f.dxl = 0.5 * wd[2];
  f.dxr = 0.5 * wd[3];
  int cr[3] = {c[0], c[1], c[2]};
  cr[d] += 1;
  f.tau_t = 0.5 * (C.taut[G.idx(c[0], c[1], c[2])] + C.taut[G.idx(cr[0], cr[1], cr[2])]);
}

int flow_step(const orc_problem* P, double* W, const double* f1, const double* f2, double dt, double* resid,
              int nthreads, std::vector<double>* mflux);

}  // namespace

// =============================================================================================
// C API
// =============================================================================================
extern "C" {

int orc_umoments(double U, double lam, int region, int nmax, double* out) {
  if (nmax < 1 || nmax > 40) return 1;
  umom(U, lam, region, nmax, out);
  return 0;
}

int orc_ximoments(double K, double lam, int lmax, double* out) {
  ximom(K, lam, lmax, out);
  return 0;
}

int orc_time_coeffs(double dt, double tau, double* T) {
  time_coeffs(dt, tau, T);
  return 0;
}

int orc_time_coeffs_hat(double dt, double tau, double eps, double* T) {
  time_coeffs_hat(dt, tau, eps, T);
  return 0;
}

int orc_slope(int D, double K, const double* w, const double* rhs, double* a_out) {
  Maxw g = make_maxw(D, K, w);
  slope(g, rhs, a_out);
  return 0;
}

int orc_face_flux(int D, double gamma, double mu, double C_a, double dt, int multid, int abar_mode,
                  int rarefaction, const orc_face* f, double* F, orc_face_diag* diag) {
  FaceWork W;
  face_setup(D, gamma, mu, C_a, dt, multid, abar_mode, *f, W, rarefaction);
  face_flux(W, F);
  fill_diag(W, diag);
  return 0;
}

// Compact form, Eq. resultingf4 (test only): F = dt int u psi fhat with
//   fhat = f_c + 1/2 Abar dt g0 + alpha (f_u - f_c) + (alpha - beta) (f~_u - f~_c),
// alpha = eps (1 - e^{-1/eps}), eps = tau/dt, beta = e^{-1/eps} (or the printed eps e^{-1/eps}).
// Reading: f~_c = -tau (abar u + bbar v) g0 and f~_u = -tau (a u + b v) g_{l,r} carry only the
// spatial-expansion terms, and the time factor of Eq. resultingf2 is (t/tau) e^{-t/tau}; with the
// leading Maxwellians kept in f~ the form no longer equals the time integral of Eq. resultingf.
int orc_face_flux_compact(int D, double gamma, double mu, double C_a, double dt, int multid, int abar_mode,
                          int rarefaction, int printed_beta, const orc_face* f, double* F) {
  FaceWork W;
  face_setup(D, gamma, mu, C_a, dt, multid, abar_mode, *f, W, rarefaction);
  const Poly u = pvar(0);
  const double r0 = W.g0.rho, rl = W.gl.rho, rr = W.gr.rho, tau = W.tau;
  // the degree of rarefaction: tau/dt (Eq. epsilonkepsilon) or tau/tauhat (Eqs. rarefactionkepsilon,
  // epsilonkomega)
  double eps = rarefaction ? tau / W.tauhat : tau / dt;
  double ex = std::exp(-1.0 / eps);
  double alpha = eps * (1.0 - ex);
  double beta = printed_beta ? eps * ex : ex;
  for (int m = 0; m < W.nv; ++m) {
    Poly up = u * psi(D, m);
    double Cg = r0 * moment(W.g0, ORC_FULL, up);
    double Ca = r0 * (moment(W.g0, ORC_POS, W.Q0l * up) + moment(W.g0, ORC_NEG, W.Q0r * up) +
                      moment(W.g0, ORC_FULL, W.Qt0 * up));
    double CA = r0 * moment(W.g0, ORC_FULL, W.PAb * up);
    double Ug = rl * moment(W.gl, ORC_POS, up) + rr * moment(W.gr, ORC_NEG, up);
    double Ua = rl * moment(W.gl, ORC_POS, W.Ql * up) + rr * moment(W.gr, ORC_NEG, W.Qr * up);
    double UA = rl * moment(W.gl, ORC_POS, W.PAl * up) + rr * moment(W.gr, ORC_NEG, W.PAr * up);
    double fc = Cg - tau * (Ca + CA), fu = Ug - tau * (Ua + UA);
    double fct = -tau * Ca, fut = -tau * Ua;
    F[m] = dt * (fc + 0.5 * dt * CA + alpha * (fu - fc) + (alpha - beta) * (fut - fct));
  }
  return 0;
}

int orc_euler_flux(int D, double gamma, const double* w, double* F) {
  double p = pressure(D, gamma, w), un = w[1] / w[0];
  F[0] = w[1];
  for (int i = 0; i < D; ++i) F[1 + i] = w[1 + i] * un + (i == 0 ? p : 0.0);
  F[D + 1] = un * (w[D + 1] + p);
  return 0;
}

int orc_fallback_count(const orc_problem* P, const double* W, const double* f1, const double* f2, long* count) {
  StepCtx C;
  prepare(P, W, f1, f2, C);
  const Grid& G = C.G;
  long total = 0;
  for (int d = 0; d < G.D; ++d) {
    int nf[3] = {G.n[0], G.n[1], G.n[2]};
    nf[d] += 1;
    for (int k = 0; k < nf[2]; ++k)
      for (int j = 0; j < nf[1]; ++j)
        for (int i = 0; i < nf[0]; ++i) {
          int c[3] = {i, j, k};
          c[d] -= 1;  // left cell of the face
          orc_face f;
          int nfb = 0;
          build_face(C, d, c, f, &nfb);
          total += nfb;
        }
  }
  *count = total;
  return 0;
}

int orc_prim_to_cons(const orc_problem* P, const double* prim, double* W, long ncell) {
  int D = P->dim, nv = D + 2;
  for (long c = 0; c < ncell; ++c) {
    double pr[5], w[5];
    for (int v = 0; v < nv; ++v) pr[v] = prim[v * ncell + c];
    cons_from_prim(D, P->gamma, pr, w);
    for (int v = 0; v < nv; ++v) W[v * ncell + c] = w[v];
  }
  return 0;
}

int orc_cons_to_prim(const orc_problem* P, const double* W, double* prim, long ncell) {
  int D = P->dim, nv = D + 2;
  for (long c = 0; c < ncell; ++c) {
    double pr[5], w[5];
    for (int v = 0; v < nv; ++v) w[v] = W[v * ncell + c];
    prim_from_cons(D, P->gamma, w, pr);
    for (int v = 0; v < nv; ++v) prim[v * ncell + c] = pr[v];
  }
  return 0;
}

// CFL time step: dt = cfl / max_cells sum_d (|U_d| + c) / dx_d, c = sqrt(gamma p / rho)
int orc_compute_dt(const orc_problem* P, const double* W, double cfl, double* dt) {
  Grid G = make_grid(P);
  double rmax = 0.0;
  for (int k = 0; k < G.n[2]; ++k)
    for (int j = 0; j < G.n[1]; ++j)
      for (int i = 0; i < G.n[0]; ++i) {
        long c = ((long)k * G.n[1] + j) * G.n[0] + i;
        double w[5];
        for (int v = 0; v < G.nv; ++v) w[v] = W[v * G.ncell + c];
        double p = pressure(G.D, P->gamma, w);
        double cs = std::sqrt(P->gamma * p / w[0]);
        int ci[3] = {i, j, k};
        double r = 0.0;
        for (int d = 0; d < G.D; ++d) r += (std::fabs(w[1 + d] / w[0]) + cs) / width(G, d, ci[d]);
        rmax = std::max(rmax, r);
      }
  *dt = cfl / rmax;
  return 0;
}

int orc_tau_turb(const orc_problem* P, const double* W, const double* f1, const double* f2, double* tau_t) {
  StepCtx C;
  prepare(P, W, f1, f2, C);
  const Grid& G = C.G;
  for (int k = 0; k < G.n[2]; ++k)
    for (int j = 0; j < G.n[1]; ++j)
      for (int i = 0; i < G.n[0]; ++i) tau_t[((long)k * G.n[1] + j) * G.n[0] + i] = C.taut[G.idx(i, j, k)];
  return 0;
}

int orc_rarefaction(const orc_problem* P, const double* W, const double* f1, const double* f2, double* eps) {
  StepCtx C;
  prepare(P, W, f1, f2, C);
  const Grid& G = C.G;
  for (int k = 0; k < G.n[2]; ++k)
    for (int j = 0; j < G.n[1]; ++j)
      for (int i = 0; i < G.n[0]; ++i) {
        double g[3][3], w[5];
        vel_grad(G, C.Wp, i, j, k, g);
        get_cell(G, C.Wp, i, j, k, w);
        double div = 0.0;
        for (int a = 0; a < G.D; ++a) div += g[a][a];
        double tau = P->mu / pressure(G.D, P->gamma, w) + C.taut[G.idx(i, j, k)];
        eps[((long)k * G.n[1] + j) * G.n[0] + i] = tau * std::fabs(div);
      }
  return 0;
}

// One unsplit single-stage step W <- W - sum_d (F_{d,j+1/2} - F_{d,j-1/2}) / dx_d with the
// time-integrated fluxes of Eq. fluxesf.  Returns 4 if a cell ends with rho <= 0 or p <= 0.
int orc_step(const orc_problem* P, double* W, const double* f1, const double* f2, double dt,
             double* resid, int nthreads) {
  return flow_step(P, W, f1, f2, dt, resid, nthreads, nullptr);
}

}  // extern "C"

namespace {
// The flow step of orc_step; mflux (if given) receives, per axis d, the time-integrated mass flux of
// every face along d (faces j-1/2, j = 0 .. n_d, x fastest).
int flow_step(const orc_problem* P, double* W, const double* f1, const double* f2, double dt, double* resid,
              int nthreads, std::vector<double>* mflux) {
  StepCtx C;
  prepare(P, W, f1, f2, C);
  const Grid& G = C.G;
  const int D = G.D, nv = G.nv;
  std::vector<double> Wnew(W, W + (size_t)nv * G.ncell);
  for (int d = 0; d < D; ++d) {
    int nf[3] = {G.n[0], G.n[1], G.n[2]};
    nf[d] += 1;  // faces j+1/2 for j = -1 .. n-1
    long nfaces = (long)nf[0] * nf[1] * nf[2];
    std::vector<double> Fd((size_t)nfaces * nv);
    int perm[3];
    perm_for(D, d, perm);
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 64) num_threads(nthreads > 0 ? nthreads : 1)
#endif
    for (long fi = 0; fi < nfaces; ++fi) {
      int c[3];
      c[0] = (int)(fi % nf[0]);
      c[1] = (int)((fi / nf[0]) % nf[1]);
      c[2] = (int)(fi / ((long)nf[0] * nf[1]));
      c[d] -= 1;  // left cell of the face
      orc_face f;
      build_face(C, d, c, f);
      double Fr[5];
      FaceWork Wk;
      face_setup(D, P->gamma, P->mu, P->C_a, dt, P->multid, P->abar_mode, f, Wk, P->rarefaction);
      face_flux(Wk, Fr);
      double* Fo = &Fd[fi * nv];
      Fo[0] = Fr[0];
      for (int k = 0; k < D; ++k) Fo[1 + perm[k]] = Fr[1 + k];
      Fo[D + 1] = Fr[D + 1];
    }
    if (mflux) {
      mflux[d].resize(nfaces);
      for (long fi = 0; fi < nfaces; ++fi) mflux[d][fi] = Fd[fi * nv];
    }
    for (int k = 0; k < G.n[2]; ++k)
      for (int j = 0; j < G.n[1]; ++j)
        for (int i = 0; i < G.n[0]; ++i) {
          int c[3] = {i, j, k};
          int cp[3] = {i, j, k};
          cp[d] += 1;
          long fm = ((long)c[2] * nf[1] + c[1]) * nf[0] + c[0];
          long fp = ((long)cp[2] * nf[1] + cp[1]) * nf[0] + cp[0];
          double h = width(G, d, c[d]);
          long cell = ((long)k * G.n[1] + j) * G.n[0] + i;
          for (int v = 0; v < nv; ++v) Wnew[v * G.ncell + cell] -= (Fd[fp * nv + v] - Fd[fm * nv + v]) / h;
        }
  }
  int status = 0;
  for (int v = 0; v < nv && resid; ++v) resid[v] = resid[nv + v] = resid[2 * nv + v] = 0.0;
  for (long c = 0; c < G.ncell; ++c) {
    double w[5];
    for (int v = 0; v < nv; ++v) w[v] = Wnew[v * G.ncell + c];
    if (!(w[0] > 0.0) || !(pressure(D, P->gamma, w) > 0.0)) status = 4;
    if (resid) {
      int i = (int)(c % G.n[0]), j = (int)((c / G.n[0]) % G.n[1]), k = (int)(c / ((long)G.n[0] * G.n[1]));
      int ci[3] = {i, j, k};
      double vol = 1.0;
      for (int d = 0; d < D; ++d) vol *= width(G, d, ci[d]);
      for (int v = 0; v < nv; ++v) {
        double r = (w[v] - W[v * G.ncell + c]) / dt;
        resid[v] += r * r;
        resid[nv + v] = std::max(resid[nv + v], std::fabs(r));
        resid[2 * nv + v] += w[v] * vol;
      }
    }
  }
  if (resid)
    for (int v = 0; v < nv; ++v) resid[v] = std::sqrt(resid[v] / G.ncell);
  std::memcpy(W, Wnew.data(), sizeof(double) * nv * G.ncell);
  return status;
}

// ---------------------------------------------------------------------------------------------
// k-omega transport (Wilcox 2006), explicit in time with the flow step's dt:
//   d(rho k)/dt + div(rho U k)     = P - beta* rho k omega + div((mu + sigma* rho k / omega) grad k)
//   d(rho w)/dt + div(rho U w)     = alpha (omega/k) P - beta rho omega^2 + sigma_d (rho/omega) grad k . grad omega
//                                    + div((mu + sigma rho k / omega) grad omega)
//   P = rho tau_ij dU_i/dx_j = mu_T (2 S:S - 2/3 (div U)^2) - 2/3 rho k div U,
//   mu_T = rho k / omega~, omega~ = max(omega, C_lim sqrt(2 Sbar:Sbar / beta*)), Sbar = S - (div U)/3 I,
//   beta = beta0 f_beta, f_beta = (1 + 85 chi)/(1 + 100 chi), chi = |Omega_ij Omega_jk Shat_ki| / (beta* omega)^3,
//   Shat = S - (div U)/2 I, sigma_d = sigma_do where grad k . grad omega > 0, else 0.
// Discretisation (a reading; the paper gives none): convective flux F_rho * phi_face with F_rho the
// face's time-integrated GKS mass flux and phi_face the upwind cell's value plus half its limited
// slope times (width - F_rho / rho), the face value at the half time (MUSCL-Hancock, second order
// for smooth advection); diffusive flux dt (mu + sigma rho k / omega |face) (phi_R - phi_L) /
// (centre distance), the coefficient the mean of the two cells; gradients in the sources by
// central differences; destruction point-implicit:
//   (rho k)^{n+1} = [(rho k)^n - sum_d dG_d / dx_d + dt P] / (1 + dt beta* omega^n),
//   (rho w)^{n+1} = [(rho w)^n - sum_d dG_d / dx_d + dt (alpha rho (omega/omega~) X
//                    - 2/3 alpha rho omega div U + CD)] / (1 + dt beta omega^n),  X = 2 S:S - 2/3 (div U)^2,
// then rho k >= 0 and omega >= omega_floor.  Ghost values of k and omega: periodic axes wrap, other
// axes repeat the nearest interior cell (zero gradient).
// ---------------------------------------------------------------------------------------------
double central_grad(const Grid& G, const std::vector<double>& fp, int a, const int* c) {
  int cm[3] = {c[0], c[1], c[2]}, cp[3] = {c[0], c[1], c[2]};
  cm[a] -= 1;
  cp[a] += 1;
  double dist = 0.5 * width(G, a, c[a] - 1) + width(G, a, c[a]) + 0.5 * width(G, a, c[a] + 1);
  return (fp[G.idx(cp[0], cp[1], cp[2])] - fp[G.idx(cm[0], cm[1], cm[2])]) / dist;
}

void komega_update(const orc_problem* P, const orc_komega* K, const Grid& G, const std::vector<double>& Wp,
                   const std::vector<double>& kp, const std::vector<double>& wp, const std::vector<double>* mflux,
                   double dt, const double* RK, const double* RW, const double* Wnew, double* RKn, double* RWn) {
  const int D = G.D;
  // face fluxes G^k, G^omega per axis, faces j - 1/2 for j = 0 .. n_d
  std::vector<double> Gk[3], Gw[3];
  for (int d = 0; d < D; ++d) {
    int nf[3] = {G.n[0], G.n[1], G.n[2]};
    nf[d] += 1;
    long nfaces = (long)nf[0] * nf[1] * nf[2];
    Gk[d].assign(nfaces, 0.0);
    Gw[d].assign(nfaces, 0.0);
    for (long fi = 0; fi < nfaces; ++fi) {
      int cr[3];
      cr[0] = (int)(fi % nf[0]);
      cr[1] = (int)((fi / nf[0]) % nf[1]);
      cr[2] = (int)(fi / ((long)nf[0] * nf[1]));
      int cl[3] = {cr[0], cr[1], cr[2]};
      cl[d] -= 1;
      const double hl = width(G, d, cl[d]), hr = width(G, d, cr[d]);
      const double fr = mflux[d][fi];
      for (int q = 0; q < 2; ++q) {
        const std::vector<double>& f = q == 0 ? kp : wp;
        // limited slopes of the two cells along d
        double s[2], v[4];
        for (int t = 0; t < 4; ++t) {
          int cc[3] = {cl[0], cl[1], cl[2]};
          cc[d] += t - 1;
          v[t] = f[G.idx(cc[0], cc[1], cc[2])];
        }
        for (int side = 0; side < 2; ++side) {
          int c0 = cl[d] + side;
          double hm = 0.5 * (width(G, d, c0 - 1) + width(G, d, c0));
          double hp = 0.5 * (width(G, d, c0) + width(G, d, c0 + 1));
          s[side] = limiter(P->limiter, (v[1 + side] - v[side]) / hm, (v[2 + side] - v[1 + side]) / hp);
        }
        // upwind face value at the half time: the fluid crossing the face in dt comes from the
        // last F_rho / rho of the upwind cell (MUSCL-Hancock form)
        double rl0 = Wp[G.idx(cl[0], cl[1], cl[2])], rr0 = Wp[G.idx(cr[0], cr[1], cr[2])];
        double phiL = v[1] + 0.5 * s[0] * (hl - fr / rl0);
        double phiR = v[2] - 0.5 * s[1] * (hr + fr / rr0);
        double g = fr * (fr >= 0.0 ? phiL : phiR);
        if (K->diffusion) {
          double sig = q == 0 ? K->sigma_star : K->sigma;
          double rl = Wp[G.idx(cl[0], cl[1], cl[2])], rr = Wp[G.idx(cr[0], cr[1], cr[2])];
          double mdl = rl * kp[G.idx(cl[0], cl[1], cl[2])] / wp[G.idx(cl[0], cl[1], cl[2])];
          double mdr = rr * kp[G.idx(cr[0], cr[1], cr[2])] / wp[G.idx(cr[0], cr[1], cr[2])];
          double coef = P->mu + sig * 0.5 * (mdl + mdr);
          g -= dt * coef * (v[2] - v[1]) / (0.5 * hl + 0.5 * hr);
        }
        (q == 0 ? Gk : Gw)[d][fi] = g;
      }
    }
  }
  for (int k = 0; k < G.n[2]; ++k)
    for (int j = 0; j < G.n[1]; ++j)
      for (int i = 0; i < G.n[0]; ++i) {
        const int c[3] = {i, j, k};
        const long cell = ((long)k * G.n[1] + j) * G.n[0] + i;
        const long id = G.idx(i, j, k);
        double rho = Wp[id];
        double kk = kp[id], om = wp[id];
        double ak = RK[cell], aw = RW[cell];
        for (int d = 0; d < D; ++d) {
          int nf[3] = {G.n[0], G.n[1], G.n[2]};
          nf[d] += 1;
          int cp[3] = {i, j, k};
          cp[d] += 1;
          long fm = ((long)c[2] * nf[1] + c[1]) * nf[0] + c[0];
          long fp = ((long)cp[2] * nf[1] + cp[1]) * nf[0] + cp[0];
          double h = width(G, d, c[d]);
          ak -= (Gk[d][fp] - Gk[d][fm]) / h;
          aw -= (Gw[d][fp] - Gw[d][fm]) / h;
        }
        double rate_k = 0.0, rate_w = 0.0;
        if (K->sources) {
          double g[3][3];  // g[a][b] = dU_b/dx_a
          vel_grad(G, Wp, i, j, k, g);
          double div = 0.0;
          for (int a = 0; a < D; ++a) div += g[a][a];
          double SS = 0.0, SbSb = 0.0;
          double Sm[3][3], Om[3][3];
          for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) {
              Sm[a][b] = 0.5 * (g[a][b] + g[b][a]);
              Om[a][b] = 0.5 * (g[b][a] - g[a][b]);  // Omega_ab = (dU_a/dx_b - dU_b/dx_a)/2
            }
          for (int a = 0; a < D; ++a)
            for (int b = 0; b < D; ++b) {
              SS += Sm[a][b] * Sm[a][b];
              double sb = Sm[a][b] - (a == b ? div / 3.0 : 0.0);
              SbSb += sb * sb;
            }
          double X = 2.0 * SS - 2.0 / 3.0 * div * div;
          double wt = std::max(om, K->C_lim * std::sqrt(2.0 * SbSb / K->beta_star));
          double muT = rho * kk / wt;
          double Pk = muT * X - 2.0 / 3.0 * rho * kk * div;
          // vortex-stretching function (zero in 1D and 2D)
          double chi = 0.0;
          if (D == 3) {
            double t = 0.0;
            for (int a = 0; a < 3; ++a)
              for (int b = 0; b < 3; ++b)
                for (int e = 0; e < 3; ++e) {
                  double sh = Sm[e][a] - (e == a ? 0.5 * div : 0.0);
                  t += Om[a][b] * Om[b][e] * sh;
                }
            double bo = K->beta_star * om;
            chi = std::fabs(t / (bo * bo * bo));
          }
          double fbeta = (1.0 + 85.0 * chi) / (1.0 + 100.0 * chi);
          double beta = K->beta0 * fbeta;
          double dkdw = 0.0;
          for (int a = 0; a < D; ++a) dkdw += central_grad(G, kp, a, c) * central_grad(G, wp, a, c);
          double sd = dkdw > 0.0 ? K->sigma_do : 0.0;
          double CD = sd * rho / om * dkdw;
          ak += dt * Pk;
          aw += dt * (K->alpha * rho * (om / wt) * X - 2.0 / 3.0 * K->alpha * rho * om * div + CD);
          rate_k = K->beta_star * om;
          rate_w = beta * om;
        }
        ak /= 1.0 + dt * rate_k;
        aw /= 1.0 + dt * rate_w;
        double rho_new = Wnew[cell];
        RKn[cell] = std::max(ak, 0.0);
        RWn[cell] = std::max(aw, rho_new * K->omega_floor);
      }
}

// ---------------------------------------------------------------------------------------------
// Curvilinear 2D geometry
// ---------------------------------------------------------------------------------------------
struct CurvGeom {
  int n0, n1;
  bool convex;  // every cell a convex, counter-clockwise quadrilateral
  std::vector<double> area, cx, cy;        // cells, [j][i]
  std::vector<double> inx, iny, iL, imx, imy;  // i-faces (i = 0..n0, j = 0..n1-1), [j][i]
  std::vector<double> jnx, jny, jL, jmx, jmy;  // j-faces (i = 0..n0-1, j = 0..n1), [j][i]
  // centroids with two ghost layers per side, padded [j + 2][i + 2]
  std::vector<double> pcx, pcy;
  double nx(const double* nodes, int i, int j) const { return nodes[((long)j * (n0 + 1) + i) * 2]; }
  double ny(const double* nodes, int i, int j) const { return nodes[((long)j * (n0 + 1) + i) * 2 + 1]; }
  long pidx(int i, int j) const { return (long)(j + 2) * (n0 + 4) + (i + 2); }
};

CurvGeom curv_geometry(const orc_problem* P, const double* nodes) {
  CurvGeom g;
  const int n0 = P->n[0], n1 = P->n[1];
  g.n0 = n0;
  g.n1 = n1;
  g.area.resize((size_t)n0 * n1);
  g.cx.resize((size_t)n0 * n1);
  g.cy.resize((size_t)n0 * n1);
  g.convex = true;
  for (int j = 0; j < n1; ++j)
    for (int i = 0; i < n0; ++i) {
      const double x00 = g.nx(nodes, i, j), y00 = g.ny(nodes, i, j);
      const double x10 = g.nx(nodes, i + 1, j), y10 = g.ny(nodes, i + 1, j);
      const double x11 = g.nx(nodes, i + 1, j + 1), y11 = g.ny(nodes, i + 1, j + 1);
      const double x01 = g.nx(nodes, i, j + 1), y01 = g.ny(nodes, i, j + 1);
      const long c = (long)j * n0 + i;
      g.area[c] = 0.5 * ((x11 - x00) * (y01 - y10) - (x01 - x10) * (y11 - y00));  // > 0: right-handed
      // every corner of the quadrilateral (counter-clockwise 00, 10, 11, 01) turns left
      const double qx[4] = {x00, x10, x11, x01}, qy[4] = {y00, y10, y11, y01};
      for (int q = 0; q < 4; ++q) {
        const int a = (q + 3) % 4, b = (q + 1) % 4;
        if (!((qx[q] - qx[a]) * (qy[b] - qy[q]) - (qy[q] - qy[a]) * (qx[b] - qx[q]) > 0.0)) g.convex = false;
      }
      g.cx[c] = 0.25 * (x00 + x10 + x11 + x01);
      g.cy[c] = 0.25 * (y00 + y10 + y11 + y01);
    }
  g.inx.resize((size_t)(n0 + 1) * n1);
  g.iny.resize(g.inx.size());
  g.iL.resize(g.inx.size());
  g.imx.resize(g.inx.size());
  g.imy.resize(g.inx.size());
  for (int j = 0; j < n1; ++j)
    for (int i = 0; i <= n0; ++i) {
      const double ex = g.nx(nodes, i, j + 1) - g.nx(nodes, i, j), ey = g.ny(nodes, i, j + 1) - g.ny(nodes, i, j);
      const double L = std::sqrt(ex * ex + ey * ey);
      const long f = (long)j * (n0 + 1) + i;
      g.iL[f] = L;
      g.inx[f] = ey / L;
      g.iny[f] = -ex / L;
      g.imx[f] = 0.5 * (g.nx(nodes, i, j) + g.nx(nodes, i, j + 1));
      g.imy[f] = 0.5 * (g.ny(nodes, i, j) + g.ny(nodes, i, j + 1));
    }
  g.jnx.resize((size_t)n0 * (n1 + 1));
  g.jny.resize(g.jnx.size());
  g.jL.resize(g.jnx.size());
  g.jmx.resize(g.jnx.size());
  g.jmy.resize(g.jnx.size());
  for (int j = 0; j <= n1; ++j)
    for (int i = 0; i < n0; ++i) {
      const double ex = g.nx(nodes, i + 1, j) - g.nx(nodes, i, j), ey = g.ny(nodes, i + 1, j) - g.ny(nodes, i, j);
      const double L = std::sqrt(ex * ex + ey * ey);
      const long f = (long)j * n0 + i;
      g.jL[f] = L;
      g.jnx[f] = -ey / L;
      g.jny[f] = ex / L;
      g.jmx[f] = 0.5 * (g.nx(nodes, i, j) + g.nx(nodes, i + 1, j));
      g.jmy[f] = 0.5 * (g.ny(nodes, i, j) + g.ny(nodes, i + 1, j));
    }
  // centroids with ghosts: on a periodic axis a ghost is its source cell translated by the period
  // (the difference of the two boundary face midpoints), on other axes the mirror image of the
  // interior cell through the boundary face midpoint -- the positions the ghost widths of a
  // rectilinear grid give.  The i ghosts first, then the j ghosts, then the corners.
  g.pcx.assign((size_t)(n0 + 4) * (n1 + 4), 0.0);
  g.pcy.assign(g.pcx.size(), 0.0);
  for (int j = 0; j < n1; ++j)
    for (int i = 0; i < n0; ++i) {
      g.pcx[g.pidx(i, j)] = g.cx[(long)j * n0 + i];
      g.pcy[g.pidx(i, j)] = g.cy[(long)j * n0 + i];
    }
  const bool per0 = P->bc[0][0] == ORC_BC_PERIODIC, per1 = P->bc[1][0] == ORC_BC_PERIODIC;
  for (int j = 0; j < n1; ++j)
    for (int k = 1; k <= 2; ++k) {
      const long fl = (long)j * (n0 + 1), fr = (long)j * (n0 + 1) + n0;
      double* X[2] = {g.pcx.data(), g.pcy.data()};
      const double ml[2] = {g.imx[fl], g.imy[fl]}, mr[2] = {g.imx[fr], g.imy[fr]};
      for (int q = 0; q < 2; ++q) {
        if (per0) {
          X[q][g.pidx(-k, j)] = X[q][g.pidx(n0 - k, j)] + (ml[q] - mr[q]);
          X[q][g.pidx(n0 - 1 + k, j)] = X[q][g.pidx(k - 1, j)] + (mr[q] - ml[q]);
        } else {
          X[q][g.pidx(-k, j)] = 2.0 * ml[q] - X[q][g.pidx(k - 1, j)];
          X[q][g.pidx(n0 - 1 + k, j)] = 2.0 * mr[q] - X[q][g.pidx(n0 - k, j)];
        }
      }
    }
  for (int i = -2; i < n0 + 2; ++i)
    for (int k = 1; k <= 2; ++k) {
      const int ii = std::min(std::max(i, 0), n0 - 1);
      const long fb = ii, ft = (long)n1 * n0 + ii;
      double* X[2] = {g.pcx.data(), g.pcy.data()};
      const double mb[2] = {g.jmx[fb], g.jmy[fb]}, mt[2] = {g.jmx[ft], g.jmy[ft]};
      for (int q = 0; q < 2; ++q) {
        if (per1) {
          X[q][g.pidx(i, -k)] = X[q][g.pidx(i, n1 - k)] + (mb[q] - mt[q]);
          X[q][g.pidx(i, n1 - 1 + k)] = X[q][g.pidx(i, k - 1)] + (mt[q] - mb[q]);
        } else {
          X[q][g.pidx(i, -k)] = 2.0 * mb[q] - X[q][g.pidx(i, k - 1)];
          X[q][g.pidx(i, n1 - 1 + k)] = 2.0 * mt[q] - X[q][g.pidx(i, n1 - k)];
        }
        if (in_cut(P, i)) X[q][g.pidx(i, -k)] = X[q][g.pidx(n0 - 1 - i, k - 1)];  // the cell across the cut
      }
    }
  // corners (both indices outside): the parallelogram of the i ghost, the j ghost and their common
  // source cell, c(i, j) = c(i, js) + c(is, j) - c(is, js) (on a rectilinear grid the ghost widths'
  // corner; only the multi-dimensional expansion reaches corners)
  auto src_of = [](int c, int n, bool per) {
    const int k = c < 0 ? -c : c - n + 1;
    return per ? (c < 0 ? n - k : k - 1) : (c < 0 ? k - 1 : n - k);
  };
  for (int j = -2; j < n1 + 2; ++j)
    for (int i = -2; i < n0 + 2; ++i) {
      if ((i >= 0 && i < n0) || (j >= 0 && j < n1)) continue;
      const int is = src_of(i, n0, per0), js = src_of(j, n1, per1);
      g.pcx[g.pidx(i, j)] = g.pcx[g.pidx(i, js)] + g.pcx[g.pidx(is, j)] - g.pcx[g.pidx(is, js)];
      g.pcy[g.pidx(i, j)] = g.pcy[g.pidx(i, js)] + g.pcy[g.pidx(is, j)] - g.pcy[g.pidx(is, js)];
    }
  return g;
}

bool curv_valid(const CurvGeom& g) {
  if (!g.convex) return false;
  for (double a : g.area)
    if (!(a > 0.0)) return false;
  for (double L : g.iL)
    if (!(L > 0.0)) return false;
  for (double L : g.jL)
    if (!(L > 0.0)) return false;
  return true;
}

double cdist(const CurvGeom& g, int i0, int j0, int i1, int j1) {
  const double dx = g.pcx[g.pidx(i1, j1)] - g.pcx[g.pidx(i0, j0)], dy = g.pcy[g.pidx(i1, j1)] - g.pcy[g.pidx(i0, j0)];
  return std::sqrt(dx * dx + dy * dy);
}

// Everything a curvilinear step or steady residual needs: geometry, the state with ghost cells,
// tau_t per interior cell.
struct CurvCtx {
  const orc_problem* P;
  CurvGeom g;
  Grid G;
  std::vector<double> Wp, taut;
  // tau_t of a (possibly ghost) cell: a ghost cell takes its source cell's value
  double tau_of(int i, int j) const { return taut[src(i, j)]; }
  long src(int i, int j) const {  // source cell of a ghost (the cell itself inside)
    const int n0 = g.n0, n1 = g.n1;
    if (j < 0 && in_cut(P, i)) return (long)(-j - 1) * n0 + (n0 - 1 - i);  // across the wake cut
    if (P->bc[0][0] == ORC_BC_PERIODIC) i = (i + n0) % n0; else i = std::min(std::max(i, 0), n0 - 1);
    if (P->bc[1][0] == ORC_BC_PERIODIC) j = (j + n1) % n1; else j = std::min(std::max(j, 0), n1 - 1);
    return (long)j * n0 + i;
  }
};

int curv_prepare(const orc_problem* P, const double* nodes, const double* W, const double* f1, const double* f2,
                 CurvCtx& C) {
  if (P->dim != 2) return 1;
  C.P = P;
  C.g = curv_geometry(P, nodes);
  if (!curv_valid(C.g)) return 2;
  C.G = make_grid(P);
  const CurvGeom& g = C.g;
  const Grid& G = C.G;
  const int n0 = g.n0, n1 = g.n1;
  const long ncell = (long)n0 * n1;
  pad_state(G, W, C.Wp);
  fill_ghosts(P, G, C.Wp);
  const std::vector<double>& Wp = C.Wp;
  std::vector<double> f1p = pad_scalar(P, G, f1), f2p = pad_scalar(P, G, f2);
  // turbulent relaxation time per cell from Green-Gauss velocity gradients
  std::vector<double>& taut = C.taut;
  taut.assign(ncell, 0.0);
  if (P->turb_model != ORC_TURB_NONE) {
    for (int j = 0; j < n1; ++j)
      for (int i = 0; i < n0; ++i) {
        const long c = (long)j * n0 + i;
        double w[5];
        get_cell(G, Wp, i, j, 0, w);
        const double rho = w[0], p = pressure(2, P->gamma, w);
        const double kk = f1p[G.idx(i, j, 0)], e2 = f2p[G.idx(i, j, 0)];
        if (P->turb_model == ORC_TURB_MUT) {
          taut[c] = kk / p;
          continue;
        }
        if (!(kk > 0.0) || !(e2 > 0.0)) continue;
        double gr[2][2] = {{0, 0}, {0, 0}};  // gr[a][b] = dU_b/dx_a
        const int nb[4][2] = {{i - 1, j}, {i + 1, j}, {i, j - 1}, {i, j + 1}};
        const double sgn[4] = {-1.0, 1.0, -1.0, 1.0};
        const long fidx[4] = {(long)j * (n0 + 1) + i, (long)j * (n0 + 1) + i + 1, (long)j * n0 + i,
                              (long)(j + 1) * n0 + i};
        for (int q = 0; q < 4; ++q) {
          double wn[5];
          get_cell(G, Wp, nb[q][0], nb[q][1], 0, wn);
          const double nxq = q < 2 ? g.inx[fidx[q]] : g.jnx[fidx[q]], nyq = q < 2 ? g.iny[fidx[q]] : g.jny[fidx[q]];
          const double L = q < 2 ? g.iL[fidx[q]] : g.jL[fidx[q]];
          for (int b = 0; b < 2; ++b) {
            const double uf = 0.5 * (w[1 + b] / w[0] + wn[1 + b] / wn[0]);
            gr[0][b] += sgn[q] * uf * nxq * L;
            gr[1][b] += sgn[q] * uf * nyq * L;
          }
        }
        double s2 = 0.0;
        for (int a = 0; a < 2; ++a)
          for (int b = 0; b < 2; ++b) {
            const double sab = 0.5 * (gr[a][b] + gr[b][a]) / g.area[c];
            s2 += sab * sab;
          }
        const double S = std::sqrt(2.0 * s2);
        double nu_t, eta;
        if (P->turb_model == ORC_TURB_KEPS) {
          nu_t = P->C_mu * kk * kk / e2;
          eta = S * kk / e2;
        } else {
          nu_t = kk / e2;
          eta = S / (P->beta_star * e2);
        }
        taut[c] = rho * nu_t / (p * std::sqrt(1.0 + eta * eta));
      }
  }
  return 0;
}

// Time-integrated flux times face length of every face, per axis ([face][v], faces x fastest), over
// the window dt, or over the per-face windows win[0] (i-faces) and win[1] (j-faces) when win is
// given; first_order: no slopes (the cell averages on both sides).
void curv_fluxes(const CurvCtx& C, double dt, const std::vector<double>* win, bool first_order, int nthreads,
                 std::vector<double>& Fi, std::vector<double>& Fj) {
  const orc_problem* P = C.P;
  const CurvGeom& g = C.g;
  const Grid& G = C.G;
  const std::vector<double>& Wp = C.Wp;
  const int n0 = g.n0, n1 = g.n1, nv = 4;
  Fi.assign((size_t)(n0 + 1) * n1 * nv, 0.0);
  Fj.assign((size_t)n0 * (n1 + 1) * nv, 0.0);
  for (int d = 0; d < 2; ++d) {
    const int nf0 = d == 0 ? n0 + 1 : n0, nf1 = d == 0 ? n1 : n1 + 1;
    const long nfaces = (long)nf0 * nf1;
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 64) num_threads(nthreads > 0 ? nthreads : 1)
#endif
    for (long f = 0; f < nfaces; ++f) {
      const int fi = (int)(f % nf0), fj = (int)(f / nf0);
      const double nxf = d == 0 ? g.inx[f] : g.jnx[f], nyf = d == 0 ? g.iny[f] : g.jny[f];
      const double L = d == 0 ? g.iL[f] : g.jL[f];
      const double mx = d == 0 ? g.imx[f] : g.jmx[f], my = d == 0 ? g.imy[f] : g.jmy[f];
      // stencil cells s = 0..3: index (face index) - 2 + s along d
      int ci[4], cj[4];
      double S4[4][4];
      for (int s2 = 0; s2 < 4; ++s2) {
        ci[s2] = d == 0 ? fi - 2 + s2 : fi;
        cj[s2] = d == 0 ? fj : fj - 2 + s2;
        double w[5];
        get_cell(G, Wp, ci[s2], cj[s2], 0, w);
        S4[s2][0] = w[0];
        S4[s2][1] = w[1] * nxf + w[2] * nyf;   // rho u_n
        S4[s2][2] = -w[1] * nyf + w[2] * nxf;  // rho u_t, t = (-n_y, n_x)
        S4[s2][3] = w[3];
      }
      const double d01 = cdist(g, ci[0], cj[0], ci[1], cj[1]), d12 = cdist(g, ci[1], cj[1], ci[2], cj[2]);
      const double d23 = cdist(g, ci[2], cj[2], ci[3], cj[3]);
      const double dl = std::sqrt((mx - g.pcx[g.pidx(ci[1], cj[1])]) * (mx - g.pcx[g.pidx(ci[1], cj[1])]) +
                                  (my - g.pcy[g.pidx(ci[1], cj[1])]) * (my - g.pcy[g.pidx(ci[1], cj[1])]));
      const double dr = std::sqrt((mx - g.pcx[g.pidx(ci[2], cj[2])]) * (mx - g.pcx[g.pidx(ci[2], cj[2])]) +
                                  (my - g.pcy[g.pidx(ci[2], cj[2])]) * (my - g.pcy[g.pidx(ci[2], cj[2])]));
      orc_face fc;
      std::memset(&fc, 0, sizeof(fc));
      if (P->recon != ORC_RECON_MUSCL2 && !first_order) {
        // MUSCL-3 / WENO-5 along the grid line in index space on the six rotated cells
        // (face index) - 3 .. (face index) + 2; the normal slopes are the one-sided differences to
        // the face values over the centroid-to-face distances
        double S6[6][4];
        for (int s6 = 0; s6 < 6; ++s6) {
          const int ii = d == 0 ? fi - 3 + s6 : fi, jj = d == 0 ? fj : fj - 3 + s6;
          double w[5];
          get_cell(G, Wp, ii, jj, 0, w);
          S6[s6][0] = w[0];
          S6[s6][1] = w[1] * nxf + w[2] * nyf;
          S6[s6][2] = -w[1] * nyf + w[2] * nxf;
          S6[s6][3] = w[3];
        }
        const double unused[6] = {1.0, 1.0, 1.0, 1.0, 1.0, 1.0};
        for (int v = 0; v < nv; ++v) {
          double st[6];
          for (int s6 = 0; s6 < 6; ++s6) st[s6] = S6[s6][v];
          recon_face(P->recon, P->limiter, st, unused, fc.wl[v], fc.wr[v]);
          fc.sl[v] = (fc.wl[v] - S6[2][v]) / dl;
          fc.sr[v] = (S6[3][v] - fc.wr[v]) / dr;
          fc.cl[v] = S6[2][v];
          fc.cr[v] = S6[3][v];
        }
      } else {
        for (int v = 0; v < nv; ++v) {
          const double sl =
              first_order ? 0.0 : limiter(P->limiter, (S4[1][v] - S4[0][v]) / d01, (S4[2][v] - S4[1][v]) / d12);
          const double sr =
              first_order ? 0.0 : limiter(P->limiter, (S4[2][v] - S4[1][v]) / d12, (S4[3][v] - S4[2][v]) / d23);
          fc.sl[v] = sl;
          fc.sr[v] = sr;
          fc.wl[v] = S4[1][v] + dl * sl;
          fc.wr[v] = S4[2][v] - dr * sr;
          fc.cl[v] = S4[1][v];
          fc.cr[v] = S4[2][v];
        }
      }
      if (!(fc.wl[0] > 0.0) || !(pressure(2, P->gamma, fc.wl) > 0.0))
        for (int v = 0; v < nv; ++v) {
          fc.wl[v] = S4[1][v];
          fc.sl[v] = 0.0;
        }
      if (!(fc.wr[0] > 0.0) || !(pressure(2, P->gamma, fc.wr) > 0.0))
        for (int v = 0; v < nv; ++v) {
          fc.wr[v] = S4[2][v];
          fc.sr[v] = 0.0;
        }
      fc.dxl = dl;
      fc.dxr = dr;
      fc.tau_t = 0.5 * (C.tau_of(ci[1], cj[1]) + C.tau_of(ci[2], cj[2]));
      if (P->multid && !first_order) {
        // tangential slopes of the two cells in the face frame: limited differences along the
        // transverse grid line, each divided by the centroid step projected on the tangent
        // t = (-n_y, n_x)
        const double tx = -nyf, ty = nxf;
        for (int side = 0; side < 2; ++side) {
          const int i0 = ci[1 + side], j0 = cj[1 + side];
          int im = i0, jm = j0, ip = i0, jp = j0;
          if (d == 0) {
            jm -= 1;
            jp += 1;
          } else {
            im -= 1;
            ip += 1;
          }
          double rm[4], r0[4], rp[4];
          const int cc[3][2] = {{im, jm}, {i0, j0}, {ip, jp}};
          double* rr[3] = {rm, r0, rp};
          for (int q = 0; q < 3; ++q) {
            double w[5];
            get_cell(G, Wp, cc[q][0], cc[q][1], 0, w);
            rr[q][0] = w[0];
            rr[q][1] = w[1] * nxf + w[2] * nyf;
            rr[q][2] = -w[1] * nyf + w[2] * nxf;
            rr[q][3] = w[3];
          }
          auto proj = [&](int ia, int ja, int ib, int jb) {
            return (g.pcx[g.pidx(ib, jb)] - g.pcx[g.pidx(ia, ja)]) * tx + (g.pcy[g.pidx(ib, jb)] - g.pcy[g.pidx(ia, ja)]) * ty;
          };
          const double hm = proj(im, jm, i0, j0), hp = proj(i0, j0, ip, jp);
          for (int v = 0; v < nv; ++v) {
            const double s = limiter(P->limiter, (r0[v] - rm[v]) / hm, (rp[v] - r0[v]) / hp);
            if (side == 0)
              fc.tl[0][v] = s;
            else
              fc.tr[0][v] = s;
          }
        }
      }
      FaceWork Wk;
      face_setup(2, P->gamma, P->mu, P->C_a, win ? win[d][f] : dt, P->multid && !first_order ? 1 : 0, P->abar_mode,
                 fc, Wk, P->rarefaction);
      double Fr[4];
      face_flux(Wk, Fr);
      double* Fo = d == 0 ? &Fi[f * nv] : &Fj[f * nv];
      Fo[0] = Fr[0] * L;
      Fo[1] = (Fr[1] * nxf - Fr[2] * nyf) * L;
      Fo[2] = (Fr[1] * nyf + Fr[2] * nxf) * L;
      Fo[3] = Fr[3] * L;
    }
  }
}

// ---------------------------------------------------------------------------------------------
// Steady-state solver on curvilinear grids (Section 4: local time steps, LU-SGS smoothing in the
// form of Yoon and Jameson, multigrid after Jameson; the paper gives no formulas).  The readings:
//   - local explicit step s_i = 2 A_i / sum_faces (|U.n| + c) L (CFL 1); a face integrates its flux
//     over the window cfl_flux min(s_l, s_r) (a ghost cell has its source cell's step) and divides by
//     the window, so the steady operator does not depend on the pseudo-time step cfl s_i of the
//     smoother (the time-accurate flux carries terms of the order of its window: with the window tied
//     to a large pseudo-time step the iteration stalls);
//   - residual R_i = sum over the faces of that flux rate times L, outward; dW/dt = -R / A;
//   - LU-SGS on cell tiles (neighbours outside a tile enter neither sweep):
//       D_i dW*_i = -R_i - sum_{lower j} 1/2 (dF_j - lambda_ij dW*_j) L_ij,
//       dW_i = dW*_i - D_i^-1 sum_{upper j} 1/2 (dF_j - lambda_ij dW_j) L_ij,
//     D_i = A_i/dt_i + 1/2 sum_faces lambda L, dF_j = F_n(W_j + dW_j) - F_n(W_j) the change of the
//     Euler flux of cell j through the face with the normal pointing away from cell i, lower =
//     (i-1, j) and (i, j-1); lambda = max over the two cells of |U.n| + c, plus 2 (mu + p tau_t)/
//     (rho d) with face means of rho, p, tau_t and d the centroid distance;
//   - multigrid: every coarse grid takes every second node; restriction of the state by area
//     weights, of residuals by sums, of prescribed turbulence fields and Dirichlet data by plain
//     means; FAS forcing P_c = sum R_f - R_c(W_c^0); coarse residuals first order; one LU-SGS
//     smoothing per level on the way down, the corrections W_c - W_c^0 injected on the way up.
// ---------------------------------------------------------------------------------------------
void curv_lts(const CurvCtx& C, std::vector<double>& dtc) {
  const CurvGeom& g = C.g;
  const int n0 = g.n0, n1 = g.n1;
  dtc.assign((size_t)n0 * n1, 0.0);
  for (int j = 0; j < n1; ++j)
    for (int i = 0; i < n0; ++i) {
      const long c = (long)j * n0 + i;
      double w[5];
      get_cell(C.G, C.Wp, i, j, 0, w);
      const double p = pressure(2, C.P->gamma, w), cs = std::sqrt(C.P->gamma * p / w[0]);
      const double u = w[1] / w[0], v = w[2] / w[0];
      const long fi[2] = {(long)j * (n0 + 1) + i, (long)j * (n0 + 1) + i + 1};
      const long fj[2] = {(long)j * n0 + i, (long)(j + 1) * n0 + i};
      double r = 0.0;
      for (int s2 = 0; s2 < 2; ++s2) {
        r += (std::fabs(u * g.inx[fi[s2]] + v * g.iny[fi[s2]]) + cs) * g.iL[fi[s2]];
        r += (std::fabs(u * g.jnx[fj[s2]] + v * g.jny[fj[s2]]) + cs) * g.jL[fj[s2]];
      }
      dtc[c] = 2.0 * g.area[c] / r;
    }
}

void curv_residual(const CurvCtx& C, double cfl_flux, bool first_order, int nthreads, std::vector<double>& dtc,
                   std::vector<double>& R, std::vector<double>* mrate = nullptr) {
  const CurvGeom& g = C.g;
  const int n0 = g.n0, n1 = g.n1, nv = 4;
  const long ncell = (long)n0 * n1;
  curv_lts(C, dtc);
  std::vector<double> win[2];
  win[0].resize((size_t)(n0 + 1) * n1);
  win[1].resize((size_t)n0 * (n1 + 1));
  for (int j = 0; j < n1; ++j)
    for (int fi = 0; fi <= n0; ++fi)
      win[0][(long)j * (n0 + 1) + fi] = cfl_flux * std::min(dtc[C.src(fi - 1, j)], dtc[C.src(fi, j)]);
  for (int fj = 0; fj <= n1; ++fj)
    for (int i = 0; i < n0; ++i)
      win[1][(long)fj * n0 + i] = cfl_flux * std::min(dtc[C.src(i, fj - 1)], dtc[C.src(i, fj)]);
  std::vector<double> Fi, Fj;
  curv_fluxes(C, 0.0, win, first_order, nthreads, Fi, Fj);
  if (mrate)  // mass flux rate times L of every face, one array per axis
    for (int d = 0; d < 2; ++d) {
      const std::vector<double>& F = d == 0 ? Fi : Fj;
      mrate[d].resize(win[d].size());
      for (size_t f = 0; f < win[d].size(); ++f) mrate[d][f] = F[f * nv] / win[d][f];
    }
  R.assign((size_t)nv * ncell, 0.0);
  for (int j = 0; j < n1; ++j)
    for (int i = 0; i < n0; ++i) {
      const long c = (long)j * n0 + i;
      const long fa = (long)j * (n0 + 1) + i, fb = fa + 1, fc2 = (long)j * n0 + i, fd = (long)(j + 1) * n0 + i;
      for (int v = 0; v < nv; ++v)
        R[v * ncell + c] = Fi[fb * nv + v] / win[0][fb] - Fi[fa * nv + v] / win[0][fa] +
                           Fj[fd * nv + v] / win[1][fd] - Fj[fc2 * nv + v] / win[1][fc2];
    }
}

// Euler flux of state w through a face of unit normal (nx, ny).
void euler_normal(double gamma, const double* w, double nx, double ny, double* F) {
  const double un = (w[1] * nx + w[2] * ny) / w[0];
  const double p = pressure(2, gamma, w);
  F[0] = w[0] * un;
  F[1] = w[1] * un + p * nx;
  F[2] = w[2] * un + p * ny;
  F[3] = (w[3] + p) * un;
}

// Spectral radius of the face between cells (ia, ja) and (ib, jb) (b on the side the normal points to).
double face_lambda(const CurvCtx& C, double nx, double ny, double d, int ia, int ja, int ib, int jb) {
  const double gamma = C.P->gamma;
  double wa[5], wb[5];
  get_cell(C.G, C.Wp, ia, ja, 0, wa);
  get_cell(C.G, C.Wp, ib, jb, 0, wb);
  auto sr = [&](const double* w) {
    const double p = pressure(2, gamma, w);
    return std::fabs((w[1] * nx + w[2] * ny) / w[0]) + std::sqrt(gamma * p / w[0]);
  };
  const double rho = 0.5 * (wa[0] + wb[0]);
  const double p = 0.5 * (pressure(2, gamma, wa) + pressure(2, gamma, wb));
  const double tau = 0.5 * (C.tau_of(ia, ja) + C.tau_of(ib, jb));
  return std::max(sr(wa), sr(wb)) + 2.0 * (C.P->mu + p * tau) / (rho * d);
}

void curv_lusgs(const CurvCtx& C, const std::vector<double>& dtc, const std::vector<double>& R, int t0, int t1,
                std::vector<double>& dW) {
  const CurvGeom& g = C.g;
  const int n0 = g.n0, n1 = g.n1, nv = 4;
  const long ncell = (long)n0 * n1;
  const double gamma = C.P->gamma;
  // per face: lambda L / 2
  std::vector<double> hli((size_t)(n0 + 1) * n1), hlj((size_t)n0 * (n1 + 1));
  for (int j = 0; j < n1; ++j)
    for (int fi = 0; fi <= n0; ++fi) {
      const long f = (long)j * (n0 + 1) + fi;
      hli[f] = 0.5 * g.iL[f] * face_lambda(C, g.inx[f], g.iny[f], cdist(g, fi - 1, j, fi, j), fi - 1, j, fi, j);
    }
  for (int fj = 0; fj <= n1; ++fj)
    for (int i = 0; i < n0; ++i) {
      const long f = (long)fj * n0 + i;
      hlj[f] = 0.5 * g.jL[f] * face_lambda(C, g.jnx[f], g.jny[f], cdist(g, i, fj - 1, i, fj), i, fj - 1, i, fj);
    }
  std::vector<double> D(ncell);
  for (int j = 0; j < n1; ++j)
    for (int i = 0; i < n0; ++i) {
      const long c = (long)j * n0 + i;
      const long fa = (long)j * (n0 + 1) + i, fc2 = (long)j * n0 + i;
      D[c] = g.area[c] / dtc[c] + hli[fa] + hli[fa + 1] + hlj[fc2] + hlj[fc2 + n0];
    }
  dW.assign((size_t)nv * ncell, 0.0);
  std::vector<double> dWs((size_t)nv * ncell, 0.0);
  // contribution 1/2 (dF - lambda dX) L of neighbour (in, jn) through a face of normal +-n
  auto offdiag = [&](int in, int jn, double nx, double ny, double hl, double L, const std::vector<double>& X,
                     double* acc) {
    const long cn = (long)jn * n0 + in;
    double w[4], wp[4], F0[4], F1[4];
    for (int v = 0; v < nv; ++v) {
      w[v] = C.Wp[v * C.G.npad + C.G.idx(in, jn, 0)];
      wp[v] = w[v] + X[v * ncell + cn];
    }
    euler_normal(gamma, wp, nx, ny, F1);
    euler_normal(gamma, w, nx, ny, F0);
    for (int v = 0; v < nv; ++v) acc[v] += 0.5 * (F1[v] - F0[v]) * L - hl * X[v * ncell + cn];
  };
  for (int tj0 = 0; tj0 < n1; tj0 += t1)
    for (int ti0 = 0; ti0 < n0; ti0 += t0) {
      const int ti1 = std::min(ti0 + t0, n0), tj1 = std::min(tj0 + t1, n1);
      // forward sweep (lower neighbours inside the tile already done)
      for (int j = tj0; j < tj1; ++j)
        for (int i = ti0; i < ti1; ++i) {
          const long c = (long)j * n0 + i;
          double acc[4] = {0, 0, 0, 0};
          if (i > ti0) {
            const long f = (long)j * (n0 + 1) + i;  // face i - 1/2; normal away from cell i: -n
            offdiag(i - 1, j, -g.inx[f], -g.iny[f], hli[f], g.iL[f], dWs, acc);
          }
          if (j > tj0) {
            const long f = (long)j * n0 + i;
            offdiag(i, j - 1, -g.jnx[f], -g.jny[f], hlj[f], g.jL[f], dWs, acc);
          }
          for (int v = 0; v < nv; ++v) dWs[v * ncell + c] = (-R[v * ncell + c] - acc[v]) / D[c];
        }
      // backward sweep
      for (int j = tj1 - 1; j >= tj0; --j)
        for (int i = ti1 - 1; i >= ti0; --i) {
          const long c = (long)j * n0 + i;
          double acc[4] = {0, 0, 0, 0};
          if (i + 1 < ti1) {
            const long f = (long)j * (n0 + 1) + i + 1;
            offdiag(i + 1, j, g.inx[f], g.iny[f], hli[f], g.iL[f], dW, acc);
          }
          if (j + 1 < tj1) {
            const long f = (long)(j + 1) * n0 + i;
            offdiag(i, j + 1, g.jnx[f], g.jny[f], hlj[f], g.jL[f], dW, acc);
          }
          for (int v = 0; v < nv; ++v) dW[v * ncell + c] = dWs[v * ncell + c] - acc[v] / D[c];
        }
    }
}

// A coarse level: every second node, data restricted from the finer level.
struct Level {
  orc_problem P;
  std::vector<double> nodes, f1, f2;
  std::vector<double> dx[2];
  std::vector<double> bcp[2][2];
};

void coarsen(const Level& F, Level& Cl) {
  const int n0 = F.P.n[0], n1 = F.P.n[1], m0 = n0 / 2, m1 = n1 / 2;
  Cl.P = F.P;
  Cl.P.n[0] = m0;
  Cl.P.n[1] = m1;
  Cl.P.wake_cut = F.P.wake_cut / 2;
  Cl.nodes.resize((size_t)(m0 + 1) * (m1 + 1) * 2);
  for (int J = 0; J <= m1; ++J)
    for (int I = 0; I <= m0; ++I)
      for (int q = 0; q < 2; ++q)
        Cl.nodes[((long)J * (m0 + 1) + I) * 2 + q] = F.nodes[((long)(2 * J) * (n0 + 1) + 2 * I) * 2 + q];
  Cl.dx[0].assign(m0, 1.0);
  Cl.dx[1].assign(m1, 1.0);
  Cl.P.dx[0] = Cl.dx[0].data();
  Cl.P.dx[1] = Cl.dx[1].data();
  auto mean4 = [&](const std::vector<double>& f, std::vector<double>& out) {
    out.clear();
    if (f.empty()) return;
    out.resize((size_t)m0 * m1);
    for (int J = 0; J < m1; ++J)
      for (int I = 0; I < m0; ++I)
        out[(long)J * m0 + I] = 0.25 * (f[(long)(2 * J) * n0 + 2 * I] + f[(long)(2 * J) * n0 + 2 * I + 1] +
                                        f[(long)(2 * J + 1) * n0 + 2 * I] + f[(long)(2 * J + 1) * n0 + 2 * I + 1]);
  };
  mean4(F.f1, Cl.f1);
  mean4(F.f2, Cl.f2);
  for (int a = 0; a < 2; ++a)
    for (int s2 = 0; s2 < 2; ++s2) {
      Cl.P.bc_prim[a][s2] = nullptr;
      if (F.P.bc[a][s2] != ORC_BC_DIRICHLET || !F.P.bc_prim[a][s2]) continue;
      const int m = a == 0 ? m1 : m0;
      Cl.bcp[a][s2].resize((size_t)m * 4);
      for (int k = 0; k < m; ++k)
        for (int v = 0; v < 4; ++v)
          Cl.bcp[a][s2][k * 4 + v] = 0.5 * (F.P.bc_prim[a][s2][(2 * k) * 4 + v] + F.P.bc_prim[a][s2][(2 * k + 1) * 4 + v]);
      Cl.P.bc_prim[a][s2] = Cl.bcp[a][s2].data();
    }
}

const double* ptr_or_null(const std::vector<double>& v) { return v.empty() ? nullptr : v.data(); }

}  // namespace

extern "C" {

int orc_compute_dt_curv(const orc_problem* P, const double* nodes, const double* W, double cfl, double* dt) {
  if (P->dim != 2) return 1;
  const CurvGeom g = curv_geometry(P, nodes);
  if (!curv_valid(g)) return 2;
  const int n0 = g.n0, n1 = g.n1;
  const long ncell = (long)n0 * n1;
  double rmax = 0.0;
  for (int j = 0; j < n1; ++j)
    for (int i = 0; i < n0; ++i) {
      const long c = (long)j * n0 + i;
      double w[4];
      for (int v = 0; v < 4; ++v) w[v] = W[v * ncell + c];
      const double p = pressure(2, P->gamma, w), cs = std::sqrt(P->gamma * p / w[0]);
      const double u = w[1] / w[0], v = w[2] / w[0];
      const long fi[2] = {(long)j * (n0 + 1) + i, (long)j * (n0 + 1) + i + 1};
      const long fj[2] = {(long)j * n0 + i, (long)(j + 1) * n0 + i};
      double r = 0.0;
      for (int s = 0; s < 2; ++s) {
        r += (std::fabs(u * g.inx[fi[s]] + v * g.iny[fi[s]]) + cs) * g.iL[fi[s]];
        r += (std::fabs(u * g.jnx[fj[s]] + v * g.jny[fj[s]]) + cs) * g.jL[fj[s]];
      }
      rmax = std::max(rmax, r / (2.0 * g.area[c]));
    }
  *dt = cfl / rmax;
  return 0;
}

int orc_step_curv(const orc_problem* P, const double* nodes, double* W, const double* f1, const double* f2,
                  double dt, int nthreads) {
  CurvCtx C;
  const int st = curv_prepare(P, nodes, W, f1, f2, C);
  if (st) return st;
  const CurvGeom& g = C.g;
  const int n0 = g.n0, n1 = g.n1, nv = 4;
  const long ncell = (long)n0 * n1;
  std::vector<double> Fi, Fj;
  curv_fluxes(C, dt, nullptr, false, nthreads, Fi, Fj);
  int status = 0;
  for (int j = 0; j < n1; ++j)
    for (int i = 0; i < n0; ++i) {
      const long c = (long)j * n0 + i;
      const long fa = (long)j * (n0 + 1) + i, fb = fa + 1, fc2 = (long)j * n0 + i, fd = (long)(j + 1) * n0 + i;
      double w[4];
      for (int v = 0; v < nv; ++v) {
        W[v * ncell + c] -= (Fi[fb * nv + v] - Fi[fa * nv + v] + Fj[fd * nv + v] - Fj[fc2 * nv + v]) / g.area[c];
        w[v] = W[v * ncell + c];
      }
      if (!(w[0] > 0.0) || !(pressure(2, P->gamma, w) > 0.0)) status = 4;
    }
  return status;
}

// Wilcox's production terms of cell (i, j) on a curvilinear grid (destruction left to the caller):
// Sk = P_k, Sw = alpha (omega / omega~) rho X - 2/3 alpha rho omega div U + the cross diffusion, with
// Green-Gauss gradients of U, k and omega (face values the means of the two cells).
void kw_sources_curv(const orc_komega* K, const CurvGeom& g, const Grid& G, const std::vector<double>& Wp,
                     const std::vector<double>& kp, const std::vector<double>& wp, int i, int j, double& Sk,
                     double& Sw) {
  const int n0 = g.n0;
  const long c = (long)j * n0 + i, id = G.idx(i, j, 0);
  const long fa = (long)j * (n0 + 1) + i, fb = fa + 1, fc2 = (long)j * n0 + i, fd = (long)(j + 1) * n0 + i;
  const double A = g.area[c];
  double w[5];
  get_cell(G, Wp, i, j, 0, w);
  const double rho = w[0], k0 = kp[id], w0 = wp[id];
  // Green-Gauss gradients: velocity (gu[a][b] = dU_b/dx_a), k and omega
  double gu[2][2] = {{0, 0}, {0, 0}}, gk[2] = {0, 0}, gw[2] = {0, 0};
  const int nb[4][2] = {{i - 1, j}, {i + 1, j}, {i, j - 1}, {i, j + 1}};
  const double sgn[4] = {-1.0, 1.0, -1.0, 1.0};
  const long fid[4] = {fa, fb, fc2, fd};
  for (int q = 0; q < 4; ++q) {
    double wn[5];
    get_cell(G, Wp, nb[q][0], nb[q][1], 0, wn);
    const long nid = G.idx(nb[q][0], nb[q][1], 0);
    const double nx = q < 2 ? g.inx[fid[q]] : g.jnx[fid[q]], ny = q < 2 ? g.iny[fid[q]] : g.jny[fid[q]];
    const double L = q < 2 ? g.iL[fid[q]] : g.jL[fid[q]];
    const double sx = sgn[q] * nx * L, sy = sgn[q] * ny * L;
    for (int b = 0; b < 2; ++b) {
      const double uf = 0.5 * (w[1 + b] / w[0] + wn[1 + b] / wn[0]);
      gu[0][b] += uf * sx;
      gu[1][b] += uf * sy;
    }
    const double kf = 0.5 * (k0 + kp[nid]), wf = 0.5 * (w0 + wp[nid]);
    gk[0] += kf * sx;
    gk[1] += kf * sy;
    gw[0] += wf * sx;
    gw[1] += wf * sy;
  }
  for (int a = 0; a < 2; ++a) {
    gk[a] /= A;
    gw[a] /= A;
    for (int b = 0; b < 2; ++b) gu[a][b] /= A;
  }
  const double div = gu[0][0] + gu[1][1];
  double SS = 0.0, SbSb = 0.0;
  for (int a = 0; a < 2; ++a)
    for (int b = 0; b < 2; ++b) {
      const double sab = 0.5 * (gu[a][b] + gu[b][a]);
      SS += sab * sab;
      const double sb = sab - (a == b ? div / 3.0 : 0.0);
      SbSb += sb * sb;
    }
  const double X = 2.0 * SS - 2.0 / 3.0 * div * div;
  const double wt = std::max(w0, K->C_lim * std::sqrt(2.0 * SbSb / K->beta_star));
  const double muT = rho * k0 / wt;
  Sk = muT * X - 2.0 / 3.0 * rho * k0 * div;
  const double dkdw = gk[0] * gw[0] + gk[1] * gw[1];
  const double sd = dkdw > 0.0 ? K->sigma_do : 0.0;
  const double CD = sd * rho / w0 * dkdw;
  Sw = K->alpha * rho * (w0 / wt) * X - 2.0 / 3.0 * K->alpha * rho * w0 * div + CD;
}

// k-omega transport on a body-fitted grid (the rectilinear transport of orc_step_komega in each
// face's frame): the flow step with tau_t from k = rho k / rho and omega = rho omega / rho, then per
// face the convective flux F_rho * phi (F_rho the face's time-integrated mass flux times its length,
// phi the upwind cell's value plus its limited slope along the grid line times (centroid-to-face
// distance - F_rho / (2 rho L)), the half-time value) minus dt (mu + sigma rho k / omega |face)
// (phi_r - phi_l) / d12 L; per cell the divergence over the area, Wilcox's sources with
// Green-Gauss gradients (face values the means of the two cells) and the point-implicit destruction.
int orc_step_komega_curv(const orc_problem* P, const double* nodes, const orc_komega* K, double* W, double* RK,
                         double* RW, double dt, int nthreads) {
  if (P->turb_model != ORC_TURB_KOMEGA) return 1;
  const int n0 = P->n[0], n1 = P->n[1], nv = 4;
  const long ncell = (long)n0 * n1;
  std::vector<double> kk(ncell), om(ncell);
  for (long c = 0; c < ncell; ++c) {
    kk[c] = RK[c] / W[c];
    om[c] = RW[c] / W[c];
  }
  CurvCtx C;
  const int st0 = curv_prepare(P, nodes, W, kk.data(), om.data(), C);
  if (st0) return st0;
  const CurvGeom& g = C.g;
  const Grid& G = C.G;
  std::vector<double> Fi, Fj;
  curv_fluxes(C, dt, nullptr, false, nthreads, Fi, Fj);
  std::vector<double> Wnew(W, W + (size_t)nv * ncell);
  int status = 0;
  for (int j = 0; j < n1; ++j)
    for (int i = 0; i < n0; ++i) {
      const long c = (long)j * n0 + i;
      const long fa = (long)j * (n0 + 1) + i, fb = fa + 1, fc2 = (long)j * n0 + i, fd = (long)(j + 1) * n0 + i;
      double w[4];
      for (int v = 0; v < nv; ++v) {
        Wnew[v * ncell + c] -= (Fi[fb * nv + v] - Fi[fa * nv + v] + Fj[fd * nv + v] - Fj[fc2 * nv + v]) / g.area[c];
        w[v] = Wnew[v * ncell + c];
      }
      if (!(w[0] > 0.0) || !(pressure(2, P->gamma, w) > 0.0)) status = 4;
    }
  // the transport sees the state at the start of the step (with the flow's ghost cells)
  const std::vector<double>& Wp = C.Wp;
  std::vector<double> kp = pad_scalar(P, G, kk.data()), wp = pad_scalar(P, G, om.data());
  std::vector<double> Gk[2], Gw[2];
  for (int d = 0; d < 2; ++d) {
    const int nf0 = d == 0 ? n0 + 1 : n0, nf1 = d == 0 ? n1 : n1 + 1;
    const long nfaces = (long)nf0 * nf1;
    Gk[d].assign(nfaces, 0.0);
    Gw[d].assign(nfaces, 0.0);
    for (long f = 0; f < nfaces; ++f) {
      const int fi = (int)(f % nf0), fj = (int)(f / nf0);
      const double L = d == 0 ? g.iL[f] : g.jL[f];
      const double mx = d == 0 ? g.imx[f] : g.jmx[f], my = d == 0 ? g.imy[f] : g.jmy[f];
      int ci[4], cj[4];
      for (int t = 0; t < 4; ++t) {
        ci[t] = d == 0 ? fi - 2 + t : fi;
        cj[t] = d == 0 ? fj : fj - 2 + t;
      }
      const double d01 = cdist(g, ci[0], cj[0], ci[1], cj[1]), d12 = cdist(g, ci[1], cj[1], ci[2], cj[2]);
      const double d23 = cdist(g, ci[2], cj[2], ci[3], cj[3]);
      const double dl = std::hypot(mx - g.pcx[g.pidx(ci[1], cj[1])], my - g.pcy[g.pidx(ci[1], cj[1])]);
      const double dr = std::hypot(mx - g.pcx[g.pidx(ci[2], cj[2])], my - g.pcy[g.pidx(ci[2], cj[2])]);
      const double fr = (d == 0 ? Fi : Fj)[f * nv];
      const long il = G.idx(ci[1], cj[1], 0), ir = G.idx(ci[2], cj[2], 0);
      const double rl0 = Wp[il], rr0 = Wp[ir];
      for (int q = 0; q < 2; ++q) {
        const std::vector<double>& fp = q == 0 ? kp : wp;
        double v[4];
        for (int t = 0; t < 4; ++t) v[t] = fp[G.idx(ci[t], cj[t], 0)];
        const double s0 = limiter(P->limiter, (v[1] - v[0]) / d01, (v[2] - v[1]) / d12);
        const double s1 = limiter(P->limiter, (v[2] - v[1]) / d12, (v[3] - v[2]) / d23);
        const double phiL = v[1] + s0 * (dl - 0.5 * fr / (rl0 * L));
        const double phiR = v[2] - s1 * (dr + 0.5 * fr / (rr0 * L));
        double gq = fr * (fr >= 0.0 ? phiL : phiR);
        if (K->diffusion) {
          const double sig = q == 0 ? K->sigma_star : K->sigma;
          const double mdl = rl0 * kp[il] / wp[il], mdr = rr0 * kp[ir] / wp[ir];
          const double coef = P->mu + sig * 0.5 * (mdl + mdr);
          gq -= dt * coef * (v[2] - v[1]) / d12 * L;
        }
        (q == 0 ? Gk : Gw)[d][f] = gq;
      }
    }
  }
  for (int j = 0; j < n1; ++j)
    for (int i = 0; i < n0; ++i) {
      const long c = (long)j * n0 + i;
      const long id = G.idx(i, j, 0);
      const long fa = (long)j * (n0 + 1) + i, fb = fa + 1, fc2 = (long)j * n0 + i, fd = (long)(j + 1) * n0 + i;
      const double A = g.area[c];
      double ak = RK[c] - (Gk[0][fb] - Gk[0][fa] + Gk[1][fd] - Gk[1][fc2]) / A;
      double aw = RW[c] - (Gw[0][fb] - Gw[0][fa] + Gw[1][fd] - Gw[1][fc2]) / A;
      double rate_k = 0.0, rate_w = 0.0;
      if (K->sources) {
        double Sk, Sw;
        kw_sources_curv(K, g, G, Wp, kp, wp, i, j, Sk, Sw);
        ak += dt * Sk;
        aw += dt * Sw;
        rate_k = K->beta_star * wp[id];
        rate_w = K->beta0 * wp[id];  // the vortex-stretching factor is 1 in 2D
      }
      ak /= 1.0 + dt * rate_k;
      aw /= 1.0 + dt * rate_w;
      RK[c] = std::max(ak, 0.0);
      RW[c] = std::max(aw, Wnew[c] * K->omega_floor);
    }
  std::memcpy(W, Wnew.data(), sizeof(double) * Wnew.size());
  return status;
}

// Steady k-omega update on a body-fitted grid (the turbulence half of a steady cycle): from the
// state W and k = RK / rho, omega = RW / rho, the flow residual gives the face mass flux rates m (times
// L) and the local explicit steps; per face the rate G = m phi - (mu + sigma rho k / omega |face)
// (phi_r - phi_l) / d12 L, phi the upwind cell's value plus its limited slope along the grid line
// times the centroid-to-face distance; per cell the residual R = sum_faces G (outward) - A (S - beta
// omega RK) with Wilcox's production terms S, and one diagonal-implicit step RK -= R / D,
// D = A / (cfl dt_loc) + sum_faces (max(m_out, 0) + (mu + sigma rho k / omega |face) L / d12) / rho
// + A beta omega (beta = beta* for k, beta0 for omega), then the floors.
int orc_steady_komega(const orc_problem* P, const double* nodes, const orc_komega* K, const double* W, double* RK,
                      double* RW, double cfl, double cfl_flux, int nthreads) {
  if (P->turb_model != ORC_TURB_KOMEGA || P->dim != 2) return 1;
  const int n0 = P->n[0], n1 = P->n[1];
  const long ncell = (long)n0 * n1;
  std::vector<double> kk(ncell), om(ncell);
  for (long c = 0; c < ncell; ++c) {
    kk[c] = RK[c] / W[c];
    om[c] = RW[c] / W[c];
  }
  CurvCtx C;
  const int st0 = curv_prepare(P, nodes, W, kk.data(), om.data(), C);
  if (st0) return st0;
  const CurvGeom& g = C.g;
  const Grid& G = C.G;
  std::vector<double> dtc, R, mr[2];
  curv_residual(C, cfl_flux, false, nthreads, dtc, R, mr);
  const std::vector<double>& Wp = C.Wp;
  std::vector<double> kp = pad_scalar(P, G, kk.data()), wp = pad_scalar(P, G, om.data());
  // per face: the rates of rho k and rho omega and the diffusive conductances (mu + sigma ...) L / d12
  std::vector<double> Gk[2], Gw[2], Ck[2], Cw[2];
  for (int d = 0; d < 2; ++d) {
    const int nf0 = d == 0 ? n0 + 1 : n0, nf1 = d == 0 ? n1 : n1 + 1;
    const long nfaces = (long)nf0 * nf1;
    Gk[d].assign(nfaces, 0.0);
    Gw[d].assign(nfaces, 0.0);
    Ck[d].assign(nfaces, 0.0);
    Cw[d].assign(nfaces, 0.0);
    for (long f = 0; f < nfaces; ++f) {
      const int fi = (int)(f % nf0), fj = (int)(f / nf0);
      const double L = d == 0 ? g.iL[f] : g.jL[f];
      const double mx = d == 0 ? g.imx[f] : g.jmx[f], my = d == 0 ? g.imy[f] : g.jmy[f];
      int ci[4], cj[4];
      for (int t = 0; t < 4; ++t) {
        ci[t] = d == 0 ? fi - 2 + t : fi;
        cj[t] = d == 0 ? fj : fj - 2 + t;
      }
      const double d01 = cdist(g, ci[0], cj[0], ci[1], cj[1]), d12 = cdist(g, ci[1], cj[1], ci[2], cj[2]);
      const double d23 = cdist(g, ci[2], cj[2], ci[3], cj[3]);
      const double dl = std::hypot(mx - g.pcx[g.pidx(ci[1], cj[1])], my - g.pcy[g.pidx(ci[1], cj[1])]);
      const double dr = std::hypot(mx - g.pcx[g.pidx(ci[2], cj[2])], my - g.pcy[g.pidx(ci[2], cj[2])]);
      const double m = mr[d][f];
      const long il = G.idx(ci[1], cj[1], 0), ir = G.idx(ci[2], cj[2], 0);
      const double rl0 = Wp[il], rr0 = Wp[ir];
      for (int q = 0; q < 2; ++q) {
        const std::vector<double>& fp = q == 0 ? kp : wp;
        double v[4];
        for (int t = 0; t < 4; ++t) v[t] = fp[G.idx(ci[t], cj[t], 0)];
        const double s0 = limiter(P->limiter, (v[1] - v[0]) / d01, (v[2] - v[1]) / d12);
        const double s1 = limiter(P->limiter, (v[2] - v[1]) / d12, (v[3] - v[2]) / d23);
        const double phiL = v[1] + s0 * dl, phiR = v[2] - s1 * dr;
        double gq = m * (m >= 0.0 ? phiL : phiR);
        if (K->diffusion) {
          const double sig = q == 0 ? K->sigma_star : K->sigma;
          const double mdl = rl0 * kp[il] / wp[il], mdr = rr0 * kp[ir] / wp[ir];
          const double cond = (P->mu + sig * 0.5 * (mdl + mdr)) * L / d12;
          gq -= cond * (v[2] - v[1]);
          (q == 0 ? Ck : Cw)[d][f] = cond;
        }
        (q == 0 ? Gk : Gw)[d][f] = gq;
      }
    }
  }
  std::vector<double> RKn(RK, RK + ncell), RWn(RW, RW + ncell);
  for (int j = 0; j < n1; ++j)
    for (int i = 0; i < n0; ++i) {
      const long c = (long)j * n0 + i;
      const long id = G.idx(i, j, 0);
      const long fa = (long)j * (n0 + 1) + i, fb = fa + 1, fc2 = (long)j * n0 + i, fd = (long)(j + 1) * n0 + i;
      const double A = g.area[c], rho = W[c];
      double rk = Gk[0][fb] - Gk[0][fa] + Gk[1][fd] - Gk[1][fc2];
      double rw = Gw[0][fb] - Gw[0][fa] + Gw[1][fd] - Gw[1][fc2];
      // outward mass rates and conductances of the four faces
      const double mout[4] = {-mr[0][fa], mr[0][fb], -mr[1][fc2], mr[1][fd]};
      const double ck[4] = {Ck[0][fa], Ck[0][fb], Ck[1][fc2], Ck[1][fd]};
      const double cw[4] = {Cw[0][fa], Cw[0][fb], Cw[1][fc2], Cw[1][fd]};
      const double base = A / (cfl * dtc[c]);
      double Dk = 0.0, Dw = 0.0;
      for (int q = 0; q < 4; ++q) {
        Dk += std::max(mout[q], 0.0) + ck[q];
        Dw += std::max(mout[q], 0.0) + cw[q];
      }
      Dk = base + Dk / rho;
      Dw = base + Dw / rho;
      if (K->sources) {
        double Sk, Sw;
        kw_sources_curv(K, g, G, Wp, kp, wp, i, j, Sk, Sw);
        const double w0 = wp[id];
        rk -= A * (Sk - K->beta_star * w0 * RK[c]);
        rw -= A * (Sw - K->beta0 * w0 * RW[c]);
        Dk += A * K->beta_star * w0;
        Dw += A * K->beta0 * w0;
      }
      RKn[c] = std::max(RK[c] - rk / Dk, 0.0);
      RWn[c] = std::max(RW[c] - rw / Dw, rho * K->omega_floor);
    }
  std::memcpy(RK, RKn.data(), sizeof(double) * ncell);
  std::memcpy(RW, RWn.data(), sizeof(double) * ncell);
  return 0;
}

// Rarefaction diagnostic on a body-fitted grid (Eqs. tautautilde, tautilde with D rho = -rho div U):
// eps = (mu / p + tau_t) |div U| per cell, div U from Green-Gauss (face values the means of the two
// cells, ghost cells by the boundary rules).
int orc_rarefaction_curv(const orc_problem* P, const double* nodes, const double* W, const double* f1,
                         const double* f2, double* eps) {
  if (P->dim != 2) return 1;
  CurvCtx C;
  const int st = curv_prepare(P, nodes, W, f1, f2, C);
  if (st) return st;
  const CurvGeom& g = C.g;
  const Grid& G = C.G;
  const int n0 = g.n0, n1 = g.n1;
  for (int j = 0; j < n1; ++j)
    for (int i = 0; i < n0; ++i) {
      const long c = (long)j * n0 + i;
      double w[5];
      get_cell(G, C.Wp, i, j, 0, w);
      const int nb[4][2] = {{i - 1, j}, {i + 1, j}, {i, j - 1}, {i, j + 1}};
      const double sgn[4] = {-1.0, 1.0, -1.0, 1.0};
      const long fidx[4] = {(long)j * (n0 + 1) + i, (long)j * (n0 + 1) + i + 1, (long)j * n0 + i,
                            (long)(j + 1) * n0 + i};
      double div = 0.0;
      for (int q = 0; q < 4; ++q) {
        double wn[5];
        get_cell(G, C.Wp, nb[q][0], nb[q][1], 0, wn);
        const double nxq = q < 2 ? g.inx[fidx[q]] : g.jnx[fidx[q]], nyq = q < 2 ? g.iny[fidx[q]] : g.jny[fidx[q]];
        const double L = q < 2 ? g.iL[fidx[q]] : g.jL[fidx[q]];
        const double ux = 0.5 * (w[1] / w[0] + wn[1] / wn[0]), uy = 0.5 * (w[2] / w[0] + wn[2] / wn[0]);
        div += sgn[q] * (ux * nxq + uy * nyq) * L;
      }
      div /= g.area[c];
      eps[c] = (P->mu / pressure(2, P->gamma, w) + C.taut[c]) * std::fabs(div);
    }
  return 0;
}

int orc_steady_residual(const orc_problem* P, const double* nodes, const double* W, const double* f1,
                        const double* f2, double cfl_flux, int first_order, double* dt_cell, double* R, int nthreads) {
  CurvCtx C;
  const int st = curv_prepare(P, nodes, W, f1, f2, C);
  if (st) return st;
  std::vector<double> dtc, Rv;
  curv_residual(C, cfl_flux, first_order != 0, nthreads, dtc, Rv);
  if (dt_cell) std::memcpy(dt_cell, dtc.data(), sizeof(double) * dtc.size());
  if (R) std::memcpy(R, Rv.data(), sizeof(double) * Rv.size());
  return 0;
}

int orc_lusgs(const orc_problem* P, const double* nodes, const double* W, const double* f1, const double* f2,
              const double* dt_cell, const double* R, int tile0, int tile1, double* dW) {
  if (tile0 < 1 || tile1 < 1) return 1;
  CurvCtx C;
  const int st = curv_prepare(P, nodes, W, f1, f2, C);
  if (st) return st;
  const long ncell = (long)P->n[0] * P->n[1];
  std::vector<double> dtc(dt_cell, dt_cell + ncell), Rv(R, R + 4 * ncell), out;
  curv_lusgs(C, dtc, Rv, tile0, tile1, out);
  std::memcpy(dW, out.data(), sizeof(double) * out.size());
  return 0;
}

int orc_steady_cycle(const orc_problem* P, const double* nodes, double* W, const double* f1, const double* f2,
                     double cfl, double cfl_flux, int levels, int tile0, int tile1, int nthreads, double* res) {
  if (P->dim != 2 || levels < 1 || levels > 6) return 1;
  for (int l = 1; l < levels; ++l)
    if (P->n[0] % (1 << l) || P->n[1] % (1 << l) || P->wake_cut % (1 << l)) return 1;
  std::vector<Level> L(levels);
  L[0].P = *P;
  const int n0 = P->n[0], n1 = P->n[1];
  L[0].nodes.assign(nodes, nodes + (size_t)(n0 + 1) * (n1 + 1) * 2);
  if (f1) L[0].f1.assign(f1, f1 + (size_t)n0 * n1);
  if (f2) L[0].f2.assign(f2, f2 + (size_t)n0 * n1);
  for (int l = 1; l < levels; ++l) coarsen(L[l - 1], L[l]);
  std::vector<std::vector<double>> Ws(levels), W0(levels), Pf(levels);
  Ws[0].assign(W, W + (size_t)4 * n0 * n1);
  for (int l = 0; l < levels; ++l) {
    const orc_problem& Pl = L[l].P;
    const long nc = (long)Pl.n[0] * Pl.n[1];
    const bool fo = l > 0;
    CurvCtx C;
    int st = curv_prepare(&Pl, L[l].nodes.data(), Ws[l].data(), ptr_or_null(L[l].f1), ptr_or_null(L[l].f2), C);
    if (st) return st;
    std::vector<double> dtc, R;
    curv_residual(C, cfl_flux, fo, nthreads, dtc, R);
    for (double& d : dtc) d *= cfl;  // pseudo-time steps of the smoother
    if (l > 0)
      for (size_t q = 0; q < R.size(); ++q) R[q] += Pf[l][q];
    if (l == 0 && res) {
      double s2 = 0.0;
      for (long c = 0; c < nc; ++c) s2 += (R[c] / C.g.area[c]) * (R[c] / C.g.area[c]);
      *res = std::sqrt(s2 / nc);
    }
    std::vector<double> dW;
    curv_lusgs(C, dtc, R, tile0, tile1, dW);
    for (size_t q = 0; q < dW.size(); ++q) Ws[l][q] += dW[q];
    if (l + 1 == levels) break;
    // restriction to level l + 1: the state by area weights, the residual after smoothing by sums
    CurvCtx C2;
    st = curv_prepare(&Pl, L[l].nodes.data(), Ws[l].data(), ptr_or_null(L[l].f1), ptr_or_null(L[l].f2), C2);
    if (st) return st;
    std::vector<double> dt2, R2;
    curv_residual(C2, cfl_flux, fo, nthreads, dt2, R2);
    if (l > 0)
      for (size_t q = 0; q < R2.size(); ++q) R2[q] += Pf[l][q];
    const int m0 = Pl.n[0] / 2, m1 = Pl.n[1] / 2, k0 = Pl.n[0];
    const long mc = (long)m0 * m1;
    W0[l + 1].assign((size_t)4 * mc, 0.0);
    std::vector<double> Rs((size_t)4 * mc, 0.0);
    for (int J = 0; J < m1; ++J)
      for (int I = 0; I < m0; ++I) {
        const long cc = (long)J * m0 + I;
        double asum = 0.0;
        for (int q = 0; q < 4; ++q) {
          const long cf = (long)(2 * J + q / 2) * k0 + 2 * I + q % 2;
          asum += C2.g.area[cf];
          for (int v = 0; v < 4; ++v) {
            W0[l + 1][v * mc + cc] += C2.g.area[cf] * Ws[l][v * nc + cf];
            Rs[v * mc + cc] += R2[v * nc + cf];
          }
        }
        for (int v = 0; v < 4; ++v) W0[l + 1][v * mc + cc] /= asum;
      }
    Ws[l + 1] = W0[l + 1];
    CurvCtx C3;
    st = curv_prepare(&L[l + 1].P, L[l + 1].nodes.data(), W0[l + 1].data(), ptr_or_null(L[l + 1].f1),
                      ptr_or_null(L[l + 1].f2), C3);
    if (st) return st;
    std::vector<double> dt3, R3;
    curv_residual(C3, cfl_flux, true, nthreads, dt3, R3);
    Pf[l + 1].resize(R3.size());
    for (size_t q = 0; q < R3.size(); ++q) Pf[l + 1][q] = Rs[q] - R3[q];
  }
  // prolongation: inject the coarse corrections
  for (int l = levels - 1; l >= 1; --l) {
    const int m0 = L[l].P.n[0], m1 = L[l].P.n[1], k0 = L[l - 1].P.n[0];
    const long mc = (long)m0 * m1, nc = (long)k0 * L[l - 1].P.n[1];
    for (int J = 0; J < m1; ++J)
      for (int I = 0; I < m0; ++I) {
        const long cc = (long)J * m0 + I;
        for (int q = 0; q < 4; ++q) {
          const long cf = (long)(2 * J + q / 2) * k0 + 2 * I + q % 2;
          for (int v = 0; v < 4; ++v) Ws[l - 1][v * nc + cf] += Ws[l][v * mc + cc] - W0[l][v * mc + cc];
        }
      }
  }
  std::memcpy(W, Ws[0].data(), sizeof(double) * Ws[0].size());
  for (long q = 0; q < (long)n0 * n1; ++q) {
    double w[4] = {W[q], W[(long)n0 * n1 + q], W[2L * n0 * n1 + q], W[3L * n0 * n1 + q]};
    if (!(w[0] > 0.0) || !(pressure(2, P->gamma, w) > 0.0)) return 4;
  }
  return 0;
}

int orc_reconstruct(int recon, int limiter, const double* v, const double* h, int n, double* wl, double* wr) {
  if (n < 6) return 1;
  for (int j = 2; j + 3 < n; ++j) {  // face between cells j and j + 1
    double st[6], wd[6], a, b;
    for (int s = 0; s < 6; ++s) {
      st[s] = v[j - 2 + s];
      wd[s] = h[j - 2 + s];
    }
    recon_face(recon, limiter, st, wd, a, b);
    wl[j] = a;
    wr[j + 1] = b;
  }
  return 0;
}

int orc_komega_defaults(orc_komega* c) {
  c->alpha = 13.0 / 25.0;
  c->beta0 = 0.0708;
  c->beta_star = 0.09;
  c->sigma = 0.5;
  c->sigma_star = 0.6;
  c->sigma_do = 0.125;
  c->C_lim = 7.0 / 8.0;
  c->omega_floor = 1e-12;
  c->sources = 1;
  c->diffusion = 1;
  return 0;
}

int orc_step_komega(const orc_problem* P, const orc_komega* c, double* W, double* RK, double* RW, double dt,
                    int nthreads) {
  if (P->turb_model != ORC_TURB_KOMEGA) return 1;
  Grid G = make_grid(P);
  const long n = G.ncell;
  std::vector<double> kk(n), om(n), Wold(W, W + (size_t)G.nv * n);
  for (long i = 0; i < n; ++i) {
    kk[i] = RK[i] / W[i];
    om[i] = RW[i] / W[i];
  }
  std::vector<double> mflux[3];
  int status = flow_step(P, W, kk.data(), om.data(), dt, nullptr, nthreads, mflux);
  // the transport step sees the state at the start of the step (with the flow's ghost cells)
  std::vector<double> Wp;
  pad_state(G, Wold.data(), Wp);
  fill_ghosts(P, G, Wp);
  std::vector<double> kp = pad_scalar(P, G, kk.data()), wp = pad_scalar(P, G, om.data());
  std::vector<double> RKn(n), RWn(n);
  komega_update(P, c, G, Wp, kp, wp, mflux, dt, RK, RW, W, RKn.data(), RWn.data());
  std::memcpy(RK, RKn.data(), sizeof(double) * n);
  std::memcpy(RW, RWn.data(), sizeof(double) * n);
  return status;
}

// Steps with dt_fixed (> 0) or the CFL step, the last one clamped so that t_end (> 0) is met.
int orc_run(const orc_problem* P, double* W, const double* f1, const double* f2, double dt_fixed,
            double cfl, int nsteps, double t_end, double* t_inout, int* steps_done, int nthreads) {
  double t = t_inout ? *t_inout : 0.0;
  int done = 0, status = 0;
  for (int s = 0; s < nsteps; ++s) {
    double dt = dt_fixed;
    if (!(dt > 0.0)) orc_compute_dt(P, W, cfl, &dt);
    if (t_end > 0.0) {
      if (t >= t_end) break;
      dt = std::min(dt, t_end - t);
    }
    status = orc_step(P, W, f1, f2, dt, nullptr, nthreads);
    t += dt;
    ++done;
    if (status) break;
  }
  if (t_inout) *t_inout = t;
  if (steps_done) *steps_done = done;
  return status;
}

}  // extern "C"
