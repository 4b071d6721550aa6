// Per-interface BGK-Navier-Stokes flux of the gas-kinetic scheme (Righi 2013 Section 2, after
// Xu 2001), device code templated on the dimension D and the arithmetic type T.
//
// All quantities are in the frame of the face: velocity index 0 is the face normal (u), indices
// 1..D-1 the tangential directions (v, w).  Moments <.> are normalised by rho.  The Maxwellian of a
// state has lambda = rho/(2p) and K = bK - D internal degrees of freedom (bK = 2/(gamma-1)).
//
// The moment algebra is hand-expanded: half-line moments of u from erfc/exp (Eq. intermediatestate),
// tangential moments from the Gaussian recursion, slope coefficients from the closed-form
// inverse of the moment matrix, and the time integral of Eq. resultingf via T0..T5.
#pragma once
#ifndef GKS_HOST_COUNT
#include <cuda_runtime.h>
#endif
#include <math.h>

#ifndef GKS_FN
#define GKS_FN __device__ __forceinline__
#endif

namespace gks {

template <class T> GKS_FN T g_sqrt(T x);
template <> GKS_FN float g_sqrt<float>(float x) { return sqrtf(x); }
template <> GKS_FN double g_sqrt<double>(double x) { return sqrt(x); }
template <class T> GKS_FN T g_exp(T x);
template <> GKS_FN float g_exp<float>(float x) { return expf(x); }
template <> GKS_FN double g_exp<double>(double x) { return exp(x); }
template <class T> GKS_FN T g_erfc(T x);
template <> GKS_FN float g_erfc<float>(float x) { return erfcf(x); }
template <> GKS_FN double g_erfc<double>(double x) { return erfc(x); }
template <class T> GKS_FN T g_abs(T x) { return x < T(0) ? -x : x; }

constexpr double kInvSqrtPi = 0.56418958354775628695;  // 1/sqrt(pi)

template <int D> struct Dims {
  static constexpr int nv = D + 2;
  static constexpr int nt = D > 1 ? D - 1 : 1;  // storage for tangential arrays (>= 1)
};

// Macroscopic description of one Maxwellian.
template <int D, class T> struct Maxw {
  T rho, U[D], lam, il;  // il = 1/(2 lambda)
};

// Gas constants used by every face.
template <class T> struct Gas {
  T bK;   // K + D = 2/(gamma - 1)
  T K;    // internal degrees of freedom
  T mu;   // molecular viscosity (tau_mol = mu / p)
  T C_a;  // artificial-dissipation coefficient (Eq. taua)
};

// (rho, U, lambda) of the Maxwellian carrying the conservative state w (Section 2: E = (u^2 + xi^2)/2,
// so rho E = rho |U|^2 / 2 + bK rho / (4 lambda)).
template <int D, class T>
GKS_FN Maxw<D, T> maxwellian(const T* w, T bK) {
  Maxw<D, T> g;
  g.rho = w[0];
  T q = T(0);
#pragma unroll
  for (int i = 0; i < D; ++i) {
    g.U[i] = w[1 + i] / w[0];
    q += g.U[i] * g.U[i];
  }
  g.lam = bK * w[0] / (T(4) * (w[D + 1] - T(0.5) * w[0] * q));
  g.il = T(0.5) / g.lam;
  return g;
}

// Moment tables of one Maxwellian restricted to one region of the normal velocity.
//   u[n] = <u^n> (n <= 6) over the region, v[t][n] = <v_t^n> (n <= 5) over the full line,
//   x[l] = <(xi^2)^l> (l <= 2).
template <int D, class T> struct Tab {
  T u[7];
  T v[Dims<D>::nt][6];
  T x[3];
};

template <int N, class T>
GKS_FN void recur(T U, T il, T* m) {
#pragma unroll
  for (int n = 0; n + 2 < N; ++n) m[n + 2] = U * m[n + 1] + T(n + 1) * il * m[n];
}

template <int D, class T>
GKS_FN void tang_and_xi(const Maxw<D, T>& g, T K, Tab<D, T>& t) {
#pragma unroll
  for (int s = 0; s < D - 1; ++s) {
    t.v[s][0] = T(1);
    t.v[s][1] = g.U[1 + s];
    recur<6>(g.U[1 + s], g.il, t.v[s]);
  }
  t.x[0] = T(1);
  t.x[1] = K * g.il;
  t.x[2] = K * (K + T(2)) * g.il * g.il;
}

// Full-line table.
template <int D, class T>
GKS_FN void tab_full(const Maxw<D, T>& g, T K, Tab<D, T>& t) {
  t.u[0] = T(1);
  t.u[1] = g.U[0];
  recur<7>(g.U[0], g.il, t.u);
  tang_and_xi(g, K, t);
}

// Half-line tables u > 0 (P) and u < 0 (N) from one erfc and one exp:
//   <1>_{u>0} = erfc(-sqrt(lam) U)/2, <u>_{u>0} = U <1>_{u>0} + exp(-lam U^2)/(2 sqrt(pi lam)).
template <int D, class T>
GKS_FN void tab_half(const Maxw<D, T>& g, T K, Tab<D, T>* P, Tab<D, T>* N) {
  const T sl = g_sqrt(g.lam);
  const T z = sl * g.U[0];
  const T h = T(0.5) * g_exp(-z * z) * T(kInvSqrtPi) / sl;
  if (P) {
    P->u[0] = T(0.5) * g_erfc(-z);
    P->u[1] = g.U[0] * P->u[0] + h;
    recur<7>(g.U[0], g.il, P->u);
    tang_and_xi(g, K, *P);
  }
  if (N) {
    N->u[0] = T(0.5) * g_erfc(z);
    N->u[1] = g.U[0] * N->u[0] - h;
    recur<7>(g.U[0], g.il, N->u);
    tang_and_xi(g, K, *N);
  }
}

// <u^a v^b0 w^b1 (xi^2)^l>
template <int D, class T>
GKS_FN T mono(const Tab<D, T>& t, int a, int b0, int b1, int l) {
  T r = t.u[a];
  if (D >= 2) r = r * t.v[0][b0];
  if (D >= 3) r = r * t.v[D >= 3 ? 1 : 0][b1];
  return r * t.x[l];
}

// out[m] = <u^a v^b0 w^b1 (xi^2)^l psi_m>, psi = (1, u, v, w, (u^2 + v^2 + w^2 + xi^2)/2)
template <int D, class T>
GKS_FN void psi_mom(const Tab<D, T>& t, int a, int b0, int b1, int l, T* out) {
  out[0] = mono(t, a, b0, b1, l);
  out[1] = mono(t, a + 1, b0, b1, l);
  if (D >= 2) out[2] = mono(t, a, b0 + 1, b1, l);
  if (D >= 3) out[3] = mono(t, a, b0, b1 + 1, l);
  T e = mono(t, a + 2, b0, b1, l) + mono(t, a, b0, b1, l + 1);
  if (D >= 2) e += mono(t, a, b0 + 2, b1, l);
  if (D >= 3) e += mono(t, a, b0, b1 + 2, l);
  out[D + 1] = T(0.5) * e;
}

// acc[m] += s * <u^a v_j^(j == tj) (a . psi) psi_m>, tj = -1 for no tangential factor.
template <int D, class T>
GKS_FN void amom(const Tab<D, T>& t, int a, int tj, const T* c, T s, T* acc) {
  constexpr int nv = D + 2;
  const int b0 = (tj == 0) ? 1 : 0, b1 = (tj == 1) ? 1 : 0;
  T r[nv], q[nv];
  psi_mom<D, T>(t, a, b0, b1, 0, r);  // c0 * 1
#pragma unroll
  for (int m = 0; m < nv; ++m) q[m] = c[0] * r[m];
  psi_mom<D, T>(t, a + 1, b0, b1, 0, r);  // c1 * u
#pragma unroll
  for (int m = 0; m < nv; ++m) q[m] += c[1] * r[m];
  if (D >= 2) {
    psi_mom<D, T>(t, a, b0 + 1, b1, 0, r);
#pragma unroll
    for (int m = 0; m < nv; ++m) q[m] += c[2] * r[m];
  }
  if (D >= 3) {
    psi_mom<D, T>(t, a, b0, b1 + 1, 0, r);
#pragma unroll
    for (int m = 0; m < nv; ++m) q[m] += c[3] * r[m];
  }
  // cE * (u^2 + v^2 + w^2 + xi^2) / 2
  T e[nv];
  psi_mom<D, T>(t, a + 2, b0, b1, 0, e);
  psi_mom<D, T>(t, a, b0, b1, 1, r);
#pragma unroll
  for (int m = 0; m < nv; ++m) e[m] += r[m];
  if (D >= 2) {
    psi_mom<D, T>(t, a, b0 + 2, b1, 0, r);
#pragma unroll
    for (int m = 0; m < nv; ++m) e[m] += r[m];
  }
  if (D >= 3) {
    psi_mom<D, T>(t, a, b0, b1 + 2, 0, r);
#pragma unroll
    for (int m = 0; m < nv; ++m) e[m] += r[m];
  }
  const T hE = T(0.5) * c[D + 1];
#pragma unroll
  for (int m = 0; m < nv; ++m) acc[m] += s * (q[m] + hE * e[m]);
}

enum { LIM_MINMOD = 0, LIM_VANLEER = 1 };

// Slope limiter on one conservative variable: minmod(a, b) = (sgn a + sgn b)/2 min(|a|, |b|), or
// van Leer (a b + |a b|)/(a + b), zero unless a b > 0.
template <class R>
GKS_FN R limiter(int lim, R a, R b) {
  if (lim == LIM_MINMOD) {
    const R sa = R((a > R(0)) - (a < R(0))), sb = R((b > R(0)) - (b < R(0)));
    const R ma = g_abs(a), mb = g_abs(b);
    return R(0.5) * (sa + sb) * (ma < mb ? ma : mb);
  }
  return (a * b > R(0)) ? R(2) * a * b / (a + b) : R(0);
}

// MUSCL on one variable at the face between cells 1 and 2 of the stencil s0..s3 with widths
// h0..h3: limited slopes of cells 1 and 2 and the face values left and right.
template <class R>
GKS_FN void muscl(int lim, R s0, R s1, R s2, R s3, R h0, R h1, R h2, R h3, R& wl, R& wr, R& sl, R& sr) {
  const R dm = (s1 - s0) / (R(0.5) * (h0 + h1));
  const R dc = (s2 - s1) / (R(0.5) * (h1 + h2));
  const R dp = (s3 - s2) / (R(0.5) * (h2 + h3));
  sl = limiter<R>(lim, dm, dc);
  sr = limiter<R>(lim, dc, dp);
  wl = s1 + R(0.5) * h1 * sl;
  wr = s2 - R(0.5) * h2 * sr;
}

// Coefficients a of a . psi with <(a . psi) psi> = rhs (already divided by rho): closed-form inverse
// of the Maxwellian moment matrix.
template <int D, class T>
GKS_FN void slope(const Maxw<D, T>& g, T bK, const T* rhs, T* a) {
  T R[D], q = T(0), UR = T(0);
#pragma unroll
  for (int i = 0; i < D; ++i) {
    R[i] = rhs[1 + i] - g.U[i] * rhs[0];
    q += g.U[i] * g.U[i];
    UR += g.U[i] * R[i];
  }
  const T c = q + bK * g.il;  // |U|^2 + bK / (2 lambda)
  const T RE = T(2) * rhs[D + 1] - c * rhs[0];
  const T aE = (T(4) * g.lam * g.lam / bK) * (RE - T(2) * UR);
  T a0 = rhs[0] - T(0.5) * aE * c;
#pragma unroll
  for (int i = 0; i < D; ++i) {
    a[1 + i] = T(2) * g.lam * R[i] - g.U[i] * aE;
    a0 -= g.U[i] * a[1 + i];
  }
  a[0] = a0;
  a[D + 1] = aE;
}

// Time integrals over [0, dt] of Eq. resultingf and the ratios used for Abar:
//   T0 = int (1 - e), T1 = int ((tau + t) e - tau), T2 = int (t - tau + tau e), T3 = int e,
//   T4 = -int (tau + t) e, T5 = -tau int e  (e = exp(-t/tau));  Dn = dt^2/2 - T2;
//   r1 = T1/Dn, r4 = T4/Dn, r5 = T5/Dn.
// With x = dt/tau and phi_k(x) = sum_m (-x)^m/(m+k)!: T0 = dt x phi2, T1 = -dt^2 x (phi2 - 2 phi3),
// T2 = dt^2 x phi3, T3 = dt phi1, T4 = tau dt (e - 2 phi1), T5 = -tau dt phi1, Dn = dt^2 phi2.
// For x < 1 phi3 is summed from its series and phi2, phi1, e by the backward recurrence
// phi_{k-1} = 1/(k-1)! - x phi_k (no cancellation); otherwise the closed forms in e = exp(-x) are used.
struct TimeCoef {
  double T[6];
  double r1, r4, r5;
};

GKS_FN void phi_series(double x, double& p1, double& p2, double& p3, double& e) {
  // 1/(m+3)! for m = 0..17
  const double c[18] = {1.0 / 6, 1.0 / 24, 1.0 / 120, 1.0 / 720, 1.0 / 5040, 1.0 / 40320, 1.0 / 362880,
                        1.0 / 3628800, 1.0 / 39916800, 1.0 / 479001600, 1.0 / 6227020800.0,
                        1.0 / 87178291200.0, 1.0 / 1307674368000.0, 1.0 / 20922789888000.0,
                        1.0 / 355687428096000.0, 1.0 / 6402373705728000.0, 1.0 / 121645100408832000.0,
                        1.0 / 2432902008176640000.0};
  double s = c[17];
#pragma unroll
  for (int m = 16; m >= 0; --m) s = c[m] - x * s;
  p3 = s;
  p2 = 0.5 - x * p3;
  p1 = 1.0 - x * p2;
  e = 1.0 - x * p1;
}

template <class T>
GKS_FN void time_coeffs(T dt, T tau, T* Tc, T& r1, T& r4, T& r5) {
  if (!(tau > T(0))) {  // tau = 0: x -> infinity
    Tc[0] = dt;
    Tc[1] = T(0);
    Tc[2] = T(0.5) * dt * dt;
    Tc[3] = Tc[4] = Tc[5] = T(0);
    r1 = T(-1);
    r4 = r5 = T(0);
    return;
  }
  const T x = dt / tau;
  if (x < T(1)) {
    // series branch in double precision for either arithmetic type
    double p1, p2, p3, e;
    const double xd = (double)x, dtd = (double)dt, taud = (double)tau;
    phi_series(xd, p1, p2, p3, e);
    const double Dn = dtd * dtd * p2;
    const double T1 = -dtd * dtd * xd * (p2 - 2.0 * p3);
    const double T4 = taud * dtd * (e - 2.0 * p1);
    const double T5 = -taud * dtd * p1;
    Tc[0] = (T)(dtd * xd * p2);
    Tc[1] = (T)T1;
    Tc[2] = (T)(dtd * dtd * xd * p3);
    Tc[3] = (T)(dtd * p1);
    Tc[4] = (T)T4;
    Tc[5] = (T)T5;
    r1 = (T)(T1 / Dn);
    r4 = (T)(T4 / Dn);
    r5 = (T)(T5 / Dn);
  } else {
    const T e = g_exp(-x);
    const T q = T(1) - e;
    const T tq = tau * q;
    Tc[0] = dt - tq;
    Tc[1] = -tau * dt * (T(1) + e) + T(2) * tau * tq;
    Tc[2] = T(0.5) * dt * dt - tau * dt + tau * tq;
    Tc[3] = tq;
    Tc[4] = tau * dt * e - T(2) * tau * tq;
    Tc[5] = -tau * tq;
    const T y = tau / dt;
    const T yq = y * q;
    const T inv = T(1) / (T(1) - yq);
    r1 = (T(2) * yq - (T(1) + e)) * inv;
    r4 = (e - T(2) * yq) * inv;
    r5 = -yq * inv;
  }
}

// One face.  Inputs in the face frame:
//   wl, wr   reconstructed states; cl, cr cell averages of the two cells; sl, sr normal slopes;
//   tl, tr   tangential slopes (multi-dimensional expansion only); dxl, dxr centre-to-face distances;
//   tau_t    turbulent relaxation time at the face; dt the time step.
// Output: F, the flux integrated over [0, dt] (Eq. fluxesf); tau_out the total relaxation time.
template <int D, class T, bool MULTID>
GKS_FN void face_flux(const T* wl, const T* wr, const T* cl, const T* cr, const T* sl,
                                          const T* sr, const T (*tl)[D + 2], const T (*tr)[D + 2], T dxl,
                                          T dxr, T tau_t, T dt, const Gas<T>& gas, int abar_t0, T* F,
                                          T* tau_out) {
  constexpr int nv = D + 2;
  constexpr int NT = Dims<D>::nt;
  const T bK = gas.bK, K = gas.K;
  const Maxw<D, T> gl = maxwellian<D, T>(wl, bK);
  const Maxw<D, T> gr = maxwellian<D, T>(wr, bK);

  // Eq. intermediatestate: w0 = rho_l <psi>_{l,u>0} + rho_r <psi>_{r,u<0}
  Tab<D, T> lP, rN;
  tab_half<D, T>(gl, K, &lP, nullptr);
  tab_half<D, T>(gr, K, nullptr, &rN);
  T w0[nv];
  {
    T a[nv], b[nv];
    psi_mom<D, T>(lP, 0, 0, 0, 0, a);
    psi_mom<D, T>(rN, 0, 0, 0, 0, b);
#pragma unroll
    for (int m = 0; m < nv; ++m) w0[m] = gl.rho * a[m] + gr.rho * b[m];
  }
  const Maxw<D, T> g0 = maxwellian<D, T>(w0, bK);
  Tab<D, T> oP, oN, oF;
  tab_half<D, T>(g0, K, &oP, &oN);
  tab_full<D, T>(g0, K, oF);

  // Eq. initialf0: spatial coefficients of the initial state from the conservative gradients
  T al[nv], ar[nv], bl[NT][nv], br[NT][nv];
  {
    T r[nv];
    const T il = T(1) / gl.rho, ir = T(1) / gr.rho;
#pragma unroll
    for (int m = 0; m < nv; ++m) r[m] = sl[m] * il;
    slope<D, T>(gl, bK, r, al);
#pragma unroll
    for (int m = 0; m < nv; ++m) r[m] = sr[m] * ir;
    slope<D, T>(gr, bK, r, ar);
#pragma unroll
    for (int s = 0; s < D - 1; ++s) {
      if (MULTID) {
#pragma unroll
        for (int m = 0; m < nv; ++m) r[m] = tl[s][m] * il;
        slope<D, T>(gl, bK, r, bl[s]);
#pragma unroll
        for (int m = 0; m < nv; ++m) r[m] = tr[s][m] * ir;
        slope<D, T>(gr, bK, r, br[s]);
      }
    }
  }
  // A from the compatibility condition at t = 0: <(a u + b v + A) psi> = 0 (full moments)
  T Al[nv], Ar[nv];
  {
    Tab<D, T> f;
    T rhs[nv];
    tab_full<D, T>(gl, K, f);
#pragma unroll
    for (int m = 0; m < nv; ++m) rhs[m] = T(0);
    amom<D, T>(f, 1, -1, al, T(-1), rhs);
    if (MULTID) {
#pragma unroll
      for (int s = 0; s < D - 1; ++s) amom<D, T>(f, 0, s, bl[s], T(-1), rhs);
    }
    slope<D, T>(gl, bK, rhs, Al);
    tab_full<D, T>(gr, K, f);
#pragma unroll
    for (int m = 0; m < nv; ++m) rhs[m] = T(0);
    amom<D, T>(f, 1, -1, ar, T(-1), rhs);
    if (MULTID) {
#pragma unroll
      for (int s = 0; s < D - 1; ++s) amom<D, T>(f, 0, s, br[s], T(-1), rhs);
    }
    slope<D, T>(gr, bK, rhs, Ar);
  }
  // Eq. eqlgform: equilibrium slopes from W_j -> w0 -> W_{j+1}
  T abl[nv], abr[nv], bb[NT][nv];
  {
    T r[nv];
    const T i0 = T(1) / g0.rho;
    const T fl = i0 / dxl, fr = i0 / dxr;
#pragma unroll
    for (int m = 0; m < nv; ++m) r[m] = (w0[m] - cl[m]) * fl;
    slope<D, T>(g0, bK, r, abl);
#pragma unroll
    for (int m = 0; m < nv; ++m) r[m] = (cr[m] - w0[m]) * fr;
    slope<D, T>(g0, bK, r, abr);
    if (MULTID) {
#pragma unroll
      for (int s = 0; s < D - 1; ++s) {
#pragma unroll
        for (int m = 0; m < nv; ++m) r[m] = T(0.5) * (tl[s][m] + tr[s][m]) * i0;
        slope<D, T>(g0, bK, r, bb[s]);
      }
    }
  }
  // Eqs. relaxation time and taua: tau = mu/p0 + tau_t + C_a |p_r - p_l| / (p_r + p_l) dt
  const T p0 = g0.rho * g0.il, pl = gl.rho * gl.il, pr = gr.rho * gr.il;
  const T tau = gas.mu / p0 + tau_t + gas.C_a * g_abs(pr - pl) / (pr + pl) * dt;
  *tau_out = tau;
  T Tc[6], r1, r4, r5;
  time_coeffs<T>(dt, tau, Tc, r1, r4, r5);
  if (abar_t0) {
    r1 = T(-1);
    r4 = r5 = T(0);
  }
  // Abar from the compatibility condition integrated over [0, dt]:
  //   <Abar psi>_0 = r1 X1 + r4 X4 + r5 X5
  T Ab[nv];
  {
    T rhs[nv];
#pragma unroll
    for (int m = 0; m < nv; ++m) rhs[m] = T(0);
    amom<D, T>(oP, 1, -1, abl, r1, rhs);
    amom<D, T>(oN, 1, -1, abr, r1, rhs);
    if (MULTID) {
#pragma unroll
      for (int s = 0; s < D - 1; ++s) amom<D, T>(oF, 0, s, bb[s], r1, rhs);
    }
    const T i0 = T(1) / g0.rho;
    const T sl4 = r4 * gl.rho * i0, sr4 = r4 * gr.rho * i0;
    const T sl5 = r5 * gl.rho * i0, sr5 = r5 * gr.rho * i0;
    amom<D, T>(lP, 1, -1, al, sl4, rhs);
    amom<D, T>(rN, 1, -1, ar, sr4, rhs);
    if (MULTID) {
#pragma unroll
      for (int s = 0; s < D - 1; ++s) {
        amom<D, T>(lP, 0, s, bl[s], sl4, rhs);
        amom<D, T>(rN, 0, s, br[s], sr4, rhs);
      }
    }
    amom<D, T>(lP, 0, -1, Al, sl5, rhs);
    amom<D, T>(rN, 0, -1, Ar, sr5, rhs);
    slope<D, T>(g0, bK, rhs, Ab);
  }
  // Eq. fluxesf with the time integral of Eq. resultingf:
  //   F = rho0 [<u (T0 + T2 Abar) psi>_0 + T1 (<u^2 abar psi>_{0,split} + <u v bbar psi>_0)]
  //     + rho_l [<u (T3 + T5 A_l) psi>_{l,u>0} + T4 (<u^2 a_l psi> + <u v b_l psi>)_{l,u>0}] + (r, u<0)
  {
    T acc0[nv], accl[nv], accr[nv], c[nv];
#pragma unroll
    for (int m = 0; m < nv; ++m) acc0[m] = accl[m] = accr[m] = T(0);
#pragma unroll
    for (int m = 0; m < nv; ++m) c[m] = Tc[2] * Ab[m];
    c[0] += Tc[0];
    amom<D, T>(oF, 1, -1, c, T(1), acc0);
    amom<D, T>(oP, 2, -1, abl, Tc[1], acc0);
    amom<D, T>(oN, 2, -1, abr, Tc[1], acc0);
    if (MULTID) {
#pragma unroll
      for (int s = 0; s < D - 1; ++s) amom<D, T>(oF, 1, s, bb[s], Tc[1], acc0);
    }
#pragma unroll
    for (int m = 0; m < nv; ++m) c[m] = Tc[5] * Al[m];
    c[0] += Tc[3];
    amom<D, T>(lP, 1, -1, c, T(1), accl);
    amom<D, T>(lP, 2, -1, al, Tc[4], accl);
#pragma unroll
    for (int m = 0; m < nv; ++m) c[m] = Tc[5] * Ar[m];
    c[0] += Tc[3];
    amom<D, T>(rN, 1, -1, c, T(1), accr);
    amom<D, T>(rN, 2, -1, ar, Tc[4], accr);
    if (MULTID) {
#pragma unroll
      for (int s = 0; s < D - 1; ++s) {
        amom<D, T>(lP, 1, s, bl[s], Tc[4], accl);
        amom<D, T>(rN, 1, s, br[s], Tc[4], accr);
      }
    }
#pragma unroll
    for (int m = 0; m < nv; ++m) F[m] = g0.rho * acc0[m] + gl.rho * accl[m] + gr.rho * accr[m];
  }
}

}  // namespace gks
