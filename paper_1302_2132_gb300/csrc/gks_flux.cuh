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

#include <type_traits>
#include "gks_f2.cuh"

#ifndef GKS_FN
#define GKS_FN __device__ __forceinline__
#endif

namespace gks {

template <class T> GKS_FN T g_sqrt(T x);
#ifdef GKS_HOST_COUNT
template <> GKS_FN float g_sqrt<float>(float x) { return sqrtf(x); }
#else
// single precision: the hardware approximate square root (relative error about 2^-23, no slow-path
// branch); double precision stays IEEE
template <> GKS_FN float g_sqrt<float>(float x) {
  float r;
  asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}
#endif
template <> GKS_FN double g_sqrt<double>(double x) { return sqrt(x); }
// 1/sqrt(x): the hardware approximate reciprocal square root in single precision, IEEE otherwise
template <class T> GKS_FN T g_rsqrt(T x) { return T(1) / g_sqrt(x); }
#ifndef GKS_HOST_COUNT
template <> GKS_FN float g_rsqrt<float>(float x) {
  float r;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}
#endif
template <class T> GKS_FN T g_exp(T x);
#ifdef GKS_HOST_COUNT
template <> GKS_FN float g_exp<float>(float x) { return expf(x); }
#endif
template <> GKS_FN double g_exp<double>(double x) { return exp(x); }
template <class T> GKS_FN T g_erfc(T x);
#ifdef GKS_HOST_COUNT
template <> GKS_FN float g_erfc<float>(float x) { return erfcf(x); }
#endif
template <> GKS_FN double g_erfc<double>(double x) { return erfc(x); }
template <class T> GKS_FN T g_abs(T x) { return x < T(0) ? -x : x; }
#ifndef GKS_HOST_COUNT
template <> GKS_FN float g_abs<float>(float x) { return fabsf(x); }
template <> GKS_FN double g_abs<double>(double x) { return fabs(x); }
#endif

// Quotient and reciprocal: IEEE in double precision (the FP64 path matches the oracle to 1e-12);
// in single precision the hardware reciprocal (about 1 ulp), which avoids the multi-instruction
// IEEE sequence and its slow-path branch.  The FP32 form's tolerances are far above this error.
template <class T> GKS_FN T g_div(T a, T b) { return a / b; }
template <class T> GKS_FN T g_rcp(T x) { return T(1) / x; }
#ifndef GKS_HOST_COUNT
template <> GKS_FN float g_div<float>(float a, float b) { return __fdividef(a, b); }
template <> GKS_FN float g_rcp<float>(float x) { return __fdividef(1.0f, x); }
template <> GKS_FN float g_exp<float>(float x) { return __expf(x); }

// Single-precision erfc from the Chebyshev-fitted form of Press, Teukolsky, Vetterling and Flannery
// (Numerical Recipes, 2nd ed., section 6.2): for z = |x|, t = 1/(1 + z/2),
// erfc(z) = t exp(-z^2 + P(t)) with a degree-9 polynomial P, fractional error below 1.2e-7;
// erfc(-z) = 2 - erfc(z).
GKS_FN float erfc_cheb(float x) {
  const float z = fabsf(x);
  const float t = __fdividef(1.0f, 1.0f + 0.5f * z);
  const float c[10] = {-1.26551223f, 1.00002368f, 0.37409196f, 0.09678418f, -0.18628806f,
                       0.27886807f, -1.13520398f, 1.48851587f, -0.82215223f, 0.17087277f};
  float p = c[9];
#pragma unroll
  for (int i = 8; i >= 0; --i) p = fmaf(p, t, c[i]);
  const float r = t * __expf(p - z * z);
  return x >= 0.0f ? r : 2.0f - r;
}
template <> GKS_FN float g_erfc<float>(float x) { return erfc_cheb(x); }
#endif

// The same functions on two lanes (two faces per thread): reciprocals, exponentials and square roots
// per lane as in single precision, erfc from the same Chebyshev fit with paired arithmetic.
GKS_FN F2 g_rcp(F2 x) { return F2(g_rcp<float>(x.v.x), g_rcp<float>(x.v.y)); }
GKS_FN F2 g_div(F2 a, F2 b) { return F2(a * g_rcp(b)); }
GKS_FN F2 g_exp(F2 x) { return F2(g_exp<float>(x.v.x), g_exp<float>(x.v.y)); }
GKS_FN F2 g_sqrt(F2 x) { return F2(g_sqrt<float>(x.v.x), g_sqrt<float>(x.v.y)); }
GKS_FN F2 g_rsqrt(F2 x) { return F2(g_rsqrt<float>(x.v.x), g_rsqrt<float>(x.v.y)); }
GKS_FN F2 g_abs(F2 x) { return F2(fabsf(x.v.x), fabsf(x.v.y)); }
GKS_FN F2 g_erfc(F2 x) {
  const F2 z = g_abs(x);
  const F2 t = g_rcp(F2(1.0f) + F2(0.5f) * z);
  const float c[10] = {-1.26551223f, 1.00002368f, 0.37409196f, 0.09678418f, -0.18628806f,
                       0.27886807f, -1.13520398f, 1.48851587f, -0.82215223f, 0.17087277f};
  F2 p = F2(c[9]);
#pragma unroll
  for (int i = 8; i >= 0; --i) p = p * t + F2(c[i]);
  const F2 r = F2(t * g_exp(p - z * z));
  return F2(x.v.x >= 0.0f ? r.v.x : 2.0f - r.v.x, x.v.y >= 0.0f ? r.v.y : 2.0f - r.v.y);
}
GKS_FN F2 f2_select(bool cx, bool cy, F2 a, F2 b) { return F2(cx ? a.v.x : b.v.x, cy ? a.v.y : b.v.y); }
// a pending product as the argument: rounded first (exact overloads, so the templates above are not
// deduced with the product type)
GKS_FN F2 g_rcp(F2Mul x) { return g_rcp(F2(x)); }
GKS_FN F2 g_div(F2Mul a, F2Mul b) { return g_div(F2(a), F2(b)); }
GKS_FN F2 g_exp(F2Mul x) { return g_exp(F2(x)); }
GKS_FN F2 g_sqrt(F2Mul x) { return g_sqrt(F2(x)); }
GKS_FN F2 g_abs(F2Mul x) { return g_abs(F2(x)); }
GKS_FN F2 g_erfc(F2Mul x) { return g_erfc(F2(x)); }

constexpr double kInvSqrtPi = 0.56418958354775628695;  // 1/sqrt(pi)

template <int D> struct Dims {
  static constexpr int nv = D + 2;
  static constexpr int nt = D > 1 ? D - 1 : 1;  // storage for tangential arrays (>= 1)
};

// Macroscopic description of one Maxwellian.
template <int D, class T> struct Maxw {
  T rho, ir, U[D], lam, il;  // ir = 1/rho, il = 1/(2 lambda)
  T c, f4;               // |U|^2 + bK il and 4 lambda^2 / bK (used by every slope solve)
};

// Gas constants used by every face.
template <class T> struct Gas {
  T bK;   // K + D = 2/(gamma - 1)
  T ibK;  // 1 / bK
  T K;    // internal degrees of freedom
  T mu;   // molecular viscosity (tau_mol = mu / p)
  T C_a;  // artificial-dissipation coefficient (Eq. taua)
};

// (rho, U, lambda) of the Maxwellian carrying the conservative state w (Section 2: E = (u^2 + xi^2)/2,
// so rho E = rho |U|^2 / 2 + bK rho / (4 lambda)).  Two reciprocals: 1/rho, and 1/(2 lambda) =
// (2 rho E - rho |U|^2) / (bK rho) is a product, lambda its reciprocal; ibK = 1/bK.
template <int D, class T>
GKS_FN Maxw<D, T> maxwellian(const T* w, T bK, T ibK) {
  Maxw<D, T> g;
  g.rho = w[0];
  g.ir = g_rcp(w[0]);
  T q = T(0);
#pragma unroll
  for (int i = 0; i < D; ++i) {
    g.U[i] = w[1 + i] * g.ir;
    q += g.U[i] * g.U[i];
  }
  g.il = (T(2) * w[D + 1] - w[0] * q) * g.ir * ibK;
  g.lam = T(0.5) * g_rcp(g.il);
  g.c = q + bK * g.il;
  g.f4 = T(4) * g.lam * g.lam * ibK;
  return g;
}

// Moments of one Maxwellian, split into the normal velocity u and the transverse part.
//
// Every polynomial the flux needs is linear in the transverse basis {1, v_s, Et}, with
// Et = (sum_s v_s^2 + xi^2)/2 (so psi_E = u^2/2 + Et), and has polynomial coefficients in u.  Under
// the Maxwellian u, the v_s and xi are independent, so a moment factors into a moment of u over the
// chosen half line and a transverse moment over the full space.  The transverse moments of products
// of up to three basis functions are tabulated once per Maxwellian.
template <int D> struct Basis {
  static constexpr int NB = D + 1;  // 0: 1, 1..D-1: v_s, D: Et
};

template <int D, class T> struct Trans {
  T m1[D + 1];                     // <beta>
  T m2[D + 1][D + 1];              // <alpha beta>
  T m3[Dims<D>::nt][D + 1][D + 1];  // <v_s alpha beta>
};

// Gaussian moments <x^n>, n = 0..N-1, of mean U and variance il: x^{n+2} = U x^{n+1} + (n+1) il x^n.
template <int N, class T>
GKS_FN void recur(T U, T il, T* m) {
#pragma unroll
  for (int n = 0; n + 2 < N; ++n) m[n + 2] = U * m[n + 1] + T(n + 1) * il * m[n];
}

template <int D, class T>
GKS_FN void transverse(const Maxw<D, T>& g, T K, Trans<D, T>& t) {
  const T X1 = K * g.il;                        // <xi^2>
  const T X2 = K * (K + T(2)) * g.il * g.il;    // <xi^4>
  T V[Dims<D>::nt][6];
#pragma unroll
  for (int s = 0; s < D - 1; ++s) {
    V[s][0] = T(1);
    V[s][1] = g.U[1 + s];
    recur<6>(g.U[1 + s], g.il, V[s]);
  }
  t.m1[0] = T(1);
#pragma unroll
  for (int b = 0; b <= D; ++b) t.m2[0][b] = T(0);
  if (D == 1) {
    // basis {1, Et}, Et = xi^2 / 2
    t.m1[1] = T(0.5) * X1;
    t.m2[0][0] = T(1);
    t.m2[0][1] = t.m2[1][0] = t.m1[1];
    t.m2[1][1] = T(0.25) * X2;
  } else if (D == 2) {
    // basis {1, v, Et}, Et = (v^2 + xi^2)/2
    const T* v = V[0];
    const T e1 = v[2] + X1;                          // <2 Et>
    const T ve = v[3] + v[1] * X1;                   // <v 2 Et>
    const T vve = v[4] + v[2] * X1;                  // <v^2 2 Et>
    const T ee = v[4] + T(2) * v[2] * X1 + X2;       // <(2 Et)^2>
    const T vee = v[5] + T(2) * v[3] * X1 + v[1] * X2;  // <v (2 Et)^2>
    t.m1[1] = v[1];
    t.m1[2] = T(0.5) * e1;
    t.m2[0][0] = T(1);
    t.m2[0][1] = t.m2[1][0] = v[1];
    t.m2[0][2] = t.m2[2][0] = t.m1[2];
    t.m2[1][1] = v[2];
    t.m2[1][2] = t.m2[2][1] = T(0.5) * ve;
    t.m2[2][2] = T(0.25) * ee;
    // <v alpha beta>
    t.m3[0][0][0] = v[1];
    t.m3[0][0][1] = t.m3[0][1][0] = v[2];
    t.m3[0][0][2] = t.m3[0][2][0] = t.m2[1][2];
    t.m3[0][1][1] = v[3];
    t.m3[0][1][2] = t.m3[0][2][1] = T(0.5) * vve;
    t.m3[0][2][2] = T(0.25) * vee;
  } else {
    // basis {1, v, w, Et}, Et = (v^2 + w^2 + xi^2)/2
    const T* v = V[0];
    const T* w = V[Dims<D>::nt - 1];
    const T rv1 = w[2] + X1, rv2 = w[4] + T(2) * w[2] * X1 + X2;  // moments of 2Et - v^2
    const T rw1 = v[2] + X1, rw2 = v[4] + T(2) * v[2] * X1 + X2;  // moments of 2Et - w^2
    const T e1 = v[2] + rv1;
    const T ee = v[4] + T(2) * v[2] * rv1 + rv2;
    t.m1[1] = v[1];
    t.m1[2] = w[1];
    t.m1[3] = T(0.5) * e1;
    t.m2[0][0] = T(1);
#pragma unroll
    for (int b = 1; b <= 3; ++b) t.m2[0][b] = t.m2[b][0] = t.m1[b];
    t.m2[1][1] = v[2];
    t.m2[1][2] = t.m2[2][1] = v[1] * w[1];
    t.m2[2][2] = w[2];
    t.m2[1][3] = t.m2[3][1] = T(0.5) * (v[3] + v[1] * rv1);
    t.m2[2][3] = t.m2[3][2] = T(0.5) * (w[3] + w[1] * rw1);
    t.m2[3][3] = T(0.25) * ee;
    const T vwe = T(0.5) * (v[3] * w[1] + v[1] * w[3] + v[1] * w[1] * X1);  // <v w Et>
    // gamma = v
    t.m3[0][0][0] = v[1];
    t.m3[0][0][1] = t.m3[0][1][0] = v[2];
    t.m3[0][0][2] = t.m3[0][2][0] = t.m2[1][2];
    t.m3[0][0][3] = t.m3[0][3][0] = t.m2[1][3];
    t.m3[0][1][1] = v[3];
    t.m3[0][1][2] = t.m3[0][2][1] = v[2] * w[1];
    t.m3[0][2][2] = v[1] * w[2];
    t.m3[0][1][3] = t.m3[0][3][1] = T(0.5) * (v[4] + v[2] * rv1);
    t.m3[0][2][3] = t.m3[0][3][2] = vwe;
    t.m3[0][3][3] = T(0.25) * (v[5] + T(2) * v[3] * rv1 + v[1] * rv2);
    // gamma = w
    t.m3[1][0][0] = w[1];
    t.m3[1][0][1] = t.m3[1][1][0] = t.m2[1][2];
    t.m3[1][0][2] = t.m3[1][2][0] = w[2];
    t.m3[1][0][3] = t.m3[1][3][0] = t.m2[2][3];
    t.m3[1][1][1] = v[2] * w[1];
    t.m3[1][1][2] = t.m3[1][2][1] = v[1] * w[2];
    t.m3[1][2][2] = w[3];
    t.m3[1][1][3] = t.m3[1][3][1] = vwe;
    t.m3[1][2][3] = t.m3[1][3][2] = T(0.5) * (w[4] + w[2] * rw1);
    t.m3[1][3][3] = T(0.25) * (w[5] + T(2) * w[3] * rw1 + w[1] * rw2);
  }
}

// <beta> for the transverse basis {1, v_s, Et} (the first row of the transverse table).
template <int D, class T>
GKS_FN void trans_mean(const Maxw<D, T>& g, T K, T* m1) {
  T e = K * g.il;  // <xi^2>
#pragma unroll
  for (int s = 0; s < D - 1; ++s) {
    m1[1 + s] = g.U[1 + s];
    e += g.U[1 + s] * g.U[1 + s] + g.il;  // <v_s^2>
  }
  m1[0] = T(1);
  m1[D] = T(0.5) * e;
}

// <u^n>, n = 0..6, over the full line.
template <int D, class T>
GKS_FN void u_full(const Maxw<D, T>& g, T* u) {
  u[0] = T(1);
  u[1] = g.U[0];
  recur<7>(g.U[0], g.il, u);
}

// <u^n> over u > 0 (sgn = +1) or u < 0 (sgn = -1), from the textbook half-line Gaussian integrals
//   <1>_{u>0} = erfc(-sqrt(lam) U)/2,  <u>_{u>0} = U <1>_{u>0} + exp(-lam U^2)/(2 sqrt(pi lam)).
template <int D, class T>
GKS_FN void u_half(const Maxw<D, T>& g, T sgn, T* u) {
  const T rs = g_rsqrt(g.lam);  // 1/sqrt(lambda); sqrt(lambda) = lambda / sqrt(lambda)
  const T z = g.lam * rs * g.U[0];
  u[0] = T(0.5) * g_erfc(-sgn * z);
  u[1] = g.U[0] * u[0] + sgn * T(0.5) * g_exp(-z * z) * T(kInvSqrtPi) * rs;
  recur<7>(g.U[0], g.il, u);
}

// <psi_m> over the region of table u, m1 the transverse means.
template <int D, class T>
GKS_FN void psi_mean(const T* u, const T* m1, T* out) {
  out[0] = u[0];
  out[1] = u[1];
#pragma unroll
  for (int s = 0; s < D - 1; ++s) out[2 + s] = u[0] * m1[1 + s];
  out[D + 1] = T(0.5) * u[2] + u[0] * m1[D];
}

// acc[m] += s * <u^k gamma (a . psi) psi_m>, gamma = 1 (tg = -1) or v_tg.
// With a . psi = A(u) + sum_beta a_beta beta, A(u) = a0 + a1 u + aE u^2 / 2, and
// psi_m = P_m(u) + (transverse part), the moment is a sum of (u moment) x (transverse moment).
template <int D, class T>
GKS_FN void amom(const T* u, const Trans<D, T>& t, int k, int tg, const T* a, T s, T* acc) {
  constexpr int NB = D + 1;
  const T hE = T(0.5) * a[D + 1];
  const T SA0 = a[0] * u[k] + a[1] * u[k + 1] + hE * u[k + 2];
  const T SA1 = a[0] * u[k + 1] + a[1] * u[k + 2] + hE * u[k + 3];
  const T SA2 = a[0] * u[k + 2] + a[1] * u[k + 3] + hE * u[k + 4];
  // transverse factors: <gamma beta> and <gamma beta tau>
  T g1[NB], c2[NB];
#pragma unroll
  for (int b = 0; b < NB; ++b) g1[b] = tg < 0 ? t.m1[b] : t.m2[1 + tg][b];
  T c1 = T(0);
#pragma unroll
  for (int b = 1; b < NB; ++b) c1 += a[b == D ? D + 1 : 1 + b] * g1[b];
#pragma unroll
  for (int tau = 1; tau < NB; ++tau) {
    T q = T(0);
#pragma unroll
    for (int b = 1; b < NB; ++b) q += a[b == D ? D + 1 : 1 + b] * (tg < 0 ? t.m2[b][tau] : t.m3[tg][b][tau]);
    c2[tau] = q;
  }
  acc[0] += s * (SA0 * g1[0] + u[k] * c1);
  acc[1] += s * (SA1 * g1[0] + u[k + 1] * c1);
#pragma unroll
  for (int v = 0; v < D - 1; ++v) acc[2 + v] += s * (SA0 * g1[1 + v] + u[k] * c2[1 + v]);
  acc[D + 1] += s * (T(0.5) * (SA2 * g1[0] + u[k + 2] * c1) + SA0 * g1[D] + u[k] * c2[D]);
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
  return (a * b > R(0)) ? g_div(R(2) * a * b, a + b) : R(0);
}

// Higher-order face values in index space (Section 4 lists third-order MUSCL and fifth-order
// WENO beside the second-order default).  muscl3_right(a, b, c) is cell b's value at its right face
// from cells a, b, c; muscl3_left(a, b, c) cell b's value at its left face: the kappa = 1/3 scheme
// with each one-sided difference limited by minmod against 4 times the other.
template <class R>
GKS_FN R muscl3_right(R a, R b, R c) {
  const R dm = b - a, dp = c - b;
  return b + limiter<R>(LIM_MINMOD, dm, R(4) * dp) * R(1.0 / 6.0) + limiter<R>(LIM_MINMOD, dp, R(4) * dm) * R(1.0 / 3.0);
}
template <class R>
GKS_FN R muscl3_left(R a, R b, R c) {
  const R dm = b - a, dp = c - b;
  return b - limiter<R>(LIM_MINMOD, dp, R(4) * dm) * R(1.0 / 6.0) - limiter<R>(LIM_MINMOD, dm, R(4) * dp) * R(1.0 / 3.0);
}
// Jiang and Shu's WENO-5: the value at the face to the right of c from cells a, b, c, d, e
// (candidate stencils' face values, smoothness indicators with 13/12 and 1/4, linear weights
// 1/10, 6/10, 3/10, epsilon 1e-6).
template <class R>
GKS_FN R weno5(R a, R b, R c, R d, R e) {
  const R s6 = R(1.0 / 6.0), c13 = R(13.0 / 12.0);
  const R q0 = (R(2) * a - R(7) * b + R(11) * c) * s6;
  const R q1 = (-b + R(5) * c + R(2) * d) * s6;
  const R q2 = (R(2) * c + R(5) * d - e) * s6;
  const R t0 = a - R(2) * b + c, u0 = a - R(4) * b + R(3) * c;
  const R t1 = b - R(2) * c + d, u1 = b - d;
  const R t2 = c - R(2) * d + e, u2 = R(3) * c - R(4) * d + e;
  const R b0 = c13 * t0 * t0 + R(0.25) * u0 * u0;
  const R b1 = c13 * t1 * t1 + R(0.25) * u1 * u1;
  const R b2 = c13 * t2 * t2 + R(0.25) * u2 * u2;
  const R eps = R(1e-6);
  const R a0 = g_div(R(0.1), (eps + b0) * (eps + b0));
  const R a1 = g_div(R(0.6), (eps + b1) * (eps + b1));
  const R a2 = g_div(R(0.3), (eps + b2) * (eps + b2));
  return g_div(a0 * q0 + a1 * q1 + a2 * q2, a0 + a1 + a2);
}

// MUSCL on one variable at the face between cells 1 and 2 of the stencil s0..s3 with widths
// h0..h3: limited slopes of cells 1 and 2 and the face values left and right.
template <class R>
GKS_FN void muscl(int lim, R s0, R s1, R s2, R s3, R h0, R h1, R h2, R h3, R& wl, R& wr, R& sl, R& sr) {
  const R dm = g_div(s1 - s0, R(0.5) * (h0 + h1));
  const R dc = g_div(s2 - s1, R(0.5) * (h1 + h2));
  const R dp = g_div(s3 - s2, R(0.5) * (h2 + h3));
  sl = limiter<R>(lim, dm, dc);
  sr = limiter<R>(lim, dc, dp);
  wl = s1 + R(0.5) * h1 * sl;
  wr = s2 - R(0.5) * h2 * sr;
}

// The pair <u^k gamma (a . psi) psi_m> and <u^(k+1) gamma (a . psi) psi_m>, which share the u-moments
// of A(u) and the transverse sums: acc_lo += s_lo * first, acc_hi += s_hi * second (k <= 1).
template <int D, class T>
GKS_FN void amom2(const T* u, const Trans<D, T>& t, int k, int tg, const T* a, T s_lo, T* acc_lo, T s_hi,
                  T* acc_hi) {
  constexpr int NB = D + 1;
  const T hE = T(0.5) * a[D + 1];
  T SA[4];
#pragma unroll
  for (int j = 0; j < 4; ++j) SA[j] = a[0] * u[k + j] + a[1] * u[k + j + 1] + hE * u[k + j + 2];
  T g1[NB], c2[NB];
#pragma unroll
  for (int b = 0; b < NB; ++b) g1[b] = tg < 0 ? t.m1[b] : t.m2[1 + tg][b];
  T c1 = T(0);
#pragma unroll
  for (int b = 1; b < NB; ++b) c1 += a[b == D ? D + 1 : 1 + b] * g1[b];
#pragma unroll
  for (int tau = 1; tau < NB; ++tau) {
    T q = T(0);
#pragma unroll
    for (int b = 1; b < NB; ++b) q += a[b == D ? D + 1 : 1 + b] * (tg < 0 ? t.m2[b][tau] : t.m3[tg][b][tau]);
    c2[tau] = q;
  }
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const T s = h ? s_hi : s_lo;
    T* acc = h ? acc_hi : acc_lo;
    const int kk = k + h;
    acc[0] += s * (SA[h] * g1[0] + u[kk] * c1);
    acc[1] += s * (SA[h + 1] * g1[0] + u[kk + 1] * c1);
#pragma unroll
    for (int v = 0; v < D - 1; ++v) acc[2 + v] += s * (SA[h] * g1[1 + v] + u[kk] * c2[1 + v]);
    acc[D + 1] += s * (T(0.5) * (SA[h + 2] * g1[0] + u[kk + 2] * c1) + SA[h] * g1[D] + u[kk] * c2[D]);
  }
}

// Coefficients a of a . psi with <(a . psi) psi> = rhs (already divided by rho): closed-form inverse
// of the Maxwellian moment matrix.
template <int D, class T>
GKS_FN void slope(const Maxw<D, T>& g, T bK, const T* rhs, T* a) {
  T R[D], UR = T(0);
#pragma unroll
  for (int i = 0; i < D; ++i) {
    R[i] = rhs[1 + i] - g.U[i] * rhs[0];
    UR += g.U[i] * R[i];
  }
  const T RE = T(2) * rhs[D + 1] - g.c * rhs[0];
  const T aE = g.f4 * (RE - T(2) * UR);
  const T l2 = T(2) * g.lam;
  T a0 = rhs[0] - T(0.5) * aE * g.c;
#pragma unroll
  for (int i = 0; i < D; ++i) {
    a[1 + i] = l2 * R[i] - g.U[i] * aE;
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
// phi_{k-1} = 1/(k-1)! - x phi_k (no cancellation), in the arithmetic type; otherwise the closed
// forms in e = exp(-x) are used.
struct TimeCoef {
  double T[6];
  double r1, r4, r5;
};

// phi3 = sum_m (-x)^m / (m+3)! by Horner, then phi2, phi1 and e = exp(-x) by the backward recurrence
// phi_{k-1} = 1/(k-1)! - x phi_k.  For 0 <= x < 1 every step is free of cancellation; 18 terms
// reach double precision, 12 leave a truncation below 1e-9 (enough in single precision).
template <class T>
GKS_FN void phi_series(T x, T& p1, T& p2, T& p3, T& e) {
  T s;
  if constexpr (std::is_same<T, double>::value) {
    const double c[18] = {1.0 / 6, 1.0 / 24, 1.0 / 120, 1.0 / 720, 1.0 / 5040, 1.0 / 40320, 1.0 / 362880,
                          1.0 / 3628800, 1.0 / 39916800, 1.0 / 479001600, 1.0 / 6227020800.0,
                          1.0 / 87178291200.0, 1.0 / 1307674368000.0, 1.0 / 20922789888000.0,
                          1.0 / 355687428096000.0, 1.0 / 6402373705728000.0, 1.0 / 121645100408832000.0,
                          1.0 / 2432902008176640000.0};
    s = c[17];
#pragma unroll
    for (int m = 16; m >= 0; --m) s = c[m] - x * s;
  } else {
    // single-precision coefficients written as such, so that no double-to-float conversion (an FP64
    // pipe instruction) is left in the series
    const float c[12] = {1.0f / 6, 1.0f / 24, 1.0f / 120, 1.0f / 720, 1.0f / 5040, 1.0f / 40320, 1.0f / 362880,
                         1.0f / 3628800, 1.0f / 39916800, 1.0f / 479001600, 1.0f / 6227020800.0f,
                         1.0f / 87178291200.0f};
    s = T(c[11]);
#pragma unroll
    for (int m = 10; m >= 0; --m) s = T(c[m]) - x * s;
  }
  p3 = s;
  p2 = T(0.5) - x * p3;
  p1 = T(1) - x * p2;
  e = T(1) - x * p1;
}

template <class T>
GKS_FN void time_coeffs(T dt, T tau, T* Tc, T& r1, T& r4, T& r5) {
  const T x = g_div(dt, tau);
  if (x < T(1)) {
    // series branch (phi_k summed, no cancellation) in the arithmetic type
    T p1, p2, p3, e;
    const T xd = x, dtd = dt, taud = tau;
    phi_series(xd, p1, p2, p3, e);
    const T Dn = dtd * dtd * p2;
    const T T1 = -dtd * dtd * xd * (p2 - T(2) * p3);
    const T T4 = taud * dtd * (e - T(2) * p1);
    const T T5 = -taud * dtd * p1;
    Tc[0] = dtd * xd * p2;
    Tc[1] = T1;
    Tc[2] = dtd * dtd * xd * p3;
    Tc[3] = dtd * p1;
    Tc[4] = T4;
    Tc[5] = T5;
    const T iDn = g_rcp(Dn);
    r1 = T1 * iDn;
    r4 = T4 * iDn;
    r5 = T5 * iDn;
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
    const T y = g_div(tau, dt);
    const T yq = y * q;
    const T inv = g_rcp(T(1) - yq);
    r1 = (T(2) * yq - (T(1) + e)) * inv;
    r4 = (e - T(2) * yq) * inv;
    r5 = -yq * inv;
  }
}

// Two lanes: both branches of time_coeffs, each lane keeping its own (x < 1: the series).
template <>
GKS_FN void time_coeffs<F2>(F2 dt, F2 tau, F2* Tc, F2& r1, F2& r4, F2& r5) {
  const F2 x = g_div(dt, tau);
  const bool sx = x.v.x < 1.0f, sy = x.v.y < 1.0f;
  F2 p1, p2, p3, e;
  phi_series(x, p1, p2, p3, e);
  const F2 dt2 = F2(dt * dt);
  const F2 Dn = F2(dt2 * p2);
  F2 Ts[6];
  const F2 T1s = F2(-dt2 * x) * (p2 - F2(2.0f) * p3);
  const F2 T4s = F2(tau * dt) * (e - F2(2.0f) * p1);
  const F2 T5s = -(F2(tau * dt) * p1);
  Ts[0] = F2(dt * x) * p2;
  Ts[1] = T1s;
  Ts[2] = F2(dt2 * x) * p3;
  Ts[3] = dt * p1;
  Ts[4] = T4s;
  Ts[5] = T5s;
  const F2 iDn = g_rcp(Dn);
  const F2 r1s = T1s * iDn, r4s = T4s * iDn, r5s = T5s * iDn;
  // closed forms in e = exp(-x)
  const F2 ec = g_exp(-x);
  const F2 q = F2(1.0f) - ec;
  const F2 tq = tau * q;
  F2 Tcl[6];
  Tcl[0] = dt - tq;
  Tcl[1] = F2(-(tau * dt)) * (F2(1.0f) + ec) + F2(2.0f) * F2(tau * tq);
  Tcl[2] = F2(0.5f) * F2(dt * dt) - tau * dt + tau * tq;
  Tcl[3] = tq;
  Tcl[4] = F2(tau * dt) * ec - F2(2.0f) * F2(tau * tq);
  Tcl[5] = -(tau * tq);
  const F2 y = g_div(tau, dt);
  const F2 yq = y * q;
  const F2 inv = g_rcp(F2(1.0f) - yq);
  const F2 r1c = (F2(2.0f) * yq - (F2(1.0f) + ec)) * inv;
  const F2 r4c = (ec - F2(2.0f) * yq) * inv;
  const F2 r5c = -(yq * inv);
#pragma unroll
  for (int i = 0; i < 6; ++i) Tc[i] = f2_select(sx, sy, Ts[i], Tcl[i]);
  r1 = f2_select(sx, sy, r1s, r1c);
  r4 = f2_select(sx, sy, r4s, r4c);
  r5 = f2_select(sx, sy, r5s, r5c);
}

// The time coefficients with the degree of rarefaction eps in place of tau/dt (Eqs. tautautilde,
// rarefactionkepsilon, epsilonkomega): Eq. fkepsilon with alpha = eps (1 - e^{-1/eps}) and
// beta = e^{-1/eps} (Eq. alphabetakepsilon with the corrected beta), in the T0..T5 form:
//   T0 = dt (1 - alpha), T1 = dt tau (2 alpha - 1 - beta), T2 = dt (dt/2 - tau (1 - alpha)),
//   T3 = dt alpha, T4 = dt tau (beta - 2 alpha), T5 = -dt tau alpha, Dn = dt tau (1 - alpha),
// so r1 = (2 alpha - 1 - beta)/(1 - alpha), r4 = (beta - 2 alpha)/(1 - alpha), r5 = -alpha/(1 - alpha).
// eps = tau/dt gives time_coeffs.  For eps > 1 (x = 1/eps < 1) alpha = phi1(x), 1 - alpha = x phi2,
// 2 alpha - 1 - beta = -x^2 (phi2 - 2 phi3), from the cancellation-free series.
template <class T>
GKS_FN void time_coeffs_hat(T dt, T tau, T eps, T* Tc, T& r1, T& r4, T& r5) {
  T a, one_a, c1, c4;
  if (eps > T(1)) {
    const T x = g_rcp(eps);
    T p1, p2, p3, e;
    phi_series(x, p1, p2, p3, e);
    a = p1;
    one_a = x * p2;
    c1 = -x * x * (p2 - T(2) * p3);
    c4 = e - T(2) * p1;
  } else {
    const T beta = eps > T(0) ? g_exp(-g_rcp(eps)) : T(0);
    a = eps * (T(1) - beta);
    one_a = T(1) - a;
    c1 = T(2) * a - T(1) - beta;
    c4 = beta - T(2) * a;
  }
  const T dtau = dt * tau;
  Tc[0] = dt * one_a;
  Tc[1] = dtau * c1;
  Tc[2] = dt * (T(0.5) * dt - tau * one_a);
  Tc[3] = dt * a;
  Tc[4] = dtau * c4;
  Tc[5] = -dtau * a;
  const T i1 = g_rcp(one_a);
  r1 = c1 * i1;
  r4 = c4 * i1;
  r5 = -a * i1;
}

// The density row <u^k gamma (a . psi)> of amom alone.
template <int D, class T>
GKS_FN T amom_rho(const T* u, const Trans<D, T>& t, int k, int tg, const T* a) {
  constexpr int NB = D + 1;
  const T hE = T(0.5) * a[D + 1];
  const T SA0 = a[0] * u[k] + a[1] * u[k + 1] + hE * u[k + 2];
  T g0 = tg < 0 ? t.m1[0] : t.m2[1 + tg][0], c1 = T(0);
#pragma unroll
  for (int b = 1; b < NB; ++b) c1 += a[b == D ? D + 1 : 1 + b] * (tg < 0 ? t.m1[b] : t.m2[1 + tg][b]);
  return SA0 * g0 + u[k] * c1;
}

// |D rho| = |d_t rho + U_n d_n rho| at the face for the rarefaction option (Eqs. tautautilde,
// tautilde): d_t rho = -rho0 (<abar_l . psi u>_{u>0} + <abar_r . psi u>_{u<0} + <bbar . psi v>) from
// the t = 0 compatibility condition of the equilibrium part, d_n rho the mean of the density slopes
// (w0 - W_j)/dxl and (W_{j+1} - w0)/dxr.  Slopes and moments of g0 as in face_flux.
template <int D, class T, bool MULTID, class In>
GKS_FN T face_drho(const Maxw<D, T>& g0, const T* w0, const In& in, T dxl, T dxr, T i0, T bK, T K) {
  constexpr int nv = D + 2;
  const T dn = T(0.5) * (g_div(w0[0] - in.c(0, 0), dxl) + g_div(in.c(1, 0) - w0[0], dxr));
  Trans<D, T> t0;
  transverse<D, T>(g0, K, t0);
  T oF[7], oP[7], half[7], r[nv], ab[nv];
  u_full<D, T>(g0, oF);
  u_half<D, T>(g0, T(1), oP);
  const T fl = g_div(i0, dxl), fr = g_div(i0, dxr);
#pragma unroll
  for (int m = 0; m < nv; ++m) r[m] = (w0[m] - in.c(0, m)) * fl;
  slope<D, T>(g0, bK, r, ab);
  T x1 = amom_rho<D, T>(oP, t0, 1, -1, ab);
#pragma unroll
  for (int m = 0; m < nv; ++m) r[m] = (in.c(1, m) - w0[m]) * fr;
  slope<D, T>(g0, bK, r, ab);
#pragma unroll
  for (int n = 0; n < 7; ++n) half[n] = oF[n] - oP[n];
  x1 += amom_rho<D, T>(half, t0, 1, -1, ab);
  if (MULTID) {
#pragma unroll
    for (int q = 0; q < D - 1; ++q) {
#pragma unroll
      for (int m = 0; m < nv; ++m) r[m] = T(0.5) * (in.t(0, q, m) + in.t(1, q, m)) * i0;
      slope<D, T>(g0, bK, r, ab);
      x1 += amom_rho<D, T>(oF, t0, 0, q, ab);
    }
  }
  return g_abs(-g0.rho * x1 + g0.U[0] * dn);
}

// One face.  Inputs in the face frame:
//   wl, wr   reconstructed states; cl, cr cell averages of the two cells; sl, sr normal slopes;
//   tl, tr   tangential slopes (multi-dimensional expansion only); dxl, dxr centre-to-face distances;
//   tau_t    turbulent relaxation time at the face; dt the time step.
// Output: F, the flux integrated over [0, dt] (Eq. fluxesf); tau_out the total relaxation time.
//
// The work is ordered so that each velocity region (u > 0 of the left Maxwellian, u < 0 of the
// right one, and the two halves and the full line of the equilibrium g0) is visited once, adding
// both its part of the right-hand side of the Abar equation and its part of the flux; only the
// Abar term of the flux waits for Abar.
// RAR: the rarefaction option -- the degree of rarefaction eps = tau/tauhat, tauhat = rho0/|D rho|
// (capped at 1e30), replaces tau/dt inside the time coefficients (Eq. epsilonkomega).
//
// The inputs other than wl, wr come through an accessor `in` (FaceArrays below, or a view of a
// shared-memory tile): in.s(sd, m) the normal slope, in.c(sd, m) the cell average and in.t(sd, q, m)
// the q-th tangential slope of component m on side sd (0 left, 1 right), each read where it is used.
template <int D, class T, bool MULTID, bool RAR = false, class In>
GKS_FN void face_flux_in(const T* wl, const T* wr, const In& in, T dxl, T dxr, T tau_t, T dt, const Gas<T>& gas,
                         int abar_t0, T* F, T* tau_out) {
  constexpr int nv = D + 2;
  const T bK = gas.bK, K = gas.K, ibK = gas.ibK;
  const Maxw<D, T> gl = maxwellian<D, T>(wl, bK, ibK);
  const Maxw<D, T> gr = maxwellian<D, T>(wr, bK, ibK);

  // Eq. intermediatestate: w0 = rho_l <psi>_{l,u>0} + rho_r <psi>_{r,u<0}
  T w0[nv];
  T lP[7], rN[7];
  u_half<D, T>(gl, T(1), lP);
  u_half<D, T>(gr, T(-1), rN);
  {
    T a[nv], b[nv], ml[D + 1], mr[D + 1];
    trans_mean<D, T>(gl, K, ml);
    trans_mean<D, T>(gr, K, mr);
    psi_mean<D, T>(lP, ml, a);
    psi_mean<D, T>(rN, mr, b);
#pragma unroll
    for (int m = 0; m < nv; ++m) w0[m] = gl.rho * a[m] + gr.rho * b[m];
  }
  const Maxw<D, T> g0 = maxwellian<D, T>(w0, bK, ibK);

  // Eqs. relaxation time and taua: tau = mu/p0 + tau_t + C_a |p_r - p_l| / (p_r + p_l) dt
  const T p0 = g0.rho * g0.il, pl = gl.rho * gl.il, pr = gr.rho * gr.il;
  const T tau = g_div(gas.mu, p0) + tau_t + g_div(gas.C_a * g_abs(pr - pl), pr + pl) * dt;
  *tau_out = tau;
  T Tc[6], r1, r4, r5;
  if constexpr (RAR) {
    const T drho = face_drho<D, T, MULTID>(g0, w0, in, dxl, dxr, g0.ir, bK, K);
    const T eps = drho > T(1e-30) * g0.rho ? g_div(tau * drho, g0.rho) : tau * T(1e-30);
    time_coeffs_hat<T>(dt, tau, eps, Tc, r1, r4, r5);
  } else {
    time_coeffs<T>(dt, tau, Tc, r1, r4, r5);
  }
  if (abar_t0) {
    r1 = T(-1);
    r4 = r5 = T(0);
  }
  const T i0 = g0.ir;

  // Abar right-hand side (per unit rho0) and flux, accumulated region by region
  T rhs[nv];
#pragma unroll
  for (int m = 0; m < nv; ++m) {
    rhs[m] = T(0);
    F[m] = T(0);
  }

  // The two sides of the initial state, one loop body (sd = 0: left Maxwellian on u > 0, sd = 1:
  // right Maxwellian on u < 0): Eq. initialf0 slopes a (normal), b (tangential), A; their parts of
  // the Abar right-hand side and of the flux.
#pragma unroll 1
  for (int sd = 0; sd < 2; ++sd) {
    const Maxw<D, T> g = sd ? gr : gl;
    Trans<D, T> ts;
    transverse<D, T>(g, K, ts);
    T half[7], a[nv], b[Dims<D>::nt][nv], A[nv], r[nv];
#pragma unroll
    for (int n = 0; n < 7; ++n) half[n] = sd ? rN[n] : lP[n];
    const T ir = g.ir;
#pragma unroll
    for (int m = 0; m < nv; ++m) r[m] = in.s(sd, m) * ir;
    slope<D, T>(g, bK, r, a);
    if (MULTID) {
#pragma unroll
      for (int q = 0; q < D - 1; ++q) {
#pragma unroll
        for (int m = 0; m < nv; ++m) r[m] = in.t(sd, q, m) * ir;
        slope<D, T>(g, bK, r, b[q]);
      }
    }
    // A from the compatibility condition at t = 0: <(a u + b v + A) psi> = 0 (full line)
    {
      T uf[7];
      u_full<D, T>(g, uf);
#pragma unroll
      for (int m = 0; m < nv; ++m) r[m] = T(0);
      amom<D, T>(uf, ts, 1, -1, a, T(-1), r);
      if (MULTID) {
#pragma unroll
        for (int q = 0; q < D - 1; ++q) amom<D, T>(uf, ts, 0, q, b[q], T(-1), r);
      }
      slope<D, T>(g, bK, r, A);
    }
    // Abar rhs: r4 rho/rho0 <(a u + b v) psi> + r5 rho/rho0 <A psi> over the half line, and the
    // flux rho [T3 <u psi> + T5 <u A psi> + T4 (<u^2 a psi> + <u v b psi>)]: each polynomial once,
    // at u^k for the rhs and u^(k+1) for the flux
    const T s4 = r4 * g.rho * i0, s5 = r5 * g.rho * i0, s4f = Tc[4] * g.rho;
    amom2<D, T>(half, ts, 1, -1, a, s4, rhs, s4f, F);
    amom2<D, T>(half, ts, 0, -1, A, s5, rhs, Tc[5] * g.rho, F);
    {
      T m[nv];
      psi_mean<D, T>(half + 1, ts.m1, m);  // <u psi> over the half line
      const T s3 = Tc[3] * g.rho;
#pragma unroll
      for (int q = 0; q < nv; ++q) F[q] += s3 * m[q];
    }
    if (MULTID) {
#pragma unroll
      for (int q = 0; q < D - 1; ++q) amom2<D, T>(half, ts, 0, q, b[q], s4, rhs, s4f, F);
    }
  }

  // equilibrium g0: Eq. eqlgform slopes from W_j -> w0 -> W_{j+1} (and the mean tangential slope)
  Trans<D, T> tr0;
  transverse<D, T>(g0, K, tr0);
  T oF[7], oP[7];
  u_full<D, T>(g0, oF);
  u_half<D, T>(g0, T(1), oP);
  {
    const T fl = g_div(i0, dxl), fr = g_div(i0, dxr);
    const T s1f = Tc[1] * g0.rho;
#pragma unroll 1
    for (int sd = 0; sd < 2; ++sd) {
      // sd = 0: abar_l on u > 0; sd = 1: abar_r on u < 0 (table = full line minus u > 0)
      T r[nv], ab[nv], half[7];
#pragma unroll
      for (int m = 0; m < nv; ++m) r[m] = sd ? (in.c(1, m) - w0[m]) * fr : (w0[m] - in.c(0, m)) * fl;
#pragma unroll
      for (int n = 0; n < 7; ++n) half[n] = sd ? oF[n] - oP[n] : oP[n];
      slope<D, T>(g0, bK, r, ab);
      amom2<D, T>(half, tr0, 1, -1, ab, r1, rhs, s1f, F);
    }
    if (MULTID) {
      T r[nv], ab[nv];
#pragma unroll
      for (int q = 0; q < D - 1; ++q) {
#pragma unroll
        for (int m = 0; m < nv; ++m) r[m] = T(0.5) * (in.t(0, q, m) + in.t(1, q, m)) * i0;
        slope<D, T>(g0, bK, r, ab);
        amom2<D, T>(oF, tr0, 0, q, ab, r1, rhs, s1f, F);
      }
    }
  }
  // Abar from the compatibility condition integrated over [0, dt]; flux rho0 <u (T0 + T2 Abar) psi>
  {
    T Ab[nv];
    slope<D, T>(g0, bK, rhs, Ab);
#pragma unroll
    for (int m = 0; m < nv; ++m) Ab[m] *= Tc[2];
    Ab[0] += Tc[0];
    amom<D, T>(oF, tr0, 1, -1, Ab, g0.rho, F);
  }
}

// Face inputs held in the caller's arrays (registers): sl, sr normal slopes, cl, cr cell averages,
// tl, tr tangential slopes (read only with the multi-dimensional expansion).
template <int D, class T> struct FaceArrays {
  const T *sl, *sr, *cl, *cr;
  const T (*tl)[D + 2];
  const T (*tr)[D + 2];
  GKS_FN T s(int sd, int m) const { return sd ? sr[m] : sl[m]; }
  GKS_FN T c(int sd, int m) const { return sd ? cr[m] : cl[m]; }
  GKS_FN T t(int sd, int q, int m) const { return sd ? tr[q][m] : tl[q][m]; }
};

// face_flux_in with the inputs in arrays.
template <int D, class T, bool MULTID, bool RAR = false>
GKS_FN void face_flux(const T* wl, const T* wr, const T* cl, const T* cr, const T* sl, const T* sr,
                      const T (*tl)[D + 2], const T (*tr)[D + 2], T dxl, T dxr, T tau_t, T dt, const Gas<T>& gas,
                      int abar_t0, T* F, T* tau_out) {
  const FaceArrays<D, T> in{sl, sr, cl, cr, tl, tr};
  face_flux_in<D, T, MULTID, RAR>(wl, wr, in, dxl, dxr, tau_t, dt, gas, abar_t0, F, tau_out);
}

// face_flux_in in single precision with the two sides of the face evaluated together on the paired
// FP32 instructions: lane x carries the left Maxwellian on u > 0, lane y the right one on u < 0, for
// the intermediate state, the slopes a, b, A and their parts of the Abar right-hand side and of the
// flux; the two one-sided equilibrium slopes abar_l (u > 0) and abar_r (u < 0) are paired the same
// way.  The paired sums are added lane x + lane y at the end of each part.  Same terms as
// face_flux_in; the order of the final additions differs, mu/p0 is taken as 2 mu lambda0 / rho0, the
// artificial part of tau is skipped when C_a = 0, and idxl, idxr are the reciprocals of dxl, dxr.
template <int D, bool MULTID, bool RAR = false, class In>
GKS_FN void face_flux_ps(const float* wl, const float* wr, const In& in, float dxl, float dxr, float idxl,
                         float idxr, float tau_t, float dt, const Gas<float>& gas, int abar_t0, float* F,
                         float* tau_out) {
  using T = float;
  constexpr int nv = D + 2;
  const T bK = gas.bK, K = gas.K, ibK = gas.ibK;
  F2 w2[nv];
#pragma unroll
  for (int m = 0; m < nv; ++m) w2[m] = F2(wl[m], wr[m]);
  const Maxw<D, F2> gs = maxwellian<D, F2>(w2, F2(bK), F2(ibK));
  F2 hs[7];  // <u^n> over u > 0 (left) and u < 0 (right)
  u_half<D, F2>(gs, F2(1.0f, -1.0f), hs);

  // Eq. intermediatestate: w0 = rho_l <psi>_{l,u>0} + rho_r <psi>_{r,u<0}
  T w0[nv];
  {
    F2 ab[nv], m1[D + 1];
    trans_mean<D, F2>(gs, F2(K), m1);
    psi_mean<D, F2>(hs, m1, ab);
#pragma unroll
    for (int m = 0; m < nv; ++m) {
      const F2 q = F2(gs.rho * ab[m]);
      w0[m] = q.v.x + q.v.y;
    }
  }
  const Maxw<D, T> g0 = maxwellian<D, T>(w0, bK, ibK);

  // Eqs. relaxation time and taua: mu/p0 = 2 mu lambda0 / rho0; the artificial part only with C_a > 0
  T tau = T(2) * gas.mu * g0.lam * g0.ir + tau_t;
  if (gas.C_a != T(0)) {
    const F2 plr = F2(gs.rho * gs.il);
    const T pl = plr.v.x, pr = plr.v.y;
    tau += g_div(gas.C_a * g_abs(pr - pl), pr + pl) * dt;
  }
  *tau_out = tau;
  T Tc[6], r1, r4, r5;
  if constexpr (RAR) {
    const T drho = face_drho<D, T, MULTID>(g0, w0, in, dxl, dxr, g0.ir, bK, K);
    const T eps = drho > T(1e-30) * g0.rho ? g_div(tau * drho, g0.rho) : tau * T(1e-30);
    time_coeffs_hat<T>(dt, tau, eps, Tc, r1, r4, r5);
  } else {
    time_coeffs<T>(dt, tau, Tc, r1, r4, r5);
  }
  if (abar_t0) {
    r1 = T(-1);
    r4 = r5 = T(0);
  }
  const T i0 = g0.ir;

  T rhs[nv];
  // the two sides of the initial state: slopes a (normal), b (tangential), A (Eq. initialf0)
  {
    Trans<D, F2> ts;
    transverse<D, F2>(gs, F2(K), ts);
    F2 a[nv], b[Dims<D>::nt][nv], A[nv], r[nv];
    const F2 ir = gs.ir;
#pragma unroll
    for (int m = 0; m < nv; ++m) r[m] = F2(F2(in.s(0, m), in.s(1, m)) * ir);
    slope<D, F2>(gs, F2(bK), r, a);
    if (MULTID) {
#pragma unroll
      for (int q = 0; q < D - 1; ++q) {
#pragma unroll
        for (int m = 0; m < nv; ++m) r[m] = F2(F2(in.t(0, q, m), in.t(1, q, m)) * ir);
        slope<D, F2>(gs, F2(bK), r, b[q]);
      }
    }
    // A from the compatibility condition at t = 0: <(a u + b v + A) psi> = 0 (full line)
    {
      F2 uf[7];
      u_full<D, F2>(gs, uf);
#pragma unroll
      for (int m = 0; m < nv; ++m) r[m] = F2(0.0f);
      amom<D, F2>(uf, ts, 1, -1, a, F2(-1.0f), r);
      if (MULTID) {
#pragma unroll
        for (int q = 0; q < D - 1; ++q) amom<D, F2>(uf, ts, 0, q, b[q], F2(-1.0f), r);
      }
      slope<D, F2>(gs, F2(bK), r, A);
    }
    // Abar rhs r4 rho/rho0 <(a u + b v) psi> + r5 rho/rho0 <A psi> and the flux
    // rho [T3 <u psi> + T5 <u A psi> + T4 (<u^2 a psi> + <u v b psi>)], over each side's half line
    const F2 s4 = F2(F2(r4 * i0) * gs.rho), s5 = F2(F2(r5 * i0) * gs.rho), s4f = F2(F2(Tc[4]) * gs.rho);
    F2 rh2[nv], F2s[nv];
#pragma unroll
    for (int m = 0; m < nv; ++m) rh2[m] = F2s[m] = F2(0.0f);
    amom2<D, F2>(hs, ts, 1, -1, a, s4, rh2, s4f, F2s);
    amom2<D, F2>(hs, ts, 0, -1, A, s5, rh2, F2(F2(Tc[5]) * gs.rho), F2s);
    {
      F2 m[nv];
      psi_mean<D, F2>(hs + 1, ts.m1, m);  // <u psi> over the half line
      const F2 s3 = F2(F2(Tc[3]) * gs.rho);
#pragma unroll
      for (int q = 0; q < nv; ++q) F2s[q] += s3 * m[q];
    }
    if (MULTID) {
#pragma unroll
      for (int q = 0; q < D - 1; ++q) amom2<D, F2>(hs, ts, 0, q, b[q], s4, rh2, s4f, F2s);
    }
#pragma unroll
    for (int m = 0; m < nv; ++m) {
      rhs[m] = rh2[m].v.x + rh2[m].v.y;
      F[m] = F2s[m].v.x + F2s[m].v.y;
    }
  }

  // equilibrium g0: Eq. eqlgform slopes from W_j -> w0 -> W_{j+1} (and the mean tangential slope)
  Trans<D, T> tr0;
  transverse<D, T>(g0, K, tr0);
  T oF[7], oP[7];
  u_full<D, T>(g0, oF);
  u_half<D, T>(g0, T(1), oP);
  {
    // lane x: abar_l on u > 0; lane y: abar_r on u < 0 (table = full line minus u > 0)
    const T fl = i0 * idxl, fr = i0 * idxr;
    Maxw<D, F2> g02;
    g02.rho = F2(g0.rho);
    g02.ir = F2(g0.ir);
#pragma unroll
    for (int i = 0; i < D; ++i) g02.U[i] = F2(g0.U[i]);
    g02.lam = F2(g0.lam);
    g02.il = F2(g0.il);
    g02.c = F2(g0.c);
    g02.f4 = F2(g0.f4);
    Trans<D, F2> t02;
#pragma unroll
    for (int b = 0; b <= D; ++b) {
      t02.m1[b] = F2(tr0.m1[b]);
#pragma unroll
      for (int c = 0; c <= D; ++c) t02.m2[b][c] = F2(tr0.m2[b][c]);
    }
    F2 r[nv], ab[nv], half[7];
#pragma unroll
    for (int m = 0; m < nv; ++m) r[m] = F2(F2(w0[m] - in.c(0, m), in.c(1, m) - w0[m]) * F2(fl, fr));
#pragma unroll
    for (int n = 0; n < 7; ++n) half[n] = F2(oP[n], oF[n] - oP[n]);
    slope<D, F2>(g02, F2(bK), r, ab);
    F2 rh2[nv], F2s[nv];
#pragma unroll
    for (int m = 0; m < nv; ++m) rh2[m] = F2s[m] = F2(0.0f);
    amom2<D, F2>(half, t02, 1, -1, ab, F2(r1), rh2, F2(Tc[1] * g0.rho), F2s);
#pragma unroll
    for (int m = 0; m < nv; ++m) {
      rhs[m] += rh2[m].v.x + rh2[m].v.y;
      F[m] += F2s[m].v.x + F2s[m].v.y;
    }
    if (MULTID) {
      const T s1f = Tc[1] * g0.rho;
      T rr[nv], abt[nv];
#pragma unroll
      for (int q = 0; q < D - 1; ++q) {
#pragma unroll
        for (int m = 0; m < nv; ++m) rr[m] = T(0.5) * (in.t(0, q, m) + in.t(1, q, m)) * i0;
        slope<D, T>(g0, bK, rr, abt);
        amom2<D, T>(oF, tr0, 0, q, abt, r1, rhs, s1f, F);
      }
    }
  }
  // Abar from the compatibility condition integrated over [0, dt]; flux rho0 <u (T0 + T2 Abar) psi>
  {
    T Ab[nv];
    slope<D, T>(g0, bK, rhs, Ab);
#pragma unroll
    for (int m = 0; m < nv; ++m) Ab[m] *= Tc[2];
    Ab[0] += Tc[0];
    amom<D, T>(oF, tr0, 1, -1, Ab, g0.rho, F);
  }
}

// face_flux_ps with the inputs in arrays, the inverse centre-to-face distances given.
template <int D, bool MULTID, bool RAR = false>
GKS_FN void face_flux_ps(const float* wl, const float* wr, const float* cl, const float* cr, const float* sl,
                         const float* sr, const float (*tl)[D + 2], const float (*tr)[D + 2], float dxl, float dxr,
                         float idxl, float idxr, float tau_t, float dt, const Gas<float>& gas, int abar_t0, float* F,
                         float* tau_out) {
  const FaceArrays<D, float> in{sl, sr, cl, cr, tl, tr};
  face_flux_ps<D, MULTID, RAR>(wl, wr, in, dxl, dxr, idxl, idxr, tau_t, dt, gas, abar_t0, F, tau_out);
}

// face_flux_ps with the inputs in arrays.
template <int D, bool MULTID, bool RAR = false>
GKS_FN void face_flux_ps(const float* wl, const float* wr, const float* cl, const float* cr, const float* sl,
                         const float* sr, const float (*tl)[D + 2], const float (*tr)[D + 2], float dxl, float dxr,
                         float tau_t, float dt, const Gas<float>& gas, int abar_t0, float* F, float* tau_out) {
  face_flux_ps<D, MULTID, RAR>(wl, wr, cl, cr, sl, sr, tl, tr, dxl, dxr, g_rcp(dxl), g_rcp(dxr), tau_t, dt, gas,
                               abar_t0, F, tau_out);
}

}  // namespace gks
