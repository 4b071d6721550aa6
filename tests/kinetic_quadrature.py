"""Independent numerical evaluation of velocity-space and time integrals (test pin only).

Everything here is computed from point values of the distribution functions, by quadrature, with
no moment recursion and no polynomial algebra:
  * velocity space: the normal velocity on a half line by composite Gauss-Legendre, tangential
    velocities by Gauss-Hermite, the K internal degrees of freedom in radial form by generalised
    Gauss-Laguerre in s = lambda |xi|^2;
  * time: Kogan's integral solution (Eq. integralbgk) at the interface, with the inner integral over
    t' and the outer one over [0, dt] both by composite Gauss-Legendre.
"""
import math

import numpy as np
from numpy.polynomial.hermite import hermgauss
from numpy.polynomial.legendre import leggauss
from scipy.special import roots_genlaguerre


def maxwellian_params(D, K, w):
    """rho, U (D,), lambda from a conservative state (definition of E in Section 2)."""
    rho = w[0]
    U = np.array([w[1 + i] / rho for i in range(D)])
    lam = (K + D) * rho / (4.0 * (w[D + 1] - 0.5 * rho * np.dot(U, U)))
    return rho, U, lam


def _half_line(U, lam, region, panels=48, order=16):
    s = 1.0 / math.sqrt(lam)
    lo, hi = U - 15 * s, U + 15 * s
    if region == "pos":
        lo = max(lo, 0.0)
    elif region == "neg":
        hi = min(hi, 0.0)
    if hi <= lo:
        return np.zeros(0), np.zeros(0)
    gx, gw = leggauss(order)
    h = (hi - lo) / panels
    xs = np.concatenate([lo + k * h + 0.5 * h * (gx + 1) for k in range(panels)])
    ws = np.concatenate([0.5 * h * gw for _ in range(panels)])
    dens = math.sqrt(lam / math.pi) * np.exp(-lam * (xs - U) ** 2)
    return xs, ws * dens


def nodes(D, K, w, region, n_herm=14, n_lag=10):
    """Quadrature nodes and weights (weights include rho and the Maxwellian density) for
    integrals over velocity space of g(w) times a smooth function; region = full|pos|neg in u."""
    rho, U, lam = maxwellian_params(D, K, w)
    if region == "full":
        z, wz = hermgauss(40)
        ux, uw = U[0] + z / math.sqrt(lam), wz / math.sqrt(math.pi)
    else:
        ux, uw = _half_line(U[0], lam, region)
    axes = [ux]
    wts = [uw]
    for t in range(1, D):
        z, wz = hermgauss(n_herm)
        axes.append(U[t] + z / math.sqrt(lam))
        wts.append(wz / math.sqrt(math.pi))
    if K > 0:
        s, ws = roots_genlaguerre(n_lag, K / 2.0 - 1.0)
        axes.append(s / lam)  # xi^2
        wts.append(ws / math.gamma(K / 2.0))
    else:
        axes.append(np.zeros(1))
        wts.append(np.ones(1))
    grids = np.meshgrid(*axes, indexing="ij")
    wgrid = np.ones_like(grids[0])
    for a, wa in enumerate(wts):
        shape = [1] * len(wts)
        shape[a] = len(wa)
        wgrid = wgrid * wa.reshape(shape)
    vel = [g.ravel() for g in grids[:D]]
    xi2 = grids[D].ravel()
    return vel, xi2, rho * wgrid.ravel()


def psi(D, vel, xi2):
    """psi = (1, u_1..u_D, (|u|^2 + xi^2)/2) at the nodes, shape (nv, n)."""
    e = 0.5 * (sum(v * v for v in vel) + xi2)
    return np.vstack([np.ones_like(xi2)] + list(vel) + [e])


def expand(D, a, vel, xi2):
    """a . psi at the nodes."""
    return np.asarray(a[: D + 2]) @ psi(D, vel, xi2)


def integrate(D, vel, xi2, wts, fvals, with_u=False):
    """int psi (u) f dXi as a vector (nv,)."""
    p = psi(D, vel, xi2)
    if with_u:
        p = p * vel[0]
    return p @ (wts * fvals)


def _gl(a, b, panels, order=12):
    gx, gw = leggauss(order)
    h = (b - a) / panels
    xs = np.concatenate([a + k * h + 0.5 * h * (gx + 1) for k in range(panels)])
    ws = np.concatenate([0.5 * h * gw for _ in range(panels)])
    return xs, ws


def kogan_time_integrals(dt, tau, panels=None):
    """Nested quadrature of the time factors of Kogan's solution at the interface:
        c1(t) = (1/tau) int_0^t e^{-(t-t')/tau} dt',   c2(t) = (1/tau) int_0^t (t-t') e^{..} dt',
        c3(t) = (1/tau) int_0^t t' e^{..} dt',          c4(t) = e^{-t/tau},  c5(t) = t e^{-t/tau};
    returns their integrals over t in [0, dt] (C1..C5)."""
    if panels is None:
        panels = int(min(400, max(40, 4 * dt / tau)))
    ts, wt = _gl(0.0, dt, panels)
    C = np.zeros(5)
    for t, w in zip(ts, wt):
        sp, sw = _gl(0.0, t, panels)  # t'
        k = np.exp(-(t - sp) / tau) / tau
        C[0] += w * np.sum(sw * k)
        C[1] += w * np.sum(sw * k * (t - sp))
        C[2] += w * np.sum(sw * k * sp)
        C[3] += w * math.exp(-t / tau)
        C[4] += w * t * math.exp(-t / tau)
    return C


def face_flux_quadrature(D, K, face, diag, dt):
    """Time-integrated flux int_0^dt int u psi f dXi dt with f from Kogan's integral solution,
    the initial state f0 = g_{l,r} (1 + a x + b y - tau (a u + b v + A)) and the equilibrium
    g = g0 (1 + abar x + bbar y + Abar t), every integral done by quadrature.  The slope and time
    coefficients are taken from ``diag`` (they are pinned separately by their defining equations).
    Also returns the residual of the time-integrated compatibility condition that defines Abar."""
    tau = diag["tau"]
    C1, C2, C3, C4, C5 = kogan_time_integrals(dt, tau)
    F = np.zeros(D + 2)
    compat = np.zeros(D + 2)
    w0 = diag["w0"]
    # equilibrium part, g0 on u>0 (abar_l) and u<0 (abar_r)
    for region, ab in (("pos", diag["abl"]), ("neg", diag["abr"])):
        vel, xi2, wts = nodes(D, K, w0, region)
        Pa = expand(D, ab, vel, xi2) * vel[0]
        for k in range(D - 1):
            Pa = Pa + expand(D, diag["bb"][k], vel, xi2) * vel[1 + k]
        PA = expand(D, diag["Ab"], vel, xi2)
        fint = C1 - C2 * Pa + C3 * PA  # time integral of the equilibrium part at each node
        F += integrate(D, vel, xi2, wts, fint, with_u=True)
        # int_0^dt (g - f) dt: g(0, t) = g0 (1 + Abar t)
        compat += integrate(D, vel, xi2, wts, dt + 0.5 * dt * dt * PA - fint)
    # non-equilibrium part, g_l on u>0, g_r on u<0
    for region, w, a, b, A in (("pos", face["wl"], diag["al"], diag["bl"], diag["Al"]),
                               ("neg", face["wr"], diag["ar"], diag["br"], diag["Ar"])):
        vel, xi2, wts = nodes(D, K, w, region)
        Q = expand(D, a, vel, xi2) * vel[0]
        for k in range(D - 1):
            Q = Q + expand(D, b[k], vel, xi2) * vel[1 + k]
        PA = expand(D, A, vel, xi2)
        fint = C4 * (1.0 - tau * (Q + PA)) - C5 * Q
        F += integrate(D, vel, xi2, wts, fint, with_u=True)
        compat -= integrate(D, vel, xi2, wts, fint)
    return F, compat
