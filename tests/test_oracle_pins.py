"""Pins of the oracle's interface flux against things other than itself.

Each test checks one part of the oracle against quadrature of the defining integrals, a textbook
closed form or an invariant, so that a dropped term, a wrong sign or index or a transposed operand
in the oracle fails at least one of them.  No GPU is needed.
"""
import math

import numpy as np
import pytest
from scipy import integrate

import kinetic_quadrature as kq

GAMMA = 1.4


def K_of(D, gamma=GAMMA):
    return 2.0 / (gamma - 1.0) - D


def cons(D, rho, U, p, gamma=GAMMA):
    U = np.asarray(U, dtype=float)
    return np.concatenate([[rho], rho * U, [p / (gamma - 1.0) + 0.5 * rho * np.dot(U, U)]])


def rnd_state(rng, D):
    rho = rng.uniform(0.5, 2.0)
    U = rng.uniform(-0.8, 0.8, D)
    p = rng.uniform(0.3, 2.0)
    return cons(D, rho, U, p)


def diag_dict(dg, D):
    nv = D + 2
    g = lambda a: np.array(a[:nv])
    return {
        "w0": g(dg.w0), "al": g(dg.al), "ar": g(dg.ar), "Al": g(dg.Al), "Ar": g(dg.Ar),
        "abl": g(dg.abl), "abr": g(dg.abr), "Ab": g(dg.Ab),
        "bl": [g(dg.bl[k]) for k in range(2)], "br": [g(dg.br[k]) for k in range(2)],
        "bb": [g(dg.bb[k]) for k in range(2)], "tau": dg.tau, "T": np.array(dg.T[:6]),
    }


def rel(a, b):
    return np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(b), 1e-300)


# ------------------------------------------------------------------------------------------------
# Moments of the Maxwellian (Eq. maxwellian, Eq. moment1)
# ------------------------------------------------------------------------------------------------
@pytest.mark.parametrize("U,lam", [(0.0, 1.0), (0.37, 0.7), (-1.3, 2.5), (2.2, 0.4), (-0.05, 12.0)])
def test_umoments_match_quadrature(orc, U, lam):
    dens = lambda u: math.sqrt(lam / math.pi) * math.exp(-lam * (u - U) ** 2)
    full = orc.umoments(U, lam, orc.FULL, 8)
    pos = orc.umoments(U, lam, orc.POS, 8)
    neg = orc.umoments(U, lam, orc.NEG, 8)
    for n in range(9):
        qp = integrate.quad(lambda u: u ** n * dens(u), 0, np.inf, epsabs=0, epsrel=1e-13, limit=200)[0]
        qn = integrate.quad(lambda u: u ** n * dens(u), -np.inf, 0, epsabs=0, epsrel=1e-13, limit=200)[0]
        scale = integrate.quad(lambda u: abs(u) ** n * dens(u), -np.inf, np.inf, epsrel=1e-13, limit=200)[0]
        assert abs(pos[n] - qp) <= 1e-13 * scale
        assert abs(neg[n] - qn) <= 1e-13 * scale
        assert abs(full[n] - (qp + qn)) <= 1e-13 * scale


@pytest.mark.parametrize("K,lam", [(1.0, 1.0), (2.0, 0.6), (3.0, 2.0), (4.0, 0.9), (2.5, 1.7)])
def test_ximoments_match_radial_quadrature(orc, K, lam):
    # <(xi^2)^l> over R^K in radial form: int r^(K-1) r^(2l) e^{-lam r^2} dr / int r^(K-1) e^{-lam r^2} dr
    m = orc.ximoments(K, lam, 4)
    den = integrate.quad(lambda r: r ** (K - 1) * math.exp(-lam * r * r), 0, np.inf, epsrel=1e-13)[0]
    for l in range(5):
        num = integrate.quad(lambda r: r ** (K - 1 + 2 * l) * math.exp(-lam * r * r), 0, np.inf, epsrel=1e-13)[0]
        assert abs(m[l] - num / den) <= 5e-11 * num / den  # quad is less accurate at r^(K-1), K non-integer


@pytest.mark.parametrize("D", [1, 2, 3])
def test_state_moments_reproduce_conservative_state(D):
    # int psi g dXi = w for the Maxwellian built from w (pins the lambda of the energy definition)
    rng = np.random.default_rng(10 + D)
    K = K_of(D)
    for _ in range(3):
        w = rnd_state(rng, D)
        vel, xi2, wts = kq.nodes(D, K, w, "full")
        assert rel(kq.integrate(D, vel, xi2, wts, np.ones_like(xi2)), w) < 1e-13


@pytest.mark.parametrize("D", [1, 2, 3])
def test_slope_solves_moment_equation(orc, D):
    # <(a . psi) psi> = rhs, checked by quadrature (Eq. initialf0, slope coefficients)
    rng = np.random.default_rng(20 + D)
    K = K_of(D)
    for _ in range(4):
        w = rnd_state(rng, D)
        rhs = rng.normal(size=D + 2)
        a = orc.slope(D, K, w, rhs)
        vel, xi2, wts = kq.nodes(D, K, w, "full")
        lhs = kq.integrate(D, vel, xi2, wts, kq.expand(D, a, vel, xi2)) / w[0]
        assert rel(lhs, rhs) < 1e-12


# ------------------------------------------------------------------------------------------------
# Time integrals of Eq. resultingf
# ------------------------------------------------------------------------------------------------
@pytest.mark.parametrize("x", [1e-4, 0.03, 0.5, 0.999, 1.001, 3.0, 40.0])
def test_time_coeffs_match_quadrature(orc, x):
    """T0..T5 against 40-digit quadrature of their kernels (the kernels cancel badly at small x
    in double precision, so the reference is integrated in extended precision)."""
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.dps = 40
    tau = mpmath.mpf("1.3e-3")
    dt = mpmath.mpf(x) * tau
    T = orc.time_coeffs(float(dt), float(tau))
    e = lambda t: mpmath.exp(-t / tau)
    kern = [lambda t: 1 - e(t), lambda t: (tau + t) * e(t) - tau, lambda t: t - tau + tau * e(t),
            lambda t: e(t), lambda t: -(tau + t) * e(t), lambda t: -tau * e(t)]
    for k in range(6):
        q = float(mpmath.quad(kern[k], [0, dt]))
        assert abs(T[k] - q) <= 1e-13 * abs(q), (k, T[k], q)
    assert abs(T[6] - float(dt * dt / 2 - mpmath.quad(kern[2], [0, dt]))) <= 1e-13 * abs(T[6])


def test_time_coeffs_limits(orc):
    dt = 2e-3
    # tau -> 0 (x -> infinity): T0 -> dt, T1 -> -tau dt, T2 -> dt^2/2 - tau dt, T3..T5 -> 0
    T = orc.time_coeffs(dt, 0.0)
    assert np.allclose(T[:6], [dt, 0, 0.5 * dt * dt, 0, 0, 0], rtol=0, atol=1e-18)
    tau = 1e-9
    T = orc.time_coeffs(dt, tau)
    assert abs(T[1] + tau * dt) < 1e-6 * tau * dt
    # x -> 0: T0 ~ tau x^2 / 2 = dt^2 / (2 tau)
    tau = 1.0
    T = orc.time_coeffs(1e-6, tau)
    assert abs(T[0] - 0.5e-12) < 1e-6 * 0.5e-12
    # every coefficient is continuous across the series / closed-form switch at x = 1
    lo, hi = orc.time_coeffs(1.0 - 1e-12, 1.0), orc.time_coeffs(1.0 + 1e-12, 1.0)
    assert np.all(np.abs(lo - hi) <= 1e-11 * np.abs(hi) + 1e-15)


# ------------------------------------------------------------------------------------------------
# The interface flux
# ------------------------------------------------------------------------------------------------
def random_face(orc, rng, D, scale=0.2):
    wl = rnd_state(rng, D)
    wr = wl * (1 + scale * rng.uniform(-1, 1, D + 2))
    wr[D + 1] = cons(D, wr[0], wr[1:D + 1] / wr[0], rng.uniform(0.4, 1.5))[D + 1]
    h = rng.uniform(0.005, 0.02)
    sl, sr = rng.normal(size=D + 2) * 0.5, rng.normal(size=D + 2) * 0.5
    cl = wl - 0.5 * h * sl
    cr = wr + 0.5 * h * sr
    tl = rng.normal(size=(2, D + 2)) * 0.3
    tr = rng.normal(size=(2, D + 2)) * 0.3
    face = orc.make_face(D, wl, wr, cl, cr, sl, sr, tl[: D - 1], tr[: D - 1], 0.5 * h, 0.5 * h,
                         tau_t=rng.uniform(0, 2e-4))
    return face, dict(wl=wl, wr=wr, cl=cl, cr=cr, sl=sl, sr=sr, tl=tl, tr=tr, h=h)


CASES = [(1, 0, 1e-4, 0.0), (1, 0, 3e-3, 0.3), (2, 0, 5e-4, 0.0), (2, 1, 5e-4, 0.0), (2, 1, 4e-3, 0.5),
         (3, 1, 1e-3, 0.0)]


@pytest.mark.parametrize("D,multid,dt,C_a", CASES)
def test_face_coefficients_satisfy_their_definitions(orc, D, multid, dt, C_a):
    rng = np.random.default_rng(100 + 10 * D + multid)
    K = K_of(D)
    face, r = random_face(orc, rng, D)
    F, dg = orc.face_flux(D, GAMMA, 1e-5, C_a, dt, face, multid=multid, diag=True)
    d = diag_dict(dg, D)
    # Eq. intermediatestate: w0 = int_{u>0} psi g_l + int_{u<0} psi g_r
    vl, xl, wtl = kq.nodes(D, K, r["wl"], "pos")
    vr, xr, wtr = kq.nodes(D, K, r["wr"], "neg")
    w0 = kq.integrate(D, vl, xl, wtl, np.ones_like(xl)) + kq.integrate(D, vr, xr, wtr, np.ones_like(xr))
    assert rel(d["w0"], w0) < 1e-12
    for side, w, s, t, a, b, A in (("l", r["wl"], r["sl"], r["tl"], d["al"], d["bl"], d["Al"]),
                                   ("r", r["wr"], r["sr"], r["tr"], d["ar"], d["br"], d["Ar"])):
        vel, xi2, wts = kq.nodes(D, K, w, "full")
        # <a psi> = dW/dn / rho and <b psi> = dW/dt / rho
        assert rel(kq.integrate(D, vel, xi2, wts, kq.expand(D, a, vel, xi2)), s) < 1e-11
        for k in range(D - 1):
            tgt = t[k] if multid else np.zeros(D + 2)
            got = kq.integrate(D, vel, xi2, wts, kq.expand(D, b[k], vel, xi2))
            assert np.linalg.norm(got - tgt) <= 1e-11 * max(1.0, np.linalg.norm(tgt))
        # compatibility at t = 0: <(a u + b v + A) psi> = 0
        Q = kq.expand(D, a, vel, xi2) * vel[0] + kq.expand(D, A, vel, xi2)
        for k in range(D - 1):
            Q = Q + kq.expand(D, b[k], vel, xi2) * vel[1 + k]
        comp = kq.integrate(D, vel, xi2, wts, Q)
        assert np.linalg.norm(comp) < 1e-11 * np.linalg.norm(s)
    # Eq. eqlgform: <abar psi>_0 = (w0 - W_j)/dxl, (W_{j+1} - w0)/dxr
    vel, xi2, wts = kq.nodes(D, K, d["w0"], "full")
    h = r["h"]
    assert rel(kq.integrate(D, vel, xi2, wts, kq.expand(D, d["abl"], vel, xi2)), (d["w0"] - r["cl"]) / (0.5 * h)) < 1e-11
    assert rel(kq.integrate(D, vel, xi2, wts, kq.expand(D, d["abr"], vel, xi2)), (r["cr"] - d["w0"]) / (0.5 * h)) < 1e-11
    # Eq. relaxation time and Eq. taua
    p = lambda w: (GAMMA - 1) * (w[D + 1] - 0.5 * np.dot(w[1:D + 1], w[1:D + 1]) / w[0])
    tau = 1e-5 / p(d["w0"]) + face.tau_t + C_a * abs(p(r["wr"]) - p(r["wl"])) / (p(r["wr"]) + p(r["wl"])) * dt
    assert abs(d["tau"] - tau) < 1e-14 * tau


@pytest.mark.parametrize("D,multid,dt,C_a", CASES)
def test_face_flux_matches_kogan_quadrature(orc, D, multid, dt, C_a):
    """The flux equals int_0^dt int u psi f with f from Kogan's solution, both by quadrature; the
    quadrature also confirms that Abar satisfies the time-integrated compatibility condition."""
    rng = np.random.default_rng(200 + 10 * D + multid)
    K = K_of(D)
    face, r = random_face(orc, rng, D)
    F, dg = orc.face_flux(D, GAMMA, 1e-5, C_a, dt, face, multid=multid, diag=True)
    d = diag_dict(dg, D)
    Fq, compat = kq.face_flux_quadrature(D, K, r, d, dt)
    assert rel(F, Fq) < 1e-10, (F, Fq)
    # the compatibility residual is tiny relative to the size of each of its terms
    scale = np.linalg.norm(d["w0"]) * dt
    assert np.linalg.norm(compat) < 1e-11 * scale


@pytest.mark.parametrize("D", [1, 2, 3])
def test_compact_form_needs_corrected_beta(orc, D):
    """Eq. resultingf4 equals the exact time integral only with beta = exp(-1/eps)."""
    rng = np.random.default_rng(300 + D)
    face, _ = random_face(orc, rng, D)
    for dt in (2e-5, 1e-4, 1e-3):
        F = orc.face_flux(D, GAMMA, 1e-5, 0.0, dt, face)
        Fc = orc.face_flux_compact(D, GAMMA, 1e-5, 0.0, dt, face)
        assert rel(Fc, F) < 1e-13
    F = orc.face_flux(D, GAMMA, 1e-5, 0.0, 2e-5, face)
    Fp = orc.face_flux_compact(D, GAMMA, 1e-5, 0.0, 2e-5, face, printed_beta=True)
    assert rel(Fp, F) > 1e-6


@pytest.mark.parametrize("D", [1, 2, 3])
def test_euler_limit_equal_states(orc, D):
    """Equal states and zero slopes: F = dt F_Euler(w) for every tau (Section 2, Euler level)."""
    rng = np.random.default_rng(400 + D)
    w = rnd_state(rng, D)
    U = w[1:D + 1] / w[0]
    p = (GAMMA - 1) * (w[D + 1] - 0.5 * w[0] * np.dot(U, U))
    FE = np.concatenate([[w[1]], w[1] * U + p * (np.arange(D) == 0), [U[0] * (w[D + 1] + p)]])
    face = orc.make_face(D, w, w, tau_t=0.0)
    for mu in (0.0, 1e-6, 1e-3, 10.0):
        dt = 1e-3
        F = orc.face_flux(D, GAMMA, mu, 0.0, dt, face)
        assert rel(F, dt * FE) < 1e-14


def test_navier_stokes_limit_1d(orc):
    """Continuous linear data: F = dt F_E - tau dt (NS viscous flux with mu = tau p, Pr = 1)
    + dt^2/2 dF_E/dt, for any tau.  1D with K internal degrees of freedom: normal stress
    2K/(K+1) mu u_x, heat flux (K+3)/2 mu d(p/rho)/dx (Chapman-Enskog, Section 2)."""
    D, K = 1, K_of(1)
    g = GAMMA
    rng = np.random.default_rng(7)
    for tau_t in (1e-6, 1e-4, 3e-3):
        w = cons(1, 1.1, [0.3], 0.9)
        s = np.array([0.4, -0.25, 0.7])
        h = 0.01
        face = orc.make_face(1, w, w, w - 0.5 * h * s, w + 0.5 * h * s, s, s, None, None, 0.5 * h, 0.5 * h, tau_t)
        dt = 1e-3
        F, dg = orc.face_flux(1, g, 0.0, 0.0, dt, face, diag=True)
        tau = dg.tau
        rho, m, E = w
        u = m / rho
        p = (g - 1) * (E - 0.5 * rho * u * u)
        H = (E + p) / rho
        FE = np.array([m, m * u + p, u * (E + p)])
        J = np.array([[0.0, 1.0, 0.0],
                      [0.5 * (g - 3) * u * u, (3 - g) * u, g - 1],
                      [u * (0.5 * (g - 1) * u * u - H), H - (g - 1) * u * u, g * u]])
        dFdt = -J @ (J @ s)
        ux = (s[1] - u * s[0]) / rho
        px = (g - 1) * (s[2] - u * s[1] + 0.5 * u * u * s[0])
        Tx = (px - p / rho * s[0]) / rho
        mu = tau * p
        visc = np.array([0.0, -2 * K / (K + 1) * mu * ux, -2 * K / (K + 1) * mu * u * ux - (K + 3) / 2 * mu * Tx])
        Fns = dt * FE + dt * visc + 0.5 * dt * dt * dFdt
        assert rel(F, Fns) < 1e-12, (F, Fns)
        # A alone: rho <A psi> = dW/dt = -dF_E/dx
        vel, xi2, wts = kq.nodes(1, K, w, "full")
        At = kq.integrate(1, vel, xi2, wts, kq.expand(1, np.array(dg.Ar[:3]), vel, xi2))
        assert rel(At, -J @ s) < 1e-12
        # continuous data: Abar = A
        assert rel(np.array(dg.Ab[:3]), np.array(dg.Al[:3])) < 1e-10


def test_two_dim_flux_reduces_to_one_dim(orc):
    """A 2D gas with no tangential gradients is a 1D gas with one more internal degree of freedom
    (same gamma); a tangential velocity V adds V F_rho to F_v and V^2/2 F_rho to F_E."""
    rng = np.random.default_rng(11)
    for V in (0.0, 0.45):
        rl, ul, pl = 1.2, 0.2, 1.1
        rr, ur, pr = 0.8, -0.1, 0.7
        w1l, w1r = cons(1, rl, [ul], pl), cons(1, rr, [ur], pr)
        w2l, w2r = cons(2, rl, [ul, V], pl), cons(2, rr, [ur, V], pr)
        s1l, s1r = np.array([0.3, 0.1, -0.2]), np.array([-0.1, 0.2, 0.4])
        # the same primitive slopes in 2D (tangential velocity constant)
        s2l = np.array([s1l[0], s1l[1], V * s1l[0], s1l[2] + 0.5 * V * V * s1l[0]])
        s2r = np.array([s1r[0], s1r[1], V * s1r[0], s1r[2] + 0.5 * V * V * s1r[0]])
        h = 0.01
        f1 = orc.make_face(1, w1l, w1r, w1l - 0.5 * h * s1l, w1r + 0.5 * h * s1r, s1l, s1r, None, None, 0.5 * h, 0.5 * h, 1e-4)
        f2 = orc.make_face(2, w2l, w2r, w2l - 0.5 * h * s2l, w2r + 0.5 * h * s2r, s2l, s2r, None, None, 0.5 * h, 0.5 * h, 1e-4)
        F1 = orc.face_flux(1, GAMMA, 1e-5, 0.2, 1e-3, f1)
        F2 = orc.face_flux(2, GAMMA, 1e-5, 0.2, 1e-3, f2)
        exp2 = np.array([F1[0], F1[1], V * F1[0], F1[2] + 0.5 * V * V * F1[0]])
        assert rel(F2, exp2) < 1e-13
