"""Pins of the rarefaction option of the oracle (Eqs. tautautilde, tautilde, rarefactionkepsilon,
epsilonkomega; reading G9): the degree of rarefaction eps = tau/tauhat, tauhat = rho/|D rho| at the
face with D rho = d_t rho + U_n d_n rho, replaces tau/dt inside alpha and beta of Eq. fkepsilon.

  - the T0..T5 written with eps equal the exact time-integral coefficients (themselves pinned by
    quadrature) when eps = tau/dt, on both sides of the series / closed-form switch;
  - the flux of the option equals the paper's compact form (Eq. fkepsilon with alpha = eps
    (1 - e^{-1/eps}), beta = e^{-1/eps}) with eps = tau/tauhat, and differs from the printed beta;
  - for continuous linear data tauhat is the closed form rho0 / |d_t rho + U_n d_n rho| with
    d_t rho = -div(rho U) (the tangential part from the tangential slopes of the multi-dimensional
    expansion) and d_n rho the normal density gradient;
  - uniform flow: |D rho| is rounding noise (tauhat above 1e10 dt, capped at 1e30, eps -> 0) and the
    flux is dt times the Euler flux.
"""
import numpy as np
import pytest

import oracle

GAMMA = 1.4


def cons(D, rho, U, p):
    U = np.asarray(U, dtype=float)
    return np.concatenate([[rho], rho * U, [p / (GAMMA - 1.0) + 0.5 * rho * np.dot(U, U)]])


@pytest.mark.parametrize("x", [1e-4, 0.3, 0.999, 1.0, 1.001, 3.0, 40.0, 1e4])
def test_coefficients_with_eps_equal_tau_over_dt_are_the_time_integral(x):
    dt = 2e-3
    tau = dt / x
    T = oracle.time_coeffs(dt, tau)
    Th = oracle.time_coeffs_hat(dt, tau, tau / dt)
    # relative 1e-13, or 1e-15 of each coefficient's natural size (T2 = dt (dt/2 - tau (1 - alpha)) is
    # a difference of two terms of size dt^2/2 when eps is large)
    scale = np.array([dt, dt * tau, dt * dt, dt, dt * tau, dt * tau, dt * tau])
    assert np.all(np.abs(Th - T) <= 1e-13 * np.abs(T) + 1e-15 * scale), (T, Th)


def random_face(rng, D):
    nv = D + 2
    wl = cons(D, rng.uniform(0.5, 1.5), rng.uniform(-0.8, 0.8, D), rng.uniform(0.4, 1.5))
    wr = cons(D, rng.uniform(0.5, 1.5), rng.uniform(-0.8, 0.8, D), rng.uniform(0.4, 1.5))
    h = rng.uniform(0.01, 0.05)
    sl, sr = rng.normal(size=nv), rng.normal(size=nv)
    tl = rng.normal(size=(max(D - 1, 1), nv))
    tr = rng.normal(size=(max(D - 1, 1), nv))
    return oracle.make_face(D, wl, wr, wl - 0.5 * h * sl, wr + 0.5 * h * sr, sl, sr, tl[: D - 1], tr[: D - 1],
                            0.5 * h, 0.5 * h, rng.uniform(0.0, 2e-3))


@pytest.mark.parametrize("D,multid", [(1, 0), (2, 0), (2, 1), (3, 1)])
def test_option_flux_is_the_compact_form_with_eps_tau_over_tauhat(D, multid):
    rng = np.random.default_rng(50 + 10 * D + multid)
    dt = 1e-3
    for _ in range(40):
        f = random_face(rng, D)
        F, dg = oracle.face_flux(D, GAMMA, 2e-5, 0.3, dt, f, multid=multid, diag=True, rarefaction=1)
        Fc = oracle.face_flux_compact(D, GAMMA, 2e-5, 0.3, dt, f, multid=multid, rarefaction=1)
        Fp = oracle.face_flux_compact(D, GAMMA, 2e-5, 0.3, dt, f, multid=multid, rarefaction=1, printed_beta=True)
        F0 = oracle.face_flux(D, GAMMA, 2e-5, 0.3, dt, f, multid=multid)
        assert 0.0 < dg.tauhat < 1e30
        assert np.linalg.norm(F - Fc) <= 1e-12 * np.linalg.norm(F), (F, Fc)
        # not vacuous: the printed beta and the plain tau/dt form give other fluxes when eps is large
        eps = dg.tau / dg.tauhat
        if eps > 0.05:
            assert np.linalg.norm(Fp - F) > 1e-9 * np.linalg.norm(F)
        if abs(eps - dg.tau / dt) > 0.1 * eps:
            assert np.linalg.norm(F0 - F) > 1e-9 * np.linalg.norm(F)


def linear_face(D, W0, Gn, Gt, h):
    """Face record of conservative fields linear in the normal (gradient Gn) and tangential (Gt)
    directions: cell averages are the centre values, face values W0, slopes the gradients."""
    return oracle.make_face(D, W0, W0, W0 - 0.5 * h * Gn, W0 + 0.5 * h * Gn, Gn, Gn,
                            None if D == 1 else [Gt] * (D - 1), None if D == 1 else [Gt] * (D - 1),
                            0.5 * h, 0.5 * h, 1e-4)


@pytest.mark.parametrize("D,multid", [(1, 0), (2, 0), (2, 1)])
def test_tauhat_of_linear_data_is_the_closed_form(D, multid):
    rng = np.random.default_rng(7 + D + multid)
    for _ in range(10):
        W0 = cons(D, rng.uniform(0.6, 1.4), rng.uniform(-0.7, 0.7, D), rng.uniform(0.5, 1.5))
        Gn = rng.normal(size=D + 2)
        Gt = rng.normal(size=D + 2)
        h = rng.uniform(0.005, 0.02)
        f = linear_face(D, W0, Gn, Gt, h)
        _, dg = oracle.face_flux(D, GAMMA, 1e-5, 0.0, 1e-3, f, multid=multid, diag=True, rarefaction=1)
        rho0, Un = W0[0], W0[1] / W0[0]
        dt_rho = -Gn[1] - (Gt[2] if (D == 2 and multid) else 0.0)  # -div(rho U)
        dn_rho = Gn[0]
        expect = rho0 / abs(dt_rho + Un * dn_rho)
        assert abs(dg.tauhat - expect) <= 1e-11 * expect, (dg.tauhat, expect)
        # the same field sampled on cells twice as wide: a property of the flow, not of the grid
        _, dg2 = oracle.face_flux(D, GAMMA, 1e-5, 0.0, 1e-3, linear_face(D, W0, Gn, Gt, 2 * h), multid=multid,
                                  diag=True, rarefaction=1)
        assert abs(dg2.tauhat - expect) <= 1e-11 * expect


@pytest.mark.parametrize("D", [1, 2, 3])
def test_uniform_flow_caps_tauhat_and_gives_the_euler_flux(D):
    w = cons(D, 0.9, np.linspace(0.3, -0.2, D), 0.8)
    f = oracle.make_face(D, w, w, w, w, dxl=0.01, dxr=0.01, tau_t=1e-3)
    dt = 1e-3
    F, dg = oracle.face_flux(D, GAMMA, 1e-5, 0.0, dt, f, diag=True, rarefaction=1)
    assert dg.tauhat > 1e10 * dt  # |D rho| is rounding noise: eps = tau/tauhat below 1e-10
    Fe = dt * oracle.euler_flux(D, GAMMA, w)
    assert np.linalg.norm(F - Fe) <= 1e-13 * np.linalg.norm(Fe)
