"""Pins of the oracle's k-omega transport step (Wilcox's 2006 k-omega model, which the paper's
Section 4 cites for the two transport equations solved with the flow).  Each test checks the
oracle against something independent of its own formulas: the closed-form solution of the
homogeneous-decay ODEs, a hand evaluation of the production of a uniform shear, the exact discrete
decay of a Fourier mode under the three-point diffusion operator, and translation by a uniform
stream."""
import math

import numpy as np
import pytest

import oracle

GAMMA = 1.4
BETA0, BETA_STAR, ALPHA, C_LIM = 0.0708, 0.09, 13.0 / 25.0, 7.0 / 8.0


def uniform_case(dim, n, u=(0.0, 0.0, 0.0), mu=1e-5, bc=None):
    L = 1.0
    dx = [np.full(n[d], L / n[d]) for d in range(dim)]
    bc = bc or [(oracle.BC_PERIODIC, oracle.BC_PERIODIC)] * dim
    case = oracle.Case(dim, n, dx, bc, gamma=GAMMA, mu=mu, turb_model=oracle.TURB_KOMEGA, beta_star=BETA_STAR)
    ncell = int(np.prod(n[:dim]))
    prim = np.zeros((dim + 2, ncell))
    prim[0] = 1.0
    for d in range(dim):
        prim[1 + d] = u[d]
    prim[dim + 1] = 1.0 / GAMMA
    return case, case.prim_to_cons(prim.ravel()), ncell


def test_homogeneous_decay_matches_closed_form():
    """No gradients: d omega/dt = -beta0 omega^2, d k/dt = -beta* k omega.  The point-implicit
    destruction makes omega exact (1/omega grows by beta0 dt per step); k converges to
    k0 (1 + beta0 omega0 t)^(-beta*/beta0) at first order in dt."""
    k0, w0, T = 0.02, 40.0, 0.05
    errs = []
    for nsteps in (50, 100, 200):
        case, W, ncell = uniform_case(2, (4, 4))
        RK = np.full(ncell, k0)
        RW = np.full(ncell, w0)
        dt = T / nsteps
        for _ in range(nsteps):
            W, RK, RW, st = case.step_komega(W, RK, RW, dt)
            assert st == 0
        w_exact = 1.0 / (1.0 / w0 + BETA0 * T)
        k_exact = k0 * (1.0 + BETA0 * w0 * T) ** (-BETA_STAR / BETA0)
        assert np.allclose(RW, w_exact, rtol=1e-12, atol=0)
        assert np.ptp(RK) == 0.0
        errs.append(abs(RK[0] - k_exact) / k_exact)
    assert errs[0] < 0.02
    for a, b in zip(errs, errs[1:]):
        assert 1.8 < a / b < 2.2  # first order in dt


@pytest.mark.parametrize("omega0", [50.0, 0.5])
def test_uniform_shear_production_and_stress_limiter(omega0):
    """u = S y, uniform k and omega: P = mu_T S^2 with mu_T = rho k / omega~, omega~ = max(omega,
    C_lim S / sqrt(beta*)) (2 Sbar:Sbar = S^2); omega production alpha rho (omega/omega~) S^2."""
    nx, ny, S, k0, dt = 4, 16, 2.0, 0.01, 1e-4
    case = oracle.Case(2, (nx, ny), [np.full(nx, 1.0 / nx), np.full(ny, 1.0 / ny)],
                       [(oracle.BC_PERIODIC, oracle.BC_PERIODIC), (oracle.BC_TRANSMISSIVE, oracle.BC_TRANSMISSIVE)],
                       gamma=GAMMA, mu=1e-5, turb_model=oracle.TURB_KOMEGA, beta_star=BETA_STAR)
    y = (np.arange(ny) + 0.5) / ny
    prim = np.zeros((4, ny, nx))
    prim[0] = 1.0
    prim[1] = S * y[:, None]
    prim[3] = 1.0 / GAMMA
    W = case.prim_to_cons(prim.ravel())
    RK = np.full(nx * ny, k0)
    RW = np.full(nx * ny, omega0)
    W1, RK1, RW1, st = case.step_komega(W, RK, RW, dt)
    assert st == 0
    # uniform k and omega are carried with the mass: advection alone gives k rho^{n+1}, omega rho^{n+1}
    rho1 = W1[:nx * ny]
    wt = max(omega0, C_LIM * S / math.sqrt(BETA_STAR))
    P = k0 / wt * S * S
    rk = (k0 * rho1 + dt * P) / (1.0 + dt * BETA_STAR * omega0)
    rw = (omega0 * rho1 + dt * ALPHA * (omega0 / wt) * S * S) / (1.0 + dt * BETA0 * omega0)
    inner = np.s_[2:ny - 2, :]
    assert np.allclose(RK1.reshape(ny, nx)[inner], rk.reshape(ny, nx)[inner], rtol=1e-12, atol=0)
    assert np.allclose(RW1.reshape(ny, nx)[inner], rw.reshape(ny, nx)[inner], rtol=1e-12, atol=0)
    # the production itself is not small here: it moves rho k by more than the tolerance
    assert abs(rk.mean() - k0 * rho1.mean() / (1.0 + dt * BETA_STAR * omega0)) > 1e-8


def test_diffusion_of_a_fourier_mode_is_exact():
    """Fluid at rest, sources off, sigma* = 0: rho k evolves by k_i += dt mu/rho (k_{i+1} - 2 k_i +
    k_{i-1}) / h^2, so a Fourier mode decays by exactly (1 - dt mu/rho 4/h^2 sin^2(kappa h/2)) per
    step."""
    n, mu, dt, steps = 32, 0.05, 1e-4, 40
    case, W, ncell = uniform_case(1, (n,), mu=mu)
    h = 1.0 / n
    x = (np.arange(n) + 0.5) * h
    kappa = 2 * math.pi * 3
    RK = 0.01 * (1.0 + 0.1 * np.cos(kappa * x))
    RW = np.full(n, 1e3)
    c = oracle.komega_defaults(sources=0, sigma_star=0.0)
    for _ in range(steps):
        W, RK, RW, st = case.step_komega(W, RK, RW, dt, coeffs=c)
        assert st == 0
    g = (1.0 - dt * mu * 4.0 / h ** 2 * math.sin(kappa * h / 2) ** 2) ** steps
    expect = 0.01 * (1.0 + 0.1 * g * np.cos(kappa * x))
    assert np.allclose(RK, expect, rtol=1e-12, atol=0)
    assert np.allclose(RW, 1e3, rtol=1e-13)


def test_advection_by_a_uniform_stream():
    """rho = 1, u = 0.5 uniform, sources and diffusion off: k translates with the stream (upwinding
    by the sign of the GKS mass flux, half-time MUSCL face values); the error falls at second order
    with resolution, the total is conserved to round-off on a periodic grid."""
    u, T = 0.5, 1.0
    errs = []
    for n in (64, 128):
        case, W, ncell = uniform_case(1, (n,), u=(u, 0, 0), mu=1e-6)
        x = (np.arange(n) + 0.5) / n
        k = lambda xx: 0.01 * (1.0 + 0.5 * np.sin(2 * math.pi * xx))
        RK = k(x)
        RW = np.full(n, 10.0)
        c = oracle.komega_defaults(sources=0, diffusion=0)
        dt = 0.4 / n / (u + math.sqrt(1.0))  # CFL 0.4 with c = 1
        steps = int(round(T / dt))
        dt = T / steps
        total0 = RK.sum()
        for _ in range(steps):
            W, RK, RW, st = case.step_komega(W, RK, RW, dt, coeffs=c)
            assert st == 0
        assert abs(RK.sum() - total0) <= 1e-13 * total0 * steps
        errs.append(np.abs(RK - k(x - u * T)).mean() / 0.01)
    assert errs[0] < 0.005
    assert errs[0] / errs[1] > 3.5  # second order


def test_flow_step_uses_k_and_omega_of_the_transported_fields():
    """The flow half of the coupled step is orc_step with f1 = RK/rho, f2 = RW/rho."""
    rng = np.random.default_rng(5)
    n = (12, 10)
    case, W, ncell = uniform_case(2, n, u=(0.2, -0.1, 0))
    prim = case.cons_to_prim(W).reshape(4, ncell)
    prim[0] *= 1.0 + 0.05 * rng.standard_normal(ncell)
    prim[1] += 0.05 * rng.standard_normal(ncell)
    W = case.prim_to_cons(prim.ravel())
    RK = 0.01 * (1.0 + 0.3 * rng.random(ncell)) * prim[0]
    RW = 20.0 * (1.0 + 0.3 * rng.random(ncell)) * prim[0]
    dt = 0.3 * case.compute_dt(W, 1.0)
    W1, _, _, st = case.step_komega(W, RK, RW, dt)
    W2, st2, _ = case.step(W, dt, f1=RK / prim[0], f2=RW / prim[0])
    assert st == 0 and st2 == 0
    assert np.array_equal(W1, W2)
