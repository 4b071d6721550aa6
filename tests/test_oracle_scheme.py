"""Pins of the oracle's whole scheme (reconstruction, boundary cells, CFL step, update, relaxation-
time field) against exact solutions and invariants."""
import math

import numpy as np
import pytest

import exact_riemann as er
from paper_1302_2132_gb300 import inputs

GAMMA = 1.4


def case_from(orc, spec, **kw):
    args = dict(gamma=GAMMA, mu=kw.pop("mu", 1e-5))
    args.update(kw)
    return orc.Case(spec["dim"], spec["n"], spec["dx"], spec["bc"], bc_prim=spec.get("bc_prim"), **args)


def test_exact_riemann_solver_textbook_star_state():
    # Toro, Riemann Solvers and Numerical Methods for Fluid Dynamics, Table 4.2, Test 1 (Sod)
    p, u = er.star_state((1.0, 0.0, 1.0), (0.125, 0.0, 0.1))
    assert abs(p - 0.30313) < 5e-6
    assert abs(u - 0.92745) < 5e-6


def sod_l1(orc, n, limiter):
    s = inputs.sod_1d(n)
    c = case_from(orc, s, C_a=1.0, limiter=limiter)
    W = c.prim_to_cons(s["prim"].ravel())
    W, t, steps, st = c.run(W, 100000, cfl=0.5, t_end=0.2, nthreads=4)
    assert st == 0 and abs(t - 0.2) < 1e-14
    edges = np.linspace(0.0, 1.0, n + 1)
    ex = er.cell_average((1.0, 0.0, 1.0), (0.125, 0.0, 0.1), edges, 0.2, sub=16)
    rho = W.reshape(3, n)[0]
    return np.sum(np.abs(rho - ex[0])) / n


@pytest.mark.slow
def test_sod_converges_to_exact_solution(orc):
    errs = [sod_l1(orc, n, orc.LIM_VANLEER) for n in (50, 100, 200, 400)]
    assert all(b < a for a, b in zip(errs, errs[1:])), errs
    order = math.log(errs[1] / errs[3]) / math.log(4.0)
    assert order >= 0.7, (errs, order)
    assert errs[2] < 0.01  # 400-cell Sod: L1(rho) of order 1e-3 for second-order schemes
    e_mm = sod_l1(orc, 100, orc.LIM_MINMOD)
    assert e_mm < 2.0 * errs[1]


def test_periodic_grid_conserves_mass_momentum_energy(orc):
    s = inputs.random_smooth_2d(20, seed=5)
    s["n"] = (20, 20)
    rng = np.random.default_rng(1)
    kf = 0.05 * (1 + 0.5 * rng.random(400))
    ef = 50.0 * (1 + 0.5 * rng.random(400))
    c = case_from(orc, s, turb_model=orc.TURB_KEPS, C_a=0.3)
    W0 = c.prim_to_cons(s["prim"].ravel())
    vol = (2 * math.pi / 20) ** 2
    tot0 = W0.reshape(4, -1).sum(axis=1) * vol
    W = W0
    for _ in range(8):
        dt = c.compute_dt(W, 0.5)
        W, st, res = c.step(W, dt, f1=kf, f2=ef, nthreads=4)
        assert st == 0
    tot = W.reshape(4, -1).sum(axis=1) * vol
    absmass = np.abs(W0.reshape(4, -1)).sum(axis=1) * vol
    assert np.all(np.abs(tot - tot0) <= 1e-13 * absmass), (tot - tot0) / absmass
    assert np.allclose(res[2], tot, rtol=1e-14, atol=1e-14 * absmass.max())


def test_free_stream_preserved_on_stretched_grid(orc):
    rng = np.random.default_rng(3)
    n = (11, 9)
    dx = [rng.uniform(0.5, 2.0, n[0]) * 0.1, rng.uniform(0.5, 2.0, n[1]) * 0.1]
    prim = np.zeros((4, n[1], n[0]))
    prim[0], prim[1], prim[2], prim[3] = 1.3, 0.4, -0.7, 0.9
    for bc in ([[1, 1], [1, 1]], [[0, 0], [0, 0]]):
        c = orc.Case(2, n, dx, bc, gamma=GAMMA, mu=1e-3, turb_model=orc.TURB_KOMEGA, C_a=0.5)
        W0 = c.prim_to_cons(prim.ravel())
        kf = rng.uniform(0.01, 0.1, n[0] * n[1])
        of = rng.uniform(10, 100, n[0] * n[1])
        W = W0
        for _ in range(3):
            W, st, _ = c.step(W, 1e-3, f1=kf, f2=of)
        assert np.max(np.abs(W - W0) / np.abs(W0).max()) < 1e-14


def test_dirichlet_inflow_and_outflow_keep_uniform_supersonic_stream(orc):
    n = (12, 8)
    dx = [np.full(12, 0.05), np.linspace(0.01, 0.05, 8)]
    state = np.array([1.0, 2.5, 0.3, 1.0 / GAMMA])
    bcp = [[np.tile(state, (8, 1)), None], [None, np.tile(state, (12, 1))]]
    c = orc.Case(2, n, dx, [[3, 4], [4, 3]], gamma=GAMMA, mu=1e-4, bc_prim=bcp)
    prim = np.broadcast_to(state[:, None, None], (4, 8, 12)).copy()
    W0 = c.prim_to_cons(prim.ravel())
    W = W0
    for _ in range(3):
        W, st, _ = c.step(W, 2e-3)
    assert np.max(np.abs(W - W0)) < 1e-14 * np.abs(W0).max()


def test_wall_mirror_symmetry(orc):
    """Isothermal no-slip walls at both ends of a tube with mirror-symmetric data: the solution
    stays mirror-symmetric (rho, p even, u odd)."""
    n = 40
    x = (np.arange(n) + 0.5) / n
    prim = np.zeros((3, n))
    prim[0] = 1.0 + 0.3 * np.cos(2 * math.pi * x)
    prim[1] = 0.2 * np.sin(4 * math.pi * x)
    prim[2] = 1.0 + 0.2 * np.cos(2 * math.pi * x) ** 2
    c = orc.Case(1, (n,), [np.full(n, 1.0 / n)], [[2, 2]], gamma=GAMMA, mu=1e-3, T_wall=0.9, C_a=0.5)
    W = c.prim_to_cons(prim.ravel())
    for _ in range(20):
        W, st, _ = c.step(W, 2e-3)
        assert st == 0
    P = c.cons_to_prim(W).reshape(3, n)
    assert np.max(np.abs(P[0] - P[0][::-1])) < 1e-12
    assert np.max(np.abs(P[1] + P[1][::-1])) < 1e-12
    assert np.max(np.abs(P[2] - P[2][::-1])) < 1e-12


def test_cfl_step_closed_form(orc):
    n = (6, 5)
    dx = [np.full(6, 0.1), np.full(5, 0.2)]
    prim = np.zeros((4, 5, 6))
    prim[0], prim[1], prim[2], prim[3] = 2.0, 0.5, -0.25, 1.5
    c = orc.Case(2, n, dx, [[0, 0], [0, 0]], gamma=GAMMA)
    cs = math.sqrt(GAMMA * 1.5 / 2.0)
    dt = c.compute_dt(c.prim_to_cons(prim.ravel()), 0.5)
    assert abs(dt - 0.5 / ((0.5 + cs) / 0.1 + (0.25 + cs) / 0.2)) < 1e-15


def test_turbulent_relaxation_time_field(orc):
    """Eqs. tauttrivial, tautchen, tautchenadjusted with T = p/rho: mu_t mode gives mu_t/p;
    k-epsilon and k-omega agree when omega = epsilon/(C_mu k) and beta* = C_mu; a linear shear
    U = (alpha y, 0) has S = |alpha|."""
    n = (8, 10)
    h = 0.1
    y = (np.arange(n[1]) + 0.5) * h
    alpha = 0.7
    prim = np.zeros((4, n[1], n[0]))
    prim[0] = 1.2
    prim[1] = alpha * y[:, None]
    prim[3] = 0.8
    rng = np.random.default_rng(9)
    k = rng.uniform(0.01, 0.05, n[0] * n[1])
    eps = rng.uniform(0.5, 2.0, n[0] * n[1])
    base = dict(gamma=GAMMA, mu=1e-5, C_mu=0.09, beta_star=0.09)
    bc = [[0, 0], [1, 1]]
    ce = orc.Case(2, n, [np.full(8, h), np.full(10, h)], bc, turb_model=orc.TURB_KEPS, **base)
    co = orc.Case(2, n, [np.full(8, h), np.full(10, h)], bc, turb_model=orc.TURB_KOMEGA, **base)
    cm = orc.Case(2, n, [np.full(8, h), np.full(10, h)], bc, turb_model=orc.TURB_MUT, **base)
    W = ce.prim_to_cons(prim.ravel())
    te = ce.tau_turb(W, k, eps)
    to = co.tau_turb(W, k, eps / (0.09 * k))
    assert np.max(np.abs(te - to) / te) < 1e-14
    mut = rng.uniform(1e-4, 1e-3, n[0] * n[1])
    assert np.max(np.abs(cm.tau_turb(W, mut) - mut / 0.8)) < 1e-18
    # interior rows see the exact shear rate
    S = alpha
    expect = 1.2 * 0.09 * k ** 2 / eps / (0.8 * np.sqrt(1 + (S * k / eps) ** 2))
    te2 = te.reshape(n[1], n[0])[1:-1]
    assert np.max(np.abs(te2 - expect.reshape(n[1], n[0])[1:-1]) / te2) < 1e-13
    # rarefaction diagnostic: shear is divergence-free
    assert np.max(np.abs(ce.rarefaction(W, k, eps).reshape(n[1], n[0])[1:-1])) < 1e-15


def test_rarefaction_of_uniform_expansion(orc):
    n = 16
    h = 1.0 / n
    x = (np.arange(n) + 0.5) * h
    prim = np.zeros((3, n))
    prim[0], prim[1], prim[2] = 1.0, 0.3 * x, 0.5
    c = orc.Case(1, (n,), [np.full(n, h)], [[1, 1]], gamma=GAMMA, mu=2e-3)
    W = c.prim_to_cons(prim.ravel())
    eps = c.rarefaction(W)
    assert np.max(np.abs(eps[1:-1] - 2e-3 / 0.5 * 0.3)) < 1e-14
