"""Pins of the oracle's k-omega transport on body-fitted grids (Wilcox's 2006 model, the reading of the
paper's Section 4, in each face's frame): equal to the rectilinear transport on a uniform grid,
conservative and free-stream preserving on a skewed grid, and the exact homogeneous decay."""
import numpy as np

import oracle
from paper_1302_2132_gb300 import inputs

GAMMA = 1.4


def fields(n, seed):
    rng = np.random.default_rng(seed)
    return 0.01 * (1.0 + 0.5 * rng.random(n)), 20.0 * (1.0 + 0.5 * rng.random(n))


def test_uniform_grid_equals_the_rectilinear_transport():
    """On a uniform periodic grid the Green-Gauss gradients are the central differences, the
    centroid steps the widths and the half-time face values the rectilinear ones: flow, rho k and
    rho omega after a step equal those of orc_step_komega to rounding."""
    n = 20
    spec = inputs.turbulence(n, 2, seed=6)
    h = spec["dx"][0][0]
    c = oracle.Case(2, (n, n), spec["dx"], [(0, 0), (0, 0)], gamma=GAMMA, mu=1e-4, turb_model=oracle.TURB_KOMEGA,
                    multid=0, C_a=0.2)
    nodes = inputs.uniform_nodes(n, n, n * h, n * h)
    W = c.prim_to_cons(spec["prim"].ravel())
    k, om = fields(n * n, 3)
    RK, RW = k * W[:n * n], om * W[:n * n]
    dt = c.compute_dt(W, 0.5)
    Wr, RKr, RWr, st = c.step_komega(W, RK, RW, dt, nthreads=4)
    Wc, RKc, RWc, stc = c.step_komega_curv(nodes, W, RK, RW, dt, nthreads=4)
    assert st == 0 and stc == 0
    assert np.abs(Wc - Wr).max() < 1e-12 * np.abs(Wr - W).max()
    assert np.abs(RKc - RKr).max() < 1e-12 * np.abs(RKr - RK).max()
    assert np.abs(RWc - RWr).max() < 1e-12 * np.abs(RWr - RW).max()


def test_transport_conserves_and_preserves_a_uniform_field_on_a_skewed_grid():
    """Without sources the transport only moves rho k and rho omega between cells: their area sums
    are unchanged on a periodic skewed grid; a uniform flow with uniform k and omega stays uniform."""
    n0, n1 = 18, 14
    nodes = inputs.wavy_nodes(n0, n1, amp=0.04, shear=0.05)
    x, y = nodes[..., 0], nodes[..., 1]
    quad = [(x[:-1, :-1], y[:-1, :-1]), (x[:-1, 1:], y[:-1, 1:]), (x[1:, 1:], y[1:, 1:]), (x[1:, :-1], y[1:, :-1])]
    area = (0.5 * sum(quad[q][0] * quad[(q + 1) % 4][1] - quad[(q + 1) % 4][0] * quad[q][1] for q in range(4))).ravel()
    c = oracle.Case(2, (n0, n1), [np.ones(n0), np.ones(n1)], [(0, 0), (0, 0)], gamma=GAMMA, mu=1e-3,
                    turb_model=oracle.TURB_KOMEGA, multid=0)
    coeffs = oracle.komega_defaults(sources=0)
    prim = inputs.smooth_state_at(inputs.cell_points(nodes), seed=2, amp=0.15)
    W = c.prim_to_cons(prim.ravel())
    k, om = fields(n0 * n1, 5)
    RK, RW = k * W[:n0 * n1], om * W[:n0 * n1]
    dt = c.compute_dt_curv(nodes, W, 0.5)
    W1, RK1, RW1, st = c.step_komega_curv(nodes, W, RK, RW, dt, coeffs=coeffs, nthreads=4)
    assert st == 0
    assert abs((RK1 * area).sum() / (RK * area).sum() - 1.0) < 1e-13
    assert abs((RW1 * area).sum() / (RW * area).sum() - 1.0) < 1e-13
    assert np.abs(RK1 - RK).max() > 1e-6 * RK.max()
    prim = np.zeros((4, n1, n0))
    prim[0], prim[1], prim[2], prim[3] = 1.1, 0.4, -0.3, 0.7
    W = c.prim_to_cons(prim.ravel())
    RK = np.full(n0 * n1, 0.02 * 1.1)
    RW = np.full(n0 * n1, 30.0 * 1.1)
    W1, RK1, RW1, st = c.step_komega_curv(nodes, W, RK, RW, 1e-3, coeffs=coeffs, nthreads=4)
    assert st == 0
    assert np.abs(RK1 - RK).max() < 1e-13 * RK.max() and np.abs(RW1 - RW).max() < 1e-13 * RW.max()


def test_homogeneous_decay_on_a_skewed_grid():
    """Fluid at rest with uniform k and omega: omega follows 1/omega = 1/omega0 + beta0 t exactly (the
    point-implicit destruction), whatever the grid."""
    n0, n1 = 12, 10
    nodes = inputs.wavy_nodes(n0, n1)
    c = oracle.Case(2, (n0, n1), [np.ones(n0), np.ones(n1)], [(0, 0), (0, 0)], gamma=GAMMA, mu=1e-4,
                    turb_model=oracle.TURB_KOMEGA, multid=0)
    prim = np.zeros((4, n1, n0))
    prim[0], prim[3] = 1.0, 1.0 / GAMMA
    W = c.prim_to_cons(prim.ravel())
    k0, w0, dt, steps = 0.02, 40.0, 1e-4, 50
    RK, RW = np.full(n0 * n1, k0), np.full(n0 * n1, w0)
    for _ in range(steps):
        W, RK, RW, st = c.step_komega_curv(nodes, W, RK, RW, dt, nthreads=4)
        assert st == 0
    assert np.allclose(RW, 1.0 / (1.0 / w0 + 0.0708 * dt * steps), rtol=1e-12, atol=0)
    kk, w = k0, w0
    for _ in range(steps):
        kk = kk / (1.0 + dt * 0.09 * w)
        w = w / (1.0 + dt * 0.0708 * w)
    assert np.allclose(RK, kk, rtol=1e-12, atol=0)
