"""Pins of the oracle's steady k-omega update on body-fitted grids (Wilcox's 2006 model in the steady
solver of the paper's Section 4, one diagonal-implicit step per cycle): the closed-form point-implicit
decay at rest, free-stream preservation, consistency with the time-accurate transport as the steps
shrink, and convergence of the iteration to the uniform steady state."""
import numpy as np

import oracle
from paper_1302_2132_gb300 import inputs

GAMMA = 1.4


def geometry(nodes):
    """Cell areas and the sum of each cell's four face lengths, from the node lattice."""
    x, y = nodes[..., 0], nodes[..., 1]
    q = [(x[:-1, :-1], y[:-1, :-1]), (x[:-1, 1:], y[:-1, 1:]), (x[1:, 1:], y[1:, 1:]), (x[1:, :-1], y[1:, :-1])]
    area = 0.5 * sum(q[a][0] * q[(a + 1) % 4][1] - q[(a + 1) % 4][0] * q[a][1] for a in range(4))
    per = sum(np.hypot(q[(a + 1) % 4][0] - q[a][0], q[(a + 1) % 4][1] - q[a][1]) for a in range(4))
    return area.ravel(), per.ravel()


def case(n0, n1, mu=1e-3, bc=((0, 0), (0, 0))):
    return oracle.Case(2, (n0, n1), [np.ones(n0), np.ones(n1)], [list(b) for b in bc], gamma=GAMMA, mu=mu,
                       turb_model=oracle.TURB_KOMEGA, multid=0, C_a=0.3, limiter=oracle.LIM_VANLEER)


def test_decay_at_rest_is_the_point_implicit_closed_form():
    """Fluid at rest with uniform k and omega, no diffusion: no flux and no production, so each cell
    takes RK / (1 + s beta* omega) and RW / (1 + s beta0 omega) with its own pseudo-time step s = cfl
    2 A / (c sum L), c the sound speed (computed here from the nodes)."""
    n0, n1 = 14, 10
    nodes = inputs.wavy_nodes(n0, n1, amp=0.05, shear=0.08)
    c = case(n0, n1)
    prim = np.zeros((4, n1, n0))
    prim[0], prim[3] = 1.3, 0.9
    W = c.prim_to_cons(prim.ravel())
    k0, w0, cfl = 0.02, 35.0, 3.0
    RK, RW = np.full(n0 * n1, 1.3 * k0), np.full(n0 * n1, 1.3 * w0)
    coeffs = oracle.komega_defaults(diffusion=0)
    RK1, RW1, st = c.steady_komega(nodes, W, RK, RW, cfl, cfl_flux=0.5, coeffs=coeffs, nthreads=4)
    assert st == 0
    area, per = geometry(nodes)
    s = cfl * 2.0 * area / (np.sqrt(GAMMA * 0.9 / 1.3) * per)
    assert np.allclose(RK1, RK / (1.0 + s * 0.09 * w0), rtol=1e-12, atol=0)
    assert np.allclose(RW1, RW / (1.0 + s * 0.0708 * w0), rtol=1e-12, atol=0)


def test_uniform_fields_in_a_uniform_stream_stay_unchanged():
    n0, n1 = 16, 12
    nodes = inputs.wavy_nodes(n0, n1, amp=0.04, shear=0.05)
    c = case(n0, n1)
    prim = np.zeros((4, n1, n0))
    prim[0], prim[1], prim[2], prim[3] = 1.1, 0.4, -0.3, 0.7
    W = c.prim_to_cons(prim.ravel())
    RK, RW = np.full(n0 * n1, 0.02 * 1.1), np.full(n0 * n1, 30.0 * 1.1)
    RK1, RW1, st = c.steady_komega(nodes, W, RK, RW, 4.0, coeffs=oracle.komega_defaults(sources=0), nthreads=4)
    assert st == 0
    assert np.abs(RK1 - RK).max() < 1e-13 * RK.max() and np.abs(RW1 - RW).max() < 1e-13 * RW.max()


def rates(c, nodes, W, RK, RW, cfl):
    """Per-cell rates of change of rho k, rho omega: the steady update over its pseudo-time steps and
    the time-accurate transport over a global step, both at pseudo-CFL cfl."""
    dtc, _ = c.steady_residual(nodes, W, cfl_flux=cfl, nthreads=4, f1=RK / W[:RK.size], f2=RW / W[:RK.size])
    RKs, RWs, st = c.steady_komega(nodes, W, RK, RW, cfl, cfl_flux=cfl, nthreads=4)
    assert st == 0
    dt = cfl * dtc.min()
    _, RKt, RWt, st = c.step_komega_curv(nodes, W, RK, RW, dt, nthreads=4)
    assert st == 0
    s = cfl * dtc
    return (RKs - RK) / s, (RWs - RW) / s, (RKt - RK) / dt, (RWt - RW) / dt


def test_consistent_with_the_time_accurate_transport_as_the_steps_shrink():
    """A sheared, compressed flow with smooth k and omega on a skewed periodic grid (convection,
    diffusion, production, cross diffusion, destruction all active): the steady update's rate of
    change, (RK' - RK) / s, and the time-accurate transport's, (RK(dt) - RK) / dt, approach each
    other at first order as the pseudo-CFL shrinks (both tend to the same right-hand side)."""
    n0, n1 = 24, 20
    nodes = inputs.wavy_nodes(n0, n1, amp=0.04, shear=0.06)
    pts = inputs.cell_points(nodes)
    c = case(n0, n1, mu=2e-3)
    prim = inputs.smooth_state_at(pts, seed=4, amp=0.2)
    W = c.prim_to_cons(prim.ravel())
    k, om = inputs.positive_fields_at(pts, seed=5)
    RK, RW = k.ravel() * W[:n0 * n1], om.ravel() * W[:n0 * n1]
    errs = []
    for cfl in (0.04, 0.02, 0.01):
        rks, rws, rkt, rwt = rates(c, nodes, W, RK, RW, cfl)
        assert np.abs(rkt).max() > 0 and np.abs(rwt).max() > 0
        errs.append(max(np.abs(rks - rkt).max() / np.abs(rkt).max(), np.abs(rws - rwt).max() / np.abs(rwt).max()))
    assert errs[-1] < 2e-2, errs
    for a, b in zip(errs[:-1], errs[1:]):
        assert 1.6 < a / b < 2.5, errs


def test_iteration_is_bounded_and_converges():
    """Frozen flow on a skewed periodic grid, no sources.  In a uniform stream at pseudo-CFL 50 the
    updates keep k within its initial range up to a tenth of it (the implicit diagonal carries the
    outflow, so the first-order part of the step is a convex combination of upwind values; the
    limited slopes add small excursions), where an explicit step at that CFL would blow up.  At rest
    with strong diffusion the iteration drives a perturbed field to the uniform steady state."""
    n0, n1 = 20, 16
    nodes = inputs.wavy_nodes(n0, n1, amp=0.04, shear=0.05)
    pts = inputs.cell_points(nodes)
    k, om = inputs.positive_fields_at(pts, seed=8)
    coeffs = oracle.komega_defaults(sources=0)
    for u, mu, cfl, iters in ((0.5, 1e-3, 50.0, 60), (0.0, 0.5, 50.0, 400)):
        c = case(n0, n1, mu=mu)
        prim = np.zeros((4, n1, n0))
        prim[0], prim[1], prim[2], prim[3] = 1.0, u, 0.4 * u, 0.7
        W = c.prim_to_cons(prim.ravel())
        RK, RW = k.ravel().copy(), om.ravel().copy()
        lo, hi = RK.min(), RK.max()
        dev0 = np.ptp(RK)
        for it in range(iters):
            RK, RW, st = c.steady_komega(nodes, W, RK, RW, cfl, coeffs=coeffs, nthreads=4)
            assert st == 0
            assert RK.min() >= lo - 0.1 * dev0 and RK.max() <= hi + 0.1 * dev0
        if u == 0.0:
            assert np.ptp(RK) < 1e-2 * dev0


def test_cycles_with_transport_run_on_a_corner_grid():
    """The composed steady cycle (k-omega update, then the flow cycle with the fields of the cycle's
    start) on the compression corner: the flow residual falls and the fields stay positive."""
    sp = inputs.compression_corner(64, 32, alpha_deg=24.0)
    c = oracle.Case(2, sp["n"], [np.ones(64), np.ones(32)], sp["bc"], gamma=GAMMA, mu=sp["mu"], T_wall=sp["T_wall"],
                    turb_model=oracle.TURB_KOMEGA, multid=0, C_a=0.5, limiter=oracle.LIM_VANLEER,
                    bc_prim=sp["bc_prim"])
    W = c.prim_to_cons(np.asarray(sp["prim"], dtype=np.float64).ravel())
    RK, RW = np.ravel(sp["f1"]) * W[:64 * 32], np.ravel(sp["f2"]) * W[:64 * 32]
    hist = []
    for it in range(40):
        W, RK, RW, res, st = c.steady_cycle_komega(sp["nodes"], W, RK, RW, 1.0 if it < 10 else 3.0, levels=3,
                                                   tiles=(16, 16), nthreads=8)
        assert st == 0
        hist.append(res)
    assert hist[-1] < 0.2 * max(hist)
    assert RK.min() >= 0.0 and RW.min() > 0.0
