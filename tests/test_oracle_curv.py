"""Pins of the oracle's curvilinear (body-fitted) 2D step, the directional expansion in each face's
(normal, tangent) frame on the grids of the paper's channel and aerofoil cases (Section 5, Table 2):
equivalence with the rectilinear oracle where the grid is rectilinear, free-stream preservation,
invariance under a rotation of grid and flow, conservation, second-order convergence of a smooth
wave on a skewed grid, and rejection of folded cells."""
import math

import numpy as np
import pytest

import oracle
from paper_1302_2132_gb300 import inputs

GAMMA = 1.4


def case_for(n0, n1, bc, turb=oracle.TURB_NONE, mu=1e-5, dx=None, multid=0, **kw):
    dx = dx if dx is not None else [np.full(n0, 1.0 / n0), np.full(n1, 1.0 / n1)]
    return oracle.Case(2, (n0, n1), dx, bc, gamma=GAMMA, mu=mu, turb_model=turb, multid=multid, **kw)


def rel(a, b):
    return np.abs(a - b).max() / np.abs(b).max()


@pytest.mark.parametrize("multid", [0, 1])
@pytest.mark.parametrize("turb", [oracle.TURB_NONE, oracle.TURB_KEPS, oracle.TURB_KOMEGA])
def test_uniform_grid_equals_the_rectilinear_step(turb, multid):
    """On a uniform grid the face frames are the axes (a j-face's tangent is -x, the mirror image
    of the rectilinear frame), centroid distances the widths and the Green-Gauss velocity gradient
    the central difference, so a step equals the rectilinear step to rounding, with the directional
    and with the multi-dimensional expansion (periodic turbulence with gradient-based tau_t)."""
    n = 20
    spec = inputs.turbulence(n, 2, seed=4)
    h = spec["dx"][0][0]
    c = case_for(n, n, [(0, 0), (0, 0)], turb=turb, dx=spec["dx"], C_a=0.3, multid=multid)
    nodes = inputs.uniform_nodes(n, n, n * h, n * h)
    W = c.prim_to_cons(spec["prim"].ravel())
    f1, f2 = spec["f1"].ravel(), spec["f2"].ravel()
    if turb == oracle.TURB_KOMEGA:
        f2 = f2 * 50.0
    dt = c.compute_dt(W, 0.5)
    assert abs(c.compute_dt_curv(nodes, W, 0.5) / dt - 1.0) < 1e-14
    Wr, st, _ = c.step(W, dt, f1=f1, f2=f2, nthreads=4)
    Wc, stc = c.step_curv(nodes, W, dt, f1=f1, f2=f2, nthreads=4)
    assert st == 0 and stc == 0
    assert rel(Wc - W, Wr - W) < 1e-12
    assert rel(Wc, Wr) < 1e-14


@pytest.mark.parametrize("multid", [0, 1])
def test_stretched_rectilinear_grid_with_walls_equals_the_rectilinear_step(multid):
    """The Mach 2.85 shock / boundary-layer case on its wall-clustered grid (no-slip wall, Dirichlet
    inflow and top, outflow): ghost centroids mirrored through the boundary faces reproduce the
    ghost widths (corner ghosts too, which the multi-dimensional expansion reaches), so the
    curvilinear step equals the rectilinear one (no turbulence model)."""
    spec = inputs.shock_boundary_layer(24, 30)
    n0, n1 = spec["n"]
    c = oracle.Case(2, spec["n"], spec["dx"], spec["bc"], gamma=GAMMA, mu=spec["mu"], T_wall=spec["T_wall"],
                    multid=multid, C_a=0.5, bc_prim=spec["bc_prim"])
    nodes = inputs.rectilinear_nodes(spec["dx"][0], spec["dx"][1])
    W = c.prim_to_cons(spec["prim"].ravel())
    for _ in range(3):
        dt = c.compute_dt(W, 0.4)
        assert abs(c.compute_dt_curv(nodes, W, 0.4) / dt - 1.0) < 1e-13
        Wr, st, _ = c.step(W, dt, nthreads=4)
        Wc, stc = c.step_curv(nodes, W, dt, nthreads=4)
        assert st == 0 and stc == 0
        nc = n0 * n1
        for v in range(4):
            d_r, d_c = Wr[v * nc:(v + 1) * nc] - W[v * nc:(v + 1) * nc], Wc[v * nc:(v + 1) * nc] - W[v * nc:(v + 1) * nc]
            assert np.abs(d_c - d_r).max() <= 1e-10 * np.abs(d_r).max() + 1e-15
        W = Wc


@pytest.mark.parametrize("multid", [0, 1])
@pytest.mark.parametrize("bc", [(0, 0), (1, 1)])
def test_free_stream_is_preserved_on_a_skewed_grid(bc, multid):
    """Uniform flow through a smoothly skewed grid stays uniform: every cell's face normals times
    lengths sum to zero, and a uniform state has zero slopes, so only rounding remains (periodic and
    transmissive boundaries; k-epsilon tau_t is active but the strain rate is zero)."""
    n0, n1 = 18, 14
    nodes = inputs.wavy_nodes(n0, n1, amp=0.04, shear=0.06)
    c = case_for(n0, n1, [bc, bc], turb=oracle.TURB_KEPS, multid=multid)
    prim = np.zeros((4, n1, n0))
    prim[0], prim[1], prim[2], prim[3] = 1.2, 0.45, -0.3, 1.0 / GAMMA
    W0 = c.prim_to_cons(prim.ravel())
    f1 = np.full(n0 * n1, 0.02)
    f2 = np.full(n0 * n1, 0.5)
    W = W0
    for _ in range(5):
        dt = c.compute_dt_curv(nodes, W, 0.6)
        W, st = c.step_curv(nodes, W, dt, f1=f1, f2=f2, nthreads=4)
        assert st == 0
    assert np.abs(W - W0).max() < 1e-13


@pytest.mark.parametrize("multid", [0, 1])
def test_rotating_grid_and_flow_rotates_the_result(multid):
    """Turning the grid nodes and the velocity by the same angle turns the momentum of the result
    and leaves density and energy unchanged (periodic box, k-omega tau_t from Green-Gauss
    gradients, whose strain-rate magnitude is frame invariant)."""
    n0, n1 = 16, 12
    theta = 0.61
    nodes = inputs.wavy_nodes(n0, n1)
    pts = inputs.cell_points(nodes)
    prim = inputs.smooth_state_at(pts, seed=3)
    f1, f2 = inputs.positive_fields_at(pts, seed=5)
    f1, f2 = f1.ravel(), f2.ravel()
    c = case_for(n0, n1, [(0, 0), (0, 0)], turb=oracle.TURB_KOMEGA, C_a=0.2, multid=multid)
    W = c.prim_to_cons(prim.ravel())
    Wt = c.prim_to_cons(inputs.rotate_prim(prim, theta).ravel())
    nodes_t = inputs.rotate_nodes(nodes, theta)
    dt = c.compute_dt_curv(nodes, W, 0.5)
    assert abs(c.compute_dt_curv(nodes_t, Wt, 0.5) / dt - 1.0) < 1e-13
    A, st = c.step_curv(nodes, W, dt, f1=f1, f2=f2, nthreads=4)
    B, st2 = c.step_curv(nodes_t, Wt, dt, f1=f1, f2=f2, nthreads=4)
    assert st == 0 and st2 == 0
    nc = n0 * n1
    A, B, W = A.reshape(4, nc), B.reshape(4, nc), W.reshape(4, nc)
    ca, sa = math.cos(theta), math.sin(theta)
    Brot = np.stack([B[0], ca * B[1] + sa * B[2], -sa * B[1] + ca * B[2], B[3]])
    for v in range(4):
        assert np.abs(Brot[v] - A[v]).max() < 1e-12 * np.abs(A[v] - W[v]).max() + 1e-14


def test_periodic_skewed_grid_conserves_mass_momentum_and_energy():
    """Sum over cells of area times the conservative state is unchanged by a step on a periodic grid:
    each face flux, weighted by the face length, leaves one cell and enters the other."""
    n0, n1 = 20, 16
    nodes = inputs.wavy_nodes(n0, n1, amp=0.05, shear=0.04)
    pts = inputs.cell_points(nodes)
    prim = inputs.smooth_state_at(pts, seed=11, amp=0.2)
    f1, f2 = inputs.positive_fields_at(pts, seed=12, om_ref=5.0)
    c = case_for(n0, n1, [(0, 0), (0, 0)], turb=oracle.TURB_KEPS)
    # cell areas from the shoelace formula over the four nodes
    x, y = nodes[..., 0], nodes[..., 1]
    quad = [(x[:-1, :-1], y[:-1, :-1]), (x[:-1, 1:], y[:-1, 1:]), (x[1:, 1:], y[1:, 1:]), (x[1:, :-1], y[1:, :-1])]
    area = 0.5 * sum(quad[k][0] * quad[(k + 1) % 4][1] - quad[(k + 1) % 4][0] * quad[k][1] for k in range(4))
    area = area.ravel()
    W = c.prim_to_cons(prim.ravel())
    tot0 = (W.reshape(4, -1) * area).sum(axis=1)
    for _ in range(4):
        dt = c.compute_dt_curv(nodes, W, 0.5)
        W, st = c.step_curv(nodes, W, dt, f1=f1.ravel(), f2=f2.ravel(), nthreads=4)
        assert st == 0
    tot = (W.reshape(4, -1) * area).sum(axis=1)
    scale = np.abs(W.reshape(4, -1) * area).sum(axis=1)
    assert np.all(np.abs(tot - tot0) < 1e-14 * scale)


def test_smooth_wave_on_a_skewed_grid_converges_at_second_order():
    """rho = 1 + 0.2 sin(2 pi (x + y)), (u, v) = (1, 0.5), p = 1 on a skewed periodic grid: the
    density error at t = 0.2 against the translated profile (both at the cell sample points, which
    is second-order accurate) falls by more than 3 when the cells are halved.  A small CFL number
    keeps the directional expansion's O(dt) cross-derivative error (the tangential slopes it leaves
    out) below the spatial error; at CFL 0.5 the rectilinear step on a uniform grid converges at
    about 1.4 on the same wave."""
    errs = []
    for n in (16, 32):
        nodes = inputs.wavy_nodes(n, n, amp=0.03, shear=0.05)
        pts = inputs.cell_points(nodes)
        X, Y = pts[..., 0], pts[..., 1]
        prim = np.zeros((4, n, n))
        prim[0] = 1.0 + 0.2 * np.sin(2 * math.pi * (X + Y))
        prim[1], prim[2], prim[3] = 1.0, 0.5, 1.0
        c = case_for(n, n, [(0, 0), (0, 0)], mu=1e-7)
        W = c.prim_to_cons(prim.ravel())
        t, T = 0.0, 0.2
        while t < T - 1e-14:
            dt = min(c.compute_dt_curv(nodes, W, 0.1), T - t)
            W, st = c.step_curv(nodes, W, dt, nthreads=8)
            assert st == 0
            t += dt
        exact = 1.0 + 0.2 * np.sin(2 * math.pi * ((X - T) + (Y - 0.5 * T)))
        errs.append(np.abs(W[: n * n] - exact.ravel()).mean())
    rate = math.log2(errs[0] / errs[1])
    assert rate > 1.65, (errs, rate)


def test_folded_cells_are_rejected():
    n0, n1 = 6, 5
    nodes = inputs.uniform_nodes(n0, n1)
    nodes[2, 3] = nodes[2, 4] + np.array([0.1, 0.0])  # node crosses its right neighbour
    c = case_for(n0, n1, [(0, 0), (0, 0)])
    prim = np.ones((4, n1, n0))
    W = c.prim_to_cons(prim.ravel())
    _, st = c.step_curv(nodes, W, 1e-3)
    assert st == 2


def test_multidimensional_expansion_changes_the_skewed_grid_step():
    """The tangential slopes are in effect: on a skewed grid with a smooth flow the multi-dimensional
    step differs from the directional one by far more than rounding, and both conserve."""
    n0, n1 = 16, 12
    nodes = inputs.wavy_nodes(n0, n1)
    prim = inputs.smooth_state_at(inputs.cell_points(nodes), seed=8, amp=0.2)
    out = []
    for md in (0, 1):
        c = case_for(n0, n1, [(0, 0), (0, 0)], multid=md, mu=1e-3)
        W = c.prim_to_cons(prim.ravel())
        dt = c.compute_dt_curv(nodes, W, 0.5)
        Wn, st = c.step_curv(nodes, W, dt)
        assert st == 0
        out.append(Wn - W)
    assert np.abs(out[1] - out[0]).max() > 1e-4 * np.abs(out[0]).max()
