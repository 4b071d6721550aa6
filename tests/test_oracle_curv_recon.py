"""Pins of the oracle's higher-order reconstructions (MUSCL-3, WENO-5; Section 4) on body-fitted
grids: index-space reconstruction of the rotated states along each grid line, normal slopes the
one-sided differences to the face values over the centroid-to-face distances.  Equal to the
rectilinear reconstruction steps where the grid is rectilinear, free-stream preserving on a skewed
grid, and invariant under a rotation of grid and flow."""
import math

import numpy as np
import pytest

import oracle
from paper_1302_2132_gb300 import inputs

GAMMA = 1.4
RECONS = [oracle.RECON_MUSCL3, oracle.RECON_WENO5]


def rel(a, b):
    return np.abs(a - b).max() / np.abs(b).max()


@pytest.mark.parametrize("multid", [0, 1])
@pytest.mark.parametrize("recon", RECONS)
def test_uniform_grid_equals_the_rectilinear_step(recon, multid):
    n = 20
    spec = inputs.turbulence(n, 2, seed=4)
    h = spec["dx"][0][0]
    c = oracle.Case(2, (n, n), spec["dx"], [(0, 0), (0, 0)], gamma=GAMMA, mu=1e-5, turb_model=oracle.TURB_KEPS,
                    multid=multid, C_a=0.3, recon=recon)
    nodes = inputs.uniform_nodes(n, n, n * h, n * h)
    W = c.prim_to_cons(spec["prim"].ravel())
    f1, f2 = spec["f1"].ravel(), spec["f2"].ravel()
    dt = c.compute_dt(W, 0.5)
    Wr, st, _ = c.step(W, dt, f1=f1, f2=f2, nthreads=4)
    Wc, stc = c.step_curv(nodes, W, dt, f1=f1, f2=f2, nthreads=4)
    assert st == 0 and stc == 0
    assert rel(Wc - W, Wr - W) < 1e-12
    # and the reconstruction matters: the MUSCL-2 step differs
    c2 = oracle.Case(2, (n, n), spec["dx"], [(0, 0), (0, 0)], gamma=GAMMA, mu=1e-5, turb_model=oracle.TURB_KEPS,
                     multid=multid, C_a=0.3)
    W2, _ = c2.step_curv(nodes, W, dt, f1=f1, f2=f2, nthreads=4)
    assert rel(W2 - W, Wr - W) > 1e-6


@pytest.mark.parametrize("recon", RECONS)
def test_stretched_rectilinear_grid_with_walls_equals_the_rectilinear_step(recon):
    """The wall-clustered shock / boundary-layer grid (wall, Dirichlet, outflow): the centroid-to-face
    distances are the half widths, so the curvilinear step equals the rectilinear one; three ghost
    layers enter the WENO-5 stencil."""
    spec = inputs.shock_boundary_layer(24, 30)
    n0, n1 = spec["n"]
    c = oracle.Case(2, spec["n"], spec["dx"], spec["bc"], gamma=GAMMA, mu=spec["mu"], T_wall=spec["T_wall"],
                    multid=1, C_a=0.5, bc_prim=spec["bc_prim"], recon=recon)
    nodes = inputs.rectilinear_nodes(spec["dx"][0], spec["dx"][1])
    W = c.prim_to_cons(spec["prim"].ravel())
    for _ in range(3):
        dt = c.compute_dt(W, 0.4)
        Wr, st, _ = c.step(W, dt, nthreads=4)
        Wc, stc = c.step_curv(nodes, W, dt, nthreads=4)
        assert st == 0 and stc == 0
        nc = n0 * n1
        for v in range(4):
            d_r, d_c = Wr[v * nc:(v + 1) * nc] - W[v * nc:(v + 1) * nc], Wc[v * nc:(v + 1) * nc] - W[v * nc:(v + 1) * nc]
            assert np.abs(d_c - d_r).max() <= 1e-10 * np.abs(d_r).max() + 1e-15
        W = Wc


@pytest.mark.parametrize("recon", RECONS)
def test_free_stream_is_preserved_on_a_skewed_grid(recon):
    n0, n1 = 18, 14
    nodes = inputs.wavy_nodes(n0, n1, amp=0.04, shear=0.06)
    c = oracle.Case(2, (n0, n1), [np.ones(n0), np.ones(n1)], [(1, 1), (1, 1)], gamma=GAMMA, mu=1e-5,
                    turb_model=oracle.TURB_KEPS, multid=1, recon=recon)
    prim = np.zeros((4, n1, n0))
    prim[0], prim[1], prim[2], prim[3] = 1.2, 0.45, -0.3, 1.0 / GAMMA
    W0 = c.prim_to_cons(prim.ravel())
    f1, f2 = np.full(n0 * n1, 0.02), np.full(n0 * n1, 0.5)
    W = W0
    for _ in range(5):
        dt = c.compute_dt_curv(nodes, W, 0.6)
        W, st = c.step_curv(nodes, W, dt, f1=f1, f2=f2, nthreads=4)
        assert st == 0
    assert np.abs(W - W0).max() < 1e-13


@pytest.mark.parametrize("recon", RECONS)
def test_rotating_grid_and_flow_rotates_the_result(recon):
    n0, n1 = 16, 12
    theta = 0.61
    nodes = inputs.wavy_nodes(n0, n1)
    pts = inputs.cell_points(nodes)
    prim = inputs.smooth_state_at(pts, seed=3)
    f1, f2 = inputs.positive_fields_at(pts, seed=5)
    f1, f2 = f1.ravel(), f2.ravel()
    c = oracle.Case(2, (n0, n1), [np.ones(n0), np.ones(n1)], [(0, 0), (0, 0)], gamma=GAMMA, mu=1e-5,
                    turb_model=oracle.TURB_KOMEGA, C_a=0.2, multid=1, recon=recon)
    W = c.prim_to_cons(prim.ravel())
    Wt = c.prim_to_cons(inputs.rotate_prim(prim, theta).ravel())
    nodes_t = inputs.rotate_nodes(nodes, theta)
    dt = c.compute_dt_curv(nodes, W, 0.5)
    A, st = c.step_curv(nodes, W, dt, f1=f1, f2=f2, nthreads=4)
    B, st2 = c.step_curv(nodes_t, Wt, dt, f1=f1, f2=f2, nthreads=4)
    assert st == 0 and st2 == 0
    nc = n0 * n1
    A, B, W = A.reshape(4, nc), B.reshape(4, nc), W.reshape(4, nc)
    ca, sa = math.cos(theta), math.sin(theta)
    Brot = np.stack([B[0], ca * B[1] + sa * B[2], -sa * B[1] + ca * B[2], B[3]])
    for v in range(4):
        assert np.abs(Brot[v] - A[v]).max() < 1e-12 * np.abs(A[v] - W[v]).max() + 1e-14
