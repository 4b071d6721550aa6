"""Pins of the oracle's steady-state solver on body-fitted grids (Section 4: local time stepping,
LU-SGS smoothing in Yoon and Jameson's form, multigrid): the local explicit steps from independent
geometry, the residual against the time-accurate step where every window is equal, free stream,
the LU-SGS increment against a dense solve of its factored system, and convergence of the multigrid
cycle to one steady state whatever the number of levels."""
import math

import numpy as np
import pytest

import oracle
from paper_1302_2132_gb300 import inputs

GAMMA = 1.4


def geometry(nodes):
    """Areas, face normals, lengths and centroid of a node lattice, computed here from the nodes."""
    x, y = nodes[..., 0], nodes[..., 1]
    quad = [(x[:-1, :-1], y[:-1, :-1]), (x[:-1, 1:], y[:-1, 1:]), (x[1:, 1:], y[1:, 1:]), (x[1:, :-1], y[1:, :-1])]
    area = 0.5 * sum(quad[k][0] * quad[(k + 1) % 4][1] - quad[(k + 1) % 4][0] * quad[k][1] for k in range(4))
    # i-faces: from node (i, j) to (i, j + 1); normal (ey, -ex)/L
    ex, ey = x[1:, :] - x[:-1, :], y[1:, :] - y[:-1, :]
    Li = np.hypot(ex, ey)
    ni = np.stack([ey / Li, -ex / Li], -1)
    ex, ey = x[:, 1:] - x[:, :-1], y[:, 1:] - y[:, :-1]
    Lj = np.hypot(ex, ey)
    nj = np.stack([-ey / Lj, ex / Lj], -1)
    cx = 0.25 * (x[:-1, :-1] + x[:-1, 1:] + x[1:, :-1] + x[1:, 1:])
    cy = 0.25 * (y[:-1, :-1] + y[:-1, 1:] + y[1:, :-1] + y[1:, 1:])
    return area, ni, Li, nj, Lj, cx, cy


def periodic_case(n0, n1, turb=oracle.TURB_NONE, mu=1e-3, C_a=0.0):
    return oracle.Case(2, (n0, n1), [np.full(n0, 1.0 / n0), np.full(n1, 1.0 / n1)], [(0, 0), (0, 0)], gamma=GAMMA,
                       mu=mu, turb_model=turb, multid=0, C_a=C_a)


def test_local_steps_from_independent_geometry():
    n0, n1 = 14, 10
    nodes = inputs.wavy_nodes(n0, n1)
    prim = inputs.smooth_state_at(inputs.cell_points(nodes), seed=2)
    c = periodic_case(n0, n1)
    W = c.prim_to_cons(prim.ravel())
    dtc, _ = c.steady_residual(nodes, W)
    area, ni, Li, nj, Lj, _, _ = geometry(nodes)
    rho, u, v, p = prim
    cs = np.sqrt(GAMMA * p / rho)
    rate = np.zeros((n1, n0))
    for s in (0, 1):
        rate += (np.abs(u * ni[:, s:n0 + s, 0] + v * ni[:, s:n0 + s, 1]) + cs) * Li[:, s:n0 + s]
        rate += (np.abs(u * nj[s:n1 + s, :, 0] + v * nj[s:n1 + s, :, 1]) + cs) * Lj[s:n1 + s, :]
    assert np.allclose(dtc, (2 * area / rate).ravel(), rtol=1e-13, atol=0)


def test_residual_is_the_time_accurate_increment_where_all_windows_are_equal():
    """With the same |u|, |v|, rho and p in every cell (velocity signs in a checkerboard of blocks) on
    a uniform grid every local step is the same, so every face window is cfl_flux times it and
    R = -A (W_step - W) / window with W_step the time-accurate step of that length."""
    n = 12
    nodes = inputs.uniform_nodes(n, n)
    X, Y = np.meshgrid((np.arange(n) + 0.5) / n, (np.arange(n) + 0.5) / n, indexing="xy")
    prim = np.zeros((4, n, n))
    prim[0] = 1.0
    prim[1] = 0.4 * np.sign(np.sin(2 * math.pi * X + 0.1))
    prim[2] = -0.25 * np.sign(np.cos(4 * math.pi * Y + 0.1))
    prim[3] = 1.0
    c = periodic_case(n, n, C_a=0.3)
    W = c.prim_to_cons(prim.ravel())
    dtc, R = c.steady_residual(nodes, W, cfl_flux=0.37)
    assert np.ptp(dtc) < 1e-14 * dtc.max()  # equal up to rounding
    window = 0.37 * dtc[0]
    Ws, st = c.step_curv(nodes, W, window)
    assert st == 0
    A = 1.0 / n ** 2
    assert np.abs(R - (-A * (Ws - W) / window)).max() < 1e-11 * np.abs(R).max()


def test_free_stream_has_zero_residual_on_a_skewed_grid():
    n0, n1 = 16, 12
    nodes = inputs.wavy_nodes(n0, n1, amp=0.05, shear=0.06)
    prim = np.zeros((4, n1, n0))
    prim[0], prim[1], prim[2], prim[3] = 1.3, 0.5, -0.2, 0.8
    c = periodic_case(n0, n1)
    W = c.prim_to_cons(prim.ravel())
    for fo in (False, True):
        _, R = c.steady_residual(nodes, W, first_order=fo)
        assert np.abs(R).max() < 1e-13
    # on a smooth state the first-order residual (no slopes) differs from the second-order one
    W = c.prim_to_cons(inputs.smooth_state_at(inputs.cell_points(nodes), seed=6).ravel())
    _, R2 = c.steady_residual(nodes, W)
    _, R1 = c.steady_residual(nodes, W, first_order=True)
    assert np.abs(R1 - R2).max() > 1e-3 * np.abs(R2).max()


def euler_flux(w, nx, ny):
    rho, mx, my, E = w
    p = (GAMMA - 1) * (E - 0.5 * (mx * mx + my * my) / rho)
    un = (mx * nx + my * ny) / rho
    return np.array([rho * un, mx * un + p * nx, my * un + p * ny, (E + p) * un])


def jac(w, nx, ny, h=1e-7):
    J = np.zeros((4, 4))
    for k in range(4):
        e = np.zeros(4)
        e[k] = h * max(1.0, abs(w[k]))
        J[:, k] = (euler_flux(w + e, nx, ny) - euler_flux(w - e, nx, ny)) / (2 * e[k])
    return J


@pytest.mark.parametrize("tiles", [(6, 5), (3, 2)])
def test_lusgs_increment_solves_its_factored_system(tiles):
    """For a tiny residual the LU-SGS increment is the solution of (D + L) D^-1 (D + U) dW = -R with
    L, U built here from Euler flux Jacobians (finite differences), lambda = max |U.n| + c + 2 mu /
    (rho d) over the two cells and D = A / dt + 1/2 sum lambda L; couplings only within a tile,
    lower = (i - 1, j), (i, j - 1)."""
    n0, n1 = 6, 5
    mu = 2e-3
    nodes = inputs.wavy_nodes(n0, n1, amp=0.05, shear=0.05)
    prim = inputs.smooth_state_at(inputs.cell_points(nodes), seed=4)
    c = periodic_case(n0, n1, mu=mu)
    W = c.prim_to_cons(prim.ravel())
    nc = n0 * n1
    rng = np.random.default_rng(1)
    R = 1e-8 * rng.normal(size=4 * nc)
    dt = 0.05 * (1.0 + rng.random(nc))
    dW = c.lusgs(nodes, W, dt, R, tiles=tiles)
    area, ni, Li, nj, Lj, cx, cy = geometry(nodes)
    Wc = W.reshape(4, nc).T  # [cell][v]
    cell = lambda i, j: (j % n1) * n0 + (i % n0)

    def lam(wa, wb, nx, ny, d):
        def sr(w):
            p = (GAMMA - 1) * (w[3] - 0.5 * (w[1] ** 2 + w[2] ** 2) / w[0])
            return abs((w[1] * nx + w[2] * ny) / w[0]) + math.sqrt(GAMMA * p / w[0])
        return max(sr(wa), sr(wb)) + 2 * mu / (0.5 * (wa[0] + wb[0]) * d)

    def cdist(i0, j0, i1, j1):
        # centroids of a periodic lattice: translate by the period where an index wraps
        def c_of(i, j):
            x = cx[j % n1, i % n0] + (i // n0) * (nodes[0, -1, 0] - nodes[0, 0, 0])
            y = cy[j % n1, i % n0] + (j // n1) * (nodes[-1, 0, 1] - nodes[0, 0, 1])
            return x, y
        a, b = c_of(i0, j0), c_of(i1, j1)
        return math.hypot(b[0] - a[0], b[1] - a[1])

    N = 4 * nc
    D = np.zeros((N, N))
    Lm = np.zeros((N, N))
    Um = np.zeros((N, N))
    for j in range(n1):
        for i in range(n0):
            ci = cell(i, j)
            faces = [  # (neighbour i, j, outward normal, length, which side)
                (i - 1, j, -ni[j, i], Li[j, i]), (i + 1, j, ni[j, i + 1], Li[j, i + 1]),
                (i, j - 1, -nj[j, i], Lj[j, i]), (i, j + 1, nj[j + 1, i], Lj[j + 1, i])]
            diag = area[j, i] / dt[ci]
            for (ii, jj, nrm, L) in faces:
                cn = cell(ii, jj)
                hl = 0.5 * L * lam(Wc[ci], Wc[cn], nrm[0], nrm[1], cdist(i, j, ii, jj))
                diag += hl
                same_tile = (ii // tiles[0] == i // tiles[0] and jj // tiles[1] == j // tiles[1]
                             and 0 <= ii < n0 and 0 <= jj < n1)
                if not same_tile:
                    continue
                block = 0.5 * L * jac(Wc[cn], nrm[0], nrm[1]) - hl * np.eye(4)
                rows = slice(4 * ci, 4 * ci + 4)
                cols = slice(4 * cn, 4 * cn + 4)
                if (ii, jj) in ((i - 1, j), (i, j - 1)):
                    Lm[rows, cols] = block
                else:
                    Um[rows, cols] = block
            D[4 * ci:4 * ci + 4, 4 * ci:4 * ci + 4] = diag * np.eye(4)
    Rc = R.reshape(4, nc).T.ravel()
    M = (D + Lm) @ np.linalg.inv(D) @ (D + Um)
    x = np.linalg.solve(M, -Rc)
    got = dW.reshape(4, nc).T.ravel()
    assert np.abs(got - x).max() < 1e-6 * np.abs(x).max()


def corner_case(nx, ny, mu=5e-3):
    spec = inputs.compression_corner(nx, ny, alpha_deg=10.0, dy1=0.01, ratio=1.0)
    prim = np.zeros((4, ny, nx))
    prim[0], prim[1], prim[3] = 1.0, 2.85, 1 / GAMMA
    inflow = np.tile([1.0, 2.85, 0.0, 1 / GAMMA], (ny, 1))
    c = oracle.Case(2, (nx, ny), [np.full(nx, 1.0 / nx), np.full(ny, 1.0 / ny)], [[3, 4], [2, 4]], gamma=GAMMA, mu=mu,
                    T_wall=spec["T_wall"], multid=0, C_a=0.5, limiter=oracle.LIM_MINMOD,
                    bc_prim=[[inflow, None], [None, None]])
    return c, spec["nodes"], c.prim_to_cons(prim.ravel())


def test_multigrid_converges_to_one_steady_state():
    """Laminar Mach 2.85 flow over a 10-degree corner (32 x 16 cells): three- and four-level cycles
    both drive the residual down by more than 1e5 and reach the same state; after 60 cycles a single
    level is 30 times behind the four-level cycle."""
    nx, ny = 32, 16
    c, nodes, W0 = corner_case(nx, ny)
    out = {}
    for levels in (1, 3, 4):
        W = W0.copy()
        hist = []
        for it in range(150 if levels > 1 else 60):
            W, res, st = c.steady_cycle(nodes, W, 1.0 if it < 15 else 10.0, levels=levels, tiles=(nx, ny), nthreads=8)
            assert st == 0
            hist.append(res)
        out[levels] = (W, hist)
    for levels in (3, 4):
        W, hist = out[levels]
        assert hist[-1] < 1e-5 * hist[0]
    assert out[1][1][-1] > 30 * out[4][1][59]
    W3, W4 = out[3][0], out[4][0]
    assert np.abs(W3 - W4).max() < 1e-6 * np.abs(W4).max()
    # the steady state: its residual is zero to the convergence level
    _, R = c.steady_residual(nodes, W4, cfl_flux=0.5)
    assert np.abs(R).max() < 1e-4 * np.abs(c.steady_residual(nodes, W0, cfl_flux=0.5)[1]).max()
