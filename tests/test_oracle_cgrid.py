"""Pins of the C-grid wake cut of the oracle's body-fitted step (the grid type of the paper's aerofoil
cases, Table 2): the cells beside the cut see the cells across it exactly as a rectilinear grid
would, a symmetric section in a symmetric flow stays symmetric, and the cut is not a wall."""
import numpy as np

import oracle
from paper_1302_2132_gb300 import inputs

GAMMA = 1.4


def profile(y):
    """A state and turbulence fields that depend on y only."""
    prim = np.stack([1.0 + 0.1 * np.exp(-(y / 0.4) ** 2), 0.7 + 0.2 * np.tanh(y / 0.3), 0.05 * np.sin(y),
                     (1.0 + 0.05 * np.exp(-y * y)) / GAMMA])
    return prim, 0.01 * (1.0 + 0.5 * np.exp(-y * y)), 5.0 * (1.0 + 0.3 * np.cos(y))


def test_wake_cells_step_as_on_a_rectilinear_grid():
    """C-grid with a rectilinear wake (vertical grid lines, rows at -eta R below and +eta^0.8 R above
    the cut) and a y-only state: every wake cell at least three cells from the trailing edge steps
    exactly as the matching cell of a periodic rectilinear grid with the same rows (k-epsilon tau_t,
    so the Green-Gauss gradients and the fields across the cut are exercised too)."""
    nw, ns, n1, R = 12, 16, 8, 3.0
    sp = inputs.naca0012_case(nw, ns, n1, R=R, x_out=4.0, mach=0.7, alpha_deg=0.0)
    nodes = sp["nodes"].copy()
    n0 = sp["n"][0]
    # rows of the upper half spaced differently from the lower half, so that the cells across the
    # cut are not mirror images of the cells beside it
    eta = -nodes[:, 0, 1] / R
    eta_up = eta ** 0.8
    for i in range(n0 // 2 + 1, n0 + 1):
        nodes[:, i] = nodes[0, i] + eta_up[:, None] * (nodes[-1, i] - nodes[0, i])
    pts = inputs.cell_points(nodes)
    prim, f1, f2 = profile(pts[..., 1])
    c = oracle.Case(2, sp["n"], sp["dx"], sp["bc"], gamma=GAMMA, mu=1e-3, T_wall=sp["T_wall"], multid=0, C_a=0.3,
                    turb_model=oracle.TURB_KEPS, bc_prim=sp["bc_prim"], wake_cut=nw)
    W = c.prim_to_cons(prim.ravel())
    dt = 2e-3
    Wc, st = c.step_curv(nodes, W, dt, f1=f1.ravel(), f2=f2.ravel(), nthreads=4)
    assert st == 0
    # the rectilinear reference: 8 periodic columns of the wake's width, rows mirrored about y = 0
    ys = np.concatenate([-eta[::-1] * R, eta_up[1:] * R])
    nx = 8
    xs = np.arange(nx + 1) * (3.0 / nw)
    X, Y = np.meshgrid(xs, ys, indexing="xy")
    rnodes = np.stack([X, Y], axis=-1)
    rpts = inputs.cell_points(rnodes)
    rprim, rf1, rf2 = profile(rpts[..., 1])
    free = sp["bc_prim"][1][1][0]
    dirich = np.tile(free, (nx, 1))
    r = oracle.Case(2, (nx, 2 * n1), [np.full(nx, 1.0), np.full(2 * n1, 1.0)], [[0, 0], [3, 3]], gamma=GAMMA, mu=1e-3,
                    multid=0, C_a=0.3, turb_model=oracle.TURB_KEPS, bc_prim=[[None, None], [dirich, dirich]])
    Wr0 = r.prim_to_cons(rprim.ravel())
    Wr, st = r.step_curv(rnodes, Wr0, dt, f1=rf1.ravel(), f2=rf2.ravel(), nthreads=4)
    assert st == 0
    Wc, W = Wc.reshape(4, n1, n0), W.reshape(4, n1, n0)
    Wr, Wr0 = Wr.reshape(4, 2 * n1, nx), Wr0.reshape(4, 2 * n1, nx)
    checked = 0
    for i in range(0, nw - 2):
        for j in range(n1):
            for (ci, rj) in ((i, n1 - 1 - j), (n0 - 1 - i, n1 + j)):
                dc = Wc[:, j, ci] - W[:, j, ci]
                dr = Wr[:, rj, 3] - Wr0[:, rj, 3]
                assert np.abs(dc - dr).max() <= 1e-10 * np.abs(dr).max() + 1e-15, (i, j, ci)
                checked += 1
    assert checked == 2 * (nw - 2) * n1


def mirror(W, n0, n1):
    W = W.reshape(4, n1, n0)
    M = W[:, :, ::-1].copy()
    M[2] = -M[2]
    return M


def test_symmetric_section_stays_symmetric_and_the_cut_is_not_a_wall():
    nw, ns, n1 = 10, 24, 10
    sp = inputs.naca0012_case(nw, ns, n1, mach=0.75, alpha_deg=0.0)
    nodes = sp["nodes"]
    n0 = sp["n"][0]
    pts = inputs.cell_points(nodes)
    prim = np.array(sp["prim"], dtype=np.float64)
    bump = np.exp(-((pts[..., 0] - 2.0) ** 2 + pts[..., 1] ** 2) / 0.5)
    prim[0] *= 1.0 + 0.1 * bump
    prim[1] *= 1.0 - 0.2 * bump
    out = {}
    for cut in (nw, 0):
        c = oracle.Case(2, sp["n"], sp["dx"], sp["bc"], gamma=GAMMA, mu=1e-3, T_wall=sp["T_wall"], multid=0, C_a=0.5,
                        bc_prim=sp["bc_prim"], wake_cut=cut)
        W = c.prim_to_cons(prim.ravel())
        for _ in range(3):
            dt = c.compute_dt_curv(nodes, W, 0.5)
            W, st = c.step_curv(nodes, W, dt, nthreads=4)
            assert st == 0
        out[cut] = W
    W = out[nw].reshape(4, n1, n0)
    M = mirror(out[nw], n0, n1)
    for v in range(4):
        assert np.abs(W[v] - M[v]).max() < 1e-12 * max(np.abs(W[v]).max(), 1.0)
    # with a wall in place of the cut the flow along the wake is held back
    Ww = out[0].reshape(4, n1, n0)
    assert np.abs(Ww[1, 0, :nw] - W[1, 0, :nw]).max() > 1e-3


def test_multigrid_cycles_run_on_a_c_grid():
    """The steady solver coarsens the cut with the grid (n_wake halves per level) and its residual
    falls."""
    sp = inputs.naca0012_case(8, 32, 16, mach=0.6, alpha_deg=2.0, Re=2e3)
    c = oracle.Case(2, sp["n"], sp["dx"], sp["bc"], gamma=GAMMA, mu=sp["mu"], T_wall=sp["T_wall"], multid=0, C_a=0.5,
                    limiter=oracle.LIM_MINMOD, bc_prim=sp["bc_prim"], wake_cut=8)
    W = c.prim_to_cons(np.array(sp["prim"]).ravel())
    hist = []
    for it in range(40):
        W, res, st = c.steady_cycle(sp["nodes"], W, 1.0 if it < 10 else 3.0, levels=3, tiles=(16, 16), nthreads=8)
        assert st == 0
        hist.append(res)
    assert hist[-1] < 0.2 * max(hist)


def kw_profile(y):
    """k and omega rising through the cut (y = 0), so that their limited slopes there are not zero."""
    return 0.01 * (1.0 + 0.4 * np.tanh(y / 0.4)), 20.0 * (1.0 + 0.3 * np.tanh((y - 0.05) / 0.5))


def test_transport_across_the_wake_cut_matches_a_rectilinear_strip():
    """The k-omega transport sees the cells across the cut as a rectilinear grid would: the same
    C-grid / periodic-strip construction as above, y-only state and fields, and every wake cell at
    least three cells from the trailing edge takes the increments of rho, rho k and rho omega of the
    matching strip cell (convection, diffusion and the Green-Gauss source gradients across the cut)."""
    nw, ns, n1, R = 12, 16, 8, 3.0
    sp = inputs.naca0012_case(nw, ns, n1, R=R, x_out=4.0, mach=0.7, alpha_deg=0.0)
    nodes = sp["nodes"].copy()
    n0 = sp["n"][0]
    eta = -nodes[:, 0, 1] / R
    eta_up = eta ** 0.8
    for i in range(n0 // 2 + 1, n0 + 1):
        nodes[:, i] = nodes[0, i] + eta_up[:, None] * (nodes[-1, i] - nodes[0, i])
    pts = inputs.cell_points(nodes)
    prim, _, _ = profile(pts[..., 1])
    k, om = kw_profile(pts[..., 1])
    c = oracle.Case(2, sp["n"], sp["dx"], sp["bc"], gamma=GAMMA, mu=1e-3, T_wall=sp["T_wall"], multid=0, C_a=0.3,
                    turb_model=oracle.TURB_KOMEGA, bc_prim=sp["bc_prim"], wake_cut=nw)
    W = c.prim_to_cons(prim.ravel())
    nc = n0 * n1
    RK, RW = k.ravel() * W[:nc], om.ravel() * W[:nc]
    dt = 2e-3
    Wc, RKc, RWc, st = c.step_komega_curv(nodes, W, RK, RW, dt, nthreads=4)
    assert st == 0
    ys = np.concatenate([-eta[::-1] * R, eta_up[1:] * R])
    nx = 8
    xs = np.arange(nx + 1) * (3.0 / nw)
    X, Y = np.meshgrid(xs, ys, indexing="xy")
    rnodes = np.stack([X, Y], axis=-1)
    rpts = inputs.cell_points(rnodes)
    rprim, _, _ = profile(rpts[..., 1])
    rk, rom = kw_profile(rpts[..., 1])
    free = sp["bc_prim"][1][1][0]
    dirich = np.tile(free, (nx, 1))
    r = oracle.Case(2, (nx, 2 * n1), [np.full(nx, 1.0), np.full(2 * n1, 1.0)], [[0, 0], [3, 3]], gamma=GAMMA, mu=1e-3,
                    multid=0, C_a=0.3, turb_model=oracle.TURB_KOMEGA, bc_prim=[[None, None], [dirich, dirich]])
    Wr0 = r.prim_to_cons(rprim.ravel())
    nr = nx * 2 * n1
    RKr0, RWr0 = rk.ravel() * Wr0[:nr], rom.ravel() * Wr0[:nr]
    Wr, RKr, RWr, st = r.step_komega_curv(rnodes, Wr0, RKr0, RWr0, dt, nthreads=4)
    assert st == 0
    fields_c = [(Wc[:nc] - W[:nc]), (RKc - RK), (RWc - RW)]
    fields_r = [(Wr[:nr] - Wr0[:nr]), (RKr - RKr0), (RWr - RWr0)]
    checked = 0
    for fc_, fr_ in zip(fields_c, fields_r):
        fc_, fr_ = fc_.reshape(n1, n0), fr_.reshape(2 * n1, nx)
        scale = np.abs(fr_).max()
        assert scale > 0
        for i in range(0, nw - 2):
            for j in range(n1):
                for (ci, rj) in ((i, n1 - 1 - j), (n0 - 1 - i, n1 + j)):
                    assert abs(fc_[j, ci] - fr_[rj, 3]) <= 1e-10 * scale + 1e-15, (i, j, ci)
                    checked += 1
    assert checked == 3 * 2 * (nw - 2) * n1
