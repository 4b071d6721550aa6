"""Pins of the oracle's rarefaction diagnostic on body-fitted grids (Eqs. tautautilde, tautilde with
D rho = -rho div U): the rectilinear diagnostic on a uniform grid, and the exact divergence of a
linear velocity field on an affine grid."""
import numpy as np

import oracle
from paper_1302_2132_gb300 import inputs

GAMMA = 1.4


def test_uniform_grid_equals_the_rectilinear_diagnostic():
    n = 20
    spec = inputs.turbulence(n, 2, seed=7)
    h = spec["dx"][0][0]
    c = oracle.Case(2, (n, n), spec["dx"], [(0, 0), (0, 0)], gamma=GAMMA, mu=1e-3, turb_model=oracle.TURB_KEPS,
                    C_mu=0.09, multid=0)
    W = c.prim_to_cons(spec["prim"].ravel())
    f1, f2 = spec["f1"].ravel(), spec["f2"].ravel()
    er = c.rarefaction(W, f1, f2)
    ec = c.rarefaction_curv(inputs.uniform_nodes(n, n, n * h, n * h), W, f1, f2)
    assert np.abs(ec - er).max() < 1e-12 * np.abs(er).max()
    assert np.abs(er).max() > 0.0


def test_linear_velocity_on_an_affine_grid_gives_the_exact_divergence():
    """U = (a x + c y, d x + b y) with uniform rho and p on a sheared, stretched parallelogram lattice:
    Green-Gauss with face means is exact for linear fields there, so every cell away from the
    boundary has eps = mu / p |a + b| (no turbulence model)."""
    n0, n1 = 16, 12
    xi, eta = np.meshgrid(np.arange(n0 + 1) * 0.1, np.arange(n1 + 1) * 0.07, indexing="xy")
    nodes = np.stack([xi + 0.4 * eta, 0.9 * eta - 0.2 * xi], axis=-1)
    pts = inputs.cell_points(nodes)
    a, b, cc, d = 0.7, -0.25, 0.3, -0.45
    rho, p, mu = 1.2, 0.8, 2e-3
    prim = np.zeros((4, n1, n0))
    prim[0], prim[3] = rho, p
    prim[1] = a * pts[..., 0] + cc * pts[..., 1]
    prim[2] = d * pts[..., 0] + b * pts[..., 1]
    c = oracle.Case(2, (n0, n1), [np.ones(n0), np.ones(n1)], [(4, 4), (4, 4)], gamma=GAMMA, mu=mu, multid=0)
    eps = c.rarefaction_curv(nodes, c.prim_to_cons(prim.ravel())).reshape(n1, n0)
    inner = eps[1:-1, 1:-1]
    assert np.allclose(inner, mu / p * abs(a + b), rtol=1e-12, atol=0)
    assert np.all(np.isfinite(eps))
