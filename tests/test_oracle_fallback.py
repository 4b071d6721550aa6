"""Pins of the oracle's first-order fallback (MUSCL on conservative variables; a face side whose
reconstructed density or pressure is not positive is evaluated at first order, reading R12).

On a 1D state with expansion kinks (inputs.near_vacuum: velocity -1, 0, +1 across a low-pressure cell)
the reconstruction gives negative pressure on both faces of each kink's middle cell.  The oracle's step must equal the step assembled here from the pinned
pieces: the oracle's row reconstruction (pinned by its convergence orders), the first-order record
(face value = cell average, slope 0) on exactly the sides with non-positive rho or p, the pinned face
flux, and the finite-volume update.  Without the fallback (a mistake planted in the oracle) the same
step is not finite or not physical.
"""
import numpy as np
import pytest

import oracle
from cases import oracle_case
from paper_1302_2132_gb300 import inputs

GAMMA = 1.4


def pressure(w):
    return (GAMMA - 1.0) * (w[2] - 0.5 * w[1] ** 2 / w[0])


def assembled_step_1d(c, spec, W, dt, mu, C_a):
    """The 1D step from the oracle's pinned pieces, with the fallback applied here."""
    n = spec["n"][0]
    h = spec["dx"][0][0]
    Wr = W.reshape(3, n)
    # transmissive ghosts: copies of the boundary cells
    Wp = np.concatenate([np.repeat(Wr[:, :1], 3, axis=1), Wr, np.repeat(Wr[:, -1:], 3, axis=1)], axis=1)
    fl = np.zeros((3, n + 6))
    fr = np.zeros((3, n + 6))
    for v in range(3):
        fl[v], fr[v] = oracle.reconstruct(oracle.RECON_MUSCL2, Wp[v], np.full(n + 6, h), limiter=oracle.LIM_VANLEER)
    def vanleer_slope(k):  # the limited slope of padded cell k (van Leer, reading R12)
        dm, dp = (Wp[:, k] - Wp[:, k - 1]) / (0.5 * (h + h)), (Wp[:, k + 1] - Wp[:, k]) / (0.5 * (h + h))
        return np.where(dm * dp > 0.0, 2.0 * dm * dp / np.where(dm + dp == 0.0, 1.0, dm + dp), 0.0)

    F = np.zeros((n + 1, 3))
    sides = 0
    for j in range(n + 1):  # face between padded cells j + 2 and j + 3
        a, b = j + 2, j + 3
        wl, wr = fl[:, a].copy(), fr[:, b].copy()
        sl, sr = vanleer_slope(a), vanleer_slope(b)
        if not (wl[0] > 0 and pressure(wl) > 0):
            wl, sl = Wp[:, a].copy(), np.zeros(3)
            sides += 1
        if not (wr[0] > 0 and pressure(wr) > 0):
            wr, sr = Wp[:, b].copy(), np.zeros(3)
            sides += 1
        face = oracle.make_face(1, wl, wr, Wp[:, a], Wp[:, b], sl, sr, None, None, 0.5 * h, 0.5 * h, 0.0)
        F[j] = oracle.face_flux(1, GAMMA, mu, C_a, dt, face, multid=0)
    Wn = Wr - (F[1:].T - F[:-1].T) / h
    return Wn.ravel(), sides


def test_fallback_step_equals_the_first_order_flux_at_the_fallback_faces():
    spec = inputs.near_vacuum(64, 1, seed=1)
    mu, C_a = 1e-3, 0.3
    c = oracle_case(spec, C_a=C_a, mu=mu, multid=0)
    W = c.prim_to_cons(spec["prim"].ravel())
    nfb = c.fallback_count(W)
    dt = c.compute_dt(W, 0.3)
    Wo, st, _ = c.step(W, dt)
    Wa, sides = assembled_step_1d(c, spec, W, dt, mu, C_a)
    assert nfb == sides == 8, (nfb, sides)
    assert st == 0 and np.all(np.isfinite(Wo))
    scale = np.abs(Wo.reshape(3, -1)).max(axis=1)[:, None]
    assert np.all(np.abs((Wo - Wa).reshape(3, -1)) <= 1e-13 * scale)


def test_step_without_the_fallback_is_not_physical():
    """The planted mistake (no fallback) on the same data: the step is not finite or not physical, so
    the fallback pin above is not vacuous."""
    spec = inputs.near_vacuum(64, 1, seed=1)
    c = oracle_case(spec, C_a=0.3, mu=1e-3, multid=0)
    W = c.prim_to_cons(spec["prim"].ravel())
    dt = c.compute_dt(W, 0.3)
    c.P.no_fallback = 1
    Wbad, st, _ = c.step(W, dt)
    assert st != 0 or not np.all(np.isfinite(Wbad))


@pytest.mark.parametrize("dim,n,seed", [(1, 64, 1), (2, 24, 3)])
def test_fallback_keeps_the_expansion_physical(dim, n, seed):
    """With the fallback, five steps at CFL 0.3 of the kinked states keep rho > 0 and p > 0."""
    spec = inputs.near_vacuum(n, dim, seed)
    c = oracle_case(spec, C_a=0.3, mu=1e-3, multid=int(dim > 1))
    W = c.prim_to_cons(spec["prim"].ravel())
    assert c.fallback_count(W) > 0
    W, t, done, st = c.run(W, 5, cfl=0.3, nthreads=4)
    assert done == 5 and st == 0 and np.all(np.isfinite(W))
