"""Pins of the oracle's higher-order face reconstructions (Section 4 lists second- and third-order
MUSCL and fifth-order WENO next to the second-order results it shows): order of accuracy of the
face values on exact cell averages of a smooth function, exactness on polynomials, and the whole
scheme on the Sod problem and a smooth density wave."""
import math

import numpy as np
import pytest

import oracle
import exact_riemann as er


def cell_averages(F, edges):
    return (F(edges[1:]) - F(edges[:-1])) / np.diff(edges)


@pytest.mark.parametrize("recon,order", [(oracle.RECON_MUSCL2, 1.8), (oracle.RECON_MUSCL3, 2.8),
                                         (oracle.RECON_WENO5, 4.6)])
def test_face_values_converge_at_the_design_order(recon, order):
    """exp(x) on [0, 1] (smooth and monotone, so no limiter clips): the error of the face values
    falls as h^2, h^3, h^5."""
    errs = []
    for n in (40, 80, 160):
        edges = np.linspace(0.0, 1.0, n + 1)
        v = cell_averages(np.exp, edges)
        wl, wr = oracle.reconstruct(recon, v, np.diff(edges))
        face = np.exp(edges[1:])  # right face of cell i
        ok = ~np.isnan(wl)
        okr = ~np.isnan(wr)
        e = max(np.abs(wl[ok] - face[ok]).max(), np.abs(wr[okr] - np.exp(edges[:-1][okr])).max())
        errs.append(e)
    rates = [math.log2(a / b) for a, b in zip(errs, errs[1:])]
    assert min(rates) > order, (errs, rates)


@pytest.mark.parametrize("recon", [oracle.RECON_MUSCL3, oracle.RECON_WENO5])
def test_quadratics_are_reproduced_exactly(recon):
    """Cell averages of a convex monotone quadratic give its exact face values (third- and
    fifth-order reconstructions are exact for degree 2; no limiting on monotone data)."""
    n = 24
    edges = np.linspace(0.0, 2.0, n + 1)
    F = lambda x: x ** 3 / 3.0 + 0.5 * x ** 2 + x  # antiderivative of x^2 + x + 1
    v = cell_averages(F, edges)
    wl, wr = oracle.reconstruct(recon, v, np.diff(edges))
    f = lambda x: x ** 2 + x + 1
    ok = ~np.isnan(wl)
    assert np.allclose(wl[ok], f(edges[1:][ok]), rtol=1e-13 if recon == oracle.RECON_MUSCL3 else 1e-6)
    okr = ~np.isnan(wr)
    assert np.allclose(wr[okr], f(edges[:-1][okr]), rtol=1e-13 if recon == oracle.RECON_MUSCL3 else 1e-6)


def sod_case(n, recon):
    dx = [np.full(n, 1.0 / n)]
    case = oracle.Case(1, (n,), dx, [(oracle.BC_TRANSMISSIVE, oracle.BC_TRANSMISSIVE)], gamma=1.4, mu=1e-5,
                       C_a=1.0, limiter=oracle.LIM_VANLEER, recon=recon)
    x = (np.arange(n) + 0.5) / n
    prim = np.zeros((3, n))
    prim[0] = np.where(x < 0.5, 1.0, 0.125)
    prim[2] = np.where(x < 0.5, 1.0, 0.1)
    return case, case.prim_to_cons(prim.ravel()), x


@pytest.mark.parametrize("recon", [oracle.RECON_MUSCL3, oracle.RECON_WENO5])
def test_sod_with_higher_order_reconstruction(recon):
    """The scheme stays stable through the shock tube and is at least as close to the exact
    solution as the second-order MUSCL default."""
    n = 200
    errs = {}
    for r in (oracle.RECON_MUSCL2, recon):
        case, W, x = sod_case(n, r)
        W, t, steps, st = case.run(W, 2000, cfl=0.5, t_end=0.2, nthreads=8)
        assert st == 0 and abs(t - 0.2) < 1e-12
        rho = W[:n]
        ex = er.cell_average((1.0, 0.0, 1.0), (0.125, 0.0, 0.1), np.linspace(0.0, 1.0, n + 1), 0.2, sub=16)
        errs[r] = np.abs(rho - ex[0]).mean()
    assert errs[recon] < 0.016
    assert errs[recon] < 1.05 * errs[oracle.RECON_MUSCL2]


def test_smooth_density_wave_is_more_accurate_with_weno():
    """rho = 1 + 0.2 sin(2 pi x), u = 1, p = 1, periodic: after one period the fifth-order
    reconstruction leaves a smaller error than the second-order one at the same resolution."""
    n, T = 64, 1.0
    errs = {}
    for r in (oracle.RECON_MUSCL2, oracle.RECON_WENO5):
        dx = [np.full(n, 1.0 / n)]
        case = oracle.Case(1, (n,), dx, [(oracle.BC_PERIODIC, oracle.BC_PERIODIC)], gamma=1.4, mu=1e-6,
                           limiter=oracle.LIM_VANLEER, recon=r)
        x = (np.arange(n) + 0.5) / n
        prim = np.zeros((3, n))
        prim[0] = 1.0 + 0.2 * np.sin(2 * math.pi * x)
        prim[1] = 1.0
        prim[2] = 1.0
        W = case.prim_to_cons(prim.ravel())
        W, t, steps, st = case.run(W, 100000, cfl=0.4, t_end=T, nthreads=8)
        assert st == 0
        h = 1.0 / n
        # cell average of the profile, unchanged after one period of the entropy wave
        exact = 1.0 + 0.2 * np.sin(2 * math.pi * x) * math.sin(math.pi * h) / (math.pi * h)
        errs[r] = np.abs(W[:n] - exact).mean()
    assert errs[oracle.RECON_WENO5] < 0.5 * errs[oracle.RECON_MUSCL2], errs
