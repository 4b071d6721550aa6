"""Parity of the CUDA k-omega transport (GKS_TURB_KOMEGA_TRANSPORT) with the oracle: the flow step
with tau_t from the transported fields, then rho k and rho omega advanced by the same dt (Wilcox's
2006 k-omega model, the reading of the paper's Section 4)."""
import math

import numpy as np
import pytest

from paper_1302_2132_gb300 import inputs
from tests.cases import gpu_solver, max_rel_elementwise, oracle_case

pytestmark = pytest.mark.gpu

KOMEGA = 3  # oracle turbulence code of the k-omega relaxation time
TRANSPORT = 4


def transport_fields(spec, seed, own=False):
    """k and omega for a case: the spec's own k-omega fields (own=True), else seeded positive fields."""
    n = spec["prim"][0].size
    if own:
        return np.asarray(spec["f1"], dtype=np.float64).ravel(), np.asarray(spec["f2"], dtype=np.float64).ravel()
    rng = np.random.default_rng(seed)
    k = 0.01 * (1.0 + 0.5 * rng.random(n))
    om = 20.0 * (1.0 + 0.5 * rng.random(n))
    return k, om


def run_both(spec, nsteps, k, om, precision="fp64", C_a=0.0, mu=1e-5, cfl=0.5, coeffs=None):
    import oracle
    dim = spec["dim"]
    nv = dim + 2
    c = oracle_case(spec, turb_model=KOMEGA, C_a=C_a, mu=mu)
    s = gpu_solver(spec, turb_model=TRANSPORT, C_a=C_a, mu=mu, precision=precision)
    s.set_state(spec["prim"].ravel(), layout="soa_prim")
    s.set_turbulence(k, om)
    if coeffs:
        s.set_komega(**coeffs)
    W = c.prim_to_cons(spec["prim"].ravel())
    rho = W[: W.size // nv]
    RK, RW = k * rho, om * rho
    oc = oracle.komega_defaults(**(coeffs or {}))
    for _ in range(nsteps):
        dt = c.compute_dt(W, cfl)
        W, RK, RW, st = c.step_komega(W, RK, RW, dt, coeffs=oc, nthreads=8)
        assert st == 0
    s.step(nsteps=nsteps, cfl=cfl)
    Wg = s.get_state()
    kg, wg = s.get_turbulence()
    rho = W[: W.size // nv]
    return s, Wg, W, kg, wg, RK / rho, RW / rho


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


@pytest.mark.parametrize("name", ["turb2d", "turb1d", "turb3d", "shock_bl"])
def test_fp64_transport_matches_oracle(name):
    if name == "turb2d":
        spec, steps = inputs.turbulence(40, 2, seed=11), 5
    elif name == "turb1d":
        spec, steps = inputs.turbulence_1d(96, seed=12), 8
    elif name == "turb3d":
        spec, steps = inputs.turbulence(12, 3, seed=13), 3
    else:
        spec, steps = inputs.shock_boundary_layer(48, 30), 4
    k, om = transport_fields(spec, seed=7, own=name == "shock_bl")
    C_a = 0.5 if name == "shock_bl" else 0.0
    mu = spec.get("mu", 1e-5)
    s, Wg, Wo, kg, wg, ko, wo = run_both(spec, steps, k, om, C_a=C_a, mu=mu)
    nv = spec["dim"] + 2
    assert np.all(max_rel_elementwise(Wg, Wo, nv, 1e-2) < 1e-12)
    assert rel(kg, ko) < 1e-12 and rel(wg, wo) < 1e-12
    # the fields did evolve
    assert rel(ko, k) > 1e-6 and rel(wo, om) > 1e-6
    s.close()


def test_fp32_transport_close_to_oracle():
    spec = inputs.turbulence(48, 2, seed=21)
    k, om = transport_fields(spec, seed=3)
    s, Wg, Wo, kg, wg, ko, wo = run_both(spec, 40, k, om, precision="fp32")
    l1 = lambda a, b: np.abs(a - b).sum() / np.abs(b).sum()
    assert l1(Wg[: ko.size], Wo[: ko.size]) < 1e-5
    assert l1(kg, ko) < 1e-5 and l1(wg, wo) < 1e-5
    s.close()


def test_homogeneous_decay_on_the_device():
    """Fluid at rest with uniform k, omega: omega follows 1/omega = 1/omega0 + beta0 t exactly (the
    point-implicit destruction), k the first-order discrete solution of dk/dt = -beta* k omega."""
    n = 16
    spec = inputs.turbulence(n, 2, seed=1)
    spec["prim"] = np.array(spec["prim"], dtype=np.float64)
    spec["prim"][1:3] = 0.0
    spec["prim"][0] = 1.0
    spec["prim"][3] = 1.0 / 1.4
    s = gpu_solver(spec, turb_model=TRANSPORT, mu=1e-5)
    s.set_state(spec["prim"].ravel(), layout="soa_prim")
    k0, w0, dt, steps = 0.02, 40.0, 1e-4, 300
    s.set_turbulence(np.full(n * n, k0), np.full(n * n, w0))
    s.step(nsteps=steps, dt=dt)
    kg, wg = s.get_turbulence()
    T = dt * steps
    assert np.allclose(wg, 1.0 / (1.0 / w0 + 0.0708 * T), rtol=1e-12, atol=0)
    kk = k0
    w = w0
    for _ in range(steps):
        kk = kk / (1.0 + dt * 0.09 * w)
        w = w / (1.0 + dt * 0.0708 * w)
    assert np.allclose(kg, kk, rtol=1e-12, atol=0)
    assert abs(kk / (k0 * (1 + 0.0708 * w0 * T) ** (-0.09 / 0.0708)) - 1) < 0.01
    s.close()


def test_graph_and_eager_transport_are_bitwise_equal():
    spec = inputs.turbulence(64, 2, seed=31)
    k, om = transport_fields(spec, seed=9)
    out = []
    for timing in (False, True):
        s = gpu_solver(spec, turb_model=TRANSPORT, precision="fp32")
        s.set_state(spec["prim"].ravel(), layout="soa_prim")
        s.set_turbulence(k, om)
        if timing:
            s.enable_timing(True)  # one launch per step, no graphs
        s.step(nsteps=100, cfl=0.5)
        out.append((s.get_state(), *s.get_turbulence()))
        s.close()
    for a, b in zip(out[0], out[1]):
        assert np.array_equal(a, b)


def test_set_state_clears_the_transported_fields():
    from paper_1302_2132_gb300 import gks
    spec = inputs.turbulence(16, 2, seed=2)
    s = gpu_solver(spec, turb_model=TRANSPORT)
    with pytest.raises(gks.GksError):
        s.set_turbulence(np.full(256, 0.01), np.full(256, 10.0))  # no state yet
    s.set_state(spec["prim"].ravel(), layout="soa_prim")
    s.set_turbulence(np.full(256, 0.01), np.full(256, 10.0))
    s.step(nsteps=2, cfl=0.5)
    s.set_state(spec["prim"].ravel(), layout="soa_prim")
    with pytest.raises(gks.GksError):
        s.step(nsteps=1, cfl=0.5)
    s.close()
