"""The first-order fallback of MUSCL on the GPU (reading R12: a face side whose reconstructed
density or pressure is not positive is evaluated at first order), against the oracle.

States with expansion kinks (inputs.near_vacuum: velocity -1, 0, +1 across a low-pressure cell in a
smooth background) make the reconstruction non-physical on both faces of each kink's middle cell;
the oracle counts them (the branch really fires) and the CUDA path must take the same decision at
the same faces: FP64 element by element at 1e-12 of each variable's scale, the
FP32 forms (whose test is the quotient-free 2 rho (rho E) > |rho U|^2) within their flux accuracy.
Every other face keeps a Mach number below 3, where the moment algebra is well conditioned (on
states with face Mach numbers of 10 to 30 the double-precision flux of any formulation loses digits
as M^4), and over the three steps compared every reconstructed pressure stays at least 0.0019 (a
tenth of the kink pressure) away from zero (checked with the oracle's reconstruction), ten
thousand times the single-precision rounding of the test.
"""
import numpy as np
import pytest

from cases import gpu_solver, max_rel_elementwise, oracle_case
from paper_1302_2132_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

CASES = {
    "1d_64": (dict(n=64, dim=1, seed=1), dict(C_a=0.3, mu=1e-3, multid=0)),
    "2d_24_multid": (dict(n=24, dim=2, seed=3), dict(C_a=0.3, mu=1e-3, multid=1)),
    "2d_24_directional_minmod": (dict(n=24, dim=2, seed=3), dict(C_a=0.3, mu=1e-3, multid=0, limiter=0)),
}


def run_both(name, precision, nsteps=3):
    ikw, kw = CASES[name]
    spec = inputs.near_vacuum(**ikw)
    nv = spec["dim"] + 2
    c = oracle_case(spec, **kw)
    W0 = c.prim_to_cons(spec["prim"].ravel())
    s = gpu_solver(spec, precision=precision, **kw)
    s.set_state(spec["prim"].ravel(), layout="soa_prim")
    W = W0
    fb = []
    for _ in range(nsteps):
        fb.append(c.fallback_count(W))
        dt = c.compute_dt(W, 0.3)
        s.step(nsteps=1, dt=dt)
        W, st, _ = c.step(W, dt, nthreads=8)
        assert st == 0
    Wg = s.get_state()
    s.close()
    return nv, W0, W, Wg, fb


@pytest.mark.parametrize("name", list(CASES))
def test_fallback_fp64_matches_oracle_elementwise(name):
    nv, W0, Wo, Wg, fb = run_both(name, "fp64")
    assert fb[0] > 0, fb  # the branch fires on the initial state
    err = max_rel_elementwise(Wg, Wo, nv, 1e-2)
    assert np.all(err < 1e-12), err
    # the increments themselves, per element, at the scale of each variable's increment
    inc = max_rel_elementwise(Wg - W0, Wo - W0, nv, 1e-2)
    assert np.all(inc < 1e-9), inc


@pytest.mark.parametrize("precision", ["fp32", "fp32_acc64"])
@pytest.mark.parametrize("name", list(CASES))
def test_fallback_fp32_forms_take_the_same_decisions(name, precision):
    """A side decided differently from the oracle changes the increments of its two cells by O(1);
    the FP32 flux itself is accurate to about 1e-4 of an increment."""
    nv, W0, Wo, Wg, fb = run_both(name, precision)
    assert fb[0] > 0 and np.all(np.isfinite(Wg))
    inc = max_rel_elementwise(Wg - W0, Wo - W0, nv, 1e-2)
    assert np.all(inc < 2e-3), inc
