"""Parity of the CUDA step kernel with third-order MUSCL and fifth-order WENO face reconstruction
(the higher-order options of the paper's Section 4) against the oracle."""
import numpy as np
import pytest

from paper_1302_2132_gb300 import inputs
from tests.cases import gpu_solver, max_rel_elementwise, oracle_case, rel_err_per_var
from tests.test_gpu_parity import step_both

pytestmark = pytest.mark.gpu

MUSCL3, WENO5 = 1, 2


def cases():
    sod = inputs.sod_1d(200)
    turb = inputs.turbulence(48, 2, seed=1302)
    sbl = inputs.shock_boundary_layer(64, 40)
    t3 = inputs.turbulence(14, 3, seed=2132)
    return {
        "sod1d": (sod, dict(C_a=1.0, limiter=1, mu=1e-5, multid=0), 4),
        "turb2d_multid": (turb, dict(turb_model=2, mu=1e-5), 3),
        "turb2d_directional": (turb, dict(turb_model=2, mu=1e-5, multid=0), 3),
        "shock_bl": (sbl, dict(turb_model=3, mu=sbl["mu"], C_a=0.5), 3),
        "turb3d": (t3, dict(turb_model=2, mu=1e-5), 2),
    }


@pytest.mark.parametrize("recon", [MUSCL3, WENO5])
@pytest.mark.parametrize("name", list(cases()))
def test_fp64_higher_order_step_matches_oracle(name, recon):
    spec, kw, steps = cases()[name]
    s, c, Wg, Wo, res = step_both(spec, nsteps=steps, recon=recon, **kw)
    assert np.all(max_rel_elementwise(Wg, Wo, spec["dim"] + 2, 1e-2) < 1e-12)
    s.close()


def test_reconstruction_changes_the_result():
    """The options are in effect: WENO5 and MUSCL3 steps differ from the MUSCL2 one by far more than
    rounding on a turbulent field."""
    spec, kw, steps = cases()["turb2d_multid"]
    out = {}
    for recon in (0, MUSCL3, WENO5):
        s, c, Wg, Wo, res = step_both(spec, nsteps=2, recon=recon, **kw)
        out[recon] = Wg
        s.close()
    nv = 4
    assert np.all(rel_err_per_var(out[WENO5], out[0], nv) > 1e-9)
    assert np.all(rel_err_per_var(out[MUSCL3], out[0], nv) > 1e-9)


@pytest.mark.parametrize("recon", [MUSCL3, WENO5])
def test_fp32_higher_order_close_to_oracle(recon):
    spec = inputs.turbulence(64, 2, seed=8)
    kw = dict(turb_model=2, mu=1e-5)
    s = gpu_solver(spec, precision="fp32", recon=recon, **kw)
    c = oracle_case(spec, recon=recon, **kw)
    s.set_state(spec["prim"].ravel(), layout="soa_prim")
    s.set_turbulence(spec["f1"].ravel(), spec["f2"].ravel())
    W = c.prim_to_cons(spec["prim"].ravel())
    for _ in range(30):
        dt = c.compute_dt(W, 0.5)
        W, st, _ = c.step(W, dt, f1=spec["f1"].ravel(), f2=spec["f2"].ravel(), nthreads=8)
        assert st == 0
    s.step(nsteps=30, cfl=0.5)
    Wg = s.get_state()
    n = W.size // 4
    assert np.abs(Wg[:n] - W[:n]).sum() / np.abs(W[:n]).sum() < 1e-5
    s.close()


def test_unsupported_combinations_are_rejected():
    from paper_1302_2132_gb300 import gks
    spec = inputs.turbulence(16, 2, seed=1)
    with pytest.raises(gks.GksError):
        gpu_solver(spec, precision="fp32_acc64", recon=WENO5)
    t3 = inputs.turbulence(8, 3, seed=1)
    with pytest.raises(gks.GksError):
        gpu_solver(t3, multid=0, recon=MUSCL3)


@pytest.mark.parametrize("recon", [MUSCL3, WENO5])
def test_higher_order_tile_shapes_agree(monkeypatch, recon):
    """The 32x15 and 32x27 tiles of the higher-order step evaluate the same faces (FP32 rounding)."""
    spec = inputs.turbulence(70, 2, seed=5)
    out = []
    for v in ("0", "3"):
        monkeypatch.setenv("GKS_TILE_VARIANT", v)
        s = gpu_solver(spec, precision="fp32", recon=recon, turb_model=2, mu=1e-5)
        s.set_state(spec["prim"].ravel(), layout="soa_prim")
        s.set_turbulence(spec["f1"].ravel(), spec["f2"].ravel())
        s.step(nsteps=20, cfl=0.5)
        assert s.tile_shape()[0] == int(v)
        out.append(s.get_state())
        s.close()
    assert np.all(rel_err_per_var(out[1], out[0], 4) < 1e-6)
