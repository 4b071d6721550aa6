"""Full-run parity of the configurations beyond one step (the parity set of the 3D and
shock / boundary-layer workloads, and the FP32 error target L1(rho) <= 1e-5 relative after the run).

  - 3D decaying turbulence: an independent 32^3 periodic instance of the 256^3 generator, 100 steps:
    GPU FP64 against the oracle element by element; both FP32 forms against the same oracle state
    (L1(rho) <= 1e-5).
  - 3D 256^3 (the bench workload), 100 steps: both FP32 forms against the GPU FP64 path (itself the
    oracle to 1e-12 per step) in the bench's launch configuration, L1(rho) <= 1e-5.
  - 3D 256^3, one FP64 step in the bench's launch configuration: sampled cells recomputed by the oracle
    on a 9^3 crop around each (a step cannot carry the crop's own boundary to its centre).
  - shock / boundary layer: the wall corner of the full-size 1024 x 384 grid (its first 16 columns and
    48 rows: the same wall-clustered rows, time step and physical time), the full 5000 steps: GPU
    FP64 against the oracle element by element and both FP32 forms at L1(rho) <= 1e-5.

State comparisons are element by element: |a - b| <= tol max(|b|, 1e-2 max|b_v|) per variable v.
"""
import math
import os

import numpy as np
import pytest

from cases import gpu_solver, l1_rho_rel, max_rel_elementwise, oracle_case
from paper_1302_2132_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

CORES = os.cpu_count() or 1
TURB = dict(turb_model=2, multid=1, mu=1e-5)


def gpu_run(spec, precision, nsteps, cfl=0.5, **kw):
    s = gpu_solver(spec, precision=precision, **kw)
    s.set_state(spec["prim"].ravel(), layout="soa_prim")
    if kw.get("turb_model", 0):
        s.set_turbulence(spec["f1"].ravel(), spec["f2"].ravel())
    s.step(nsteps=nsteps, cfl=cfl)
    t, steps = s.time()
    W = s.get_state()
    s.close()
    return W, t, steps


@pytest.fixture(scope="module")
def turb3d_32_oracle():
    spec = inputs.turbulence(32, 3, seed=2132)
    c = oracle_case(spec, **TURB)
    W0 = c.prim_to_cons(spec["prim"].ravel())
    Wo, t, n, st = c.run(W0, 100, cfl=0.5, f1=spec["f1"].ravel(), f2=spec["f2"].ravel(), nthreads=CORES)
    assert st == 0 and n == 100
    return spec, Wo, t


def test_3d_32_fp64_100_steps_matches_oracle_elementwise(turb3d_32_oracle):
    spec, Wo, to = turb3d_32_oracle
    Wg, tg, n = gpu_run(spec, "fp64", 100, **TURB)
    assert n == 100 and abs(tg - to) <= 1e-12 * to
    err = max_rel_elementwise(Wg, Wo, 5, 1e-2)
    assert np.all(err < 1e-11), err


@pytest.mark.parametrize("precision", ["fp32", "fp32_acc64"])
def test_3d_32_fp32_forms_meet_the_l1_target_after_100_steps(turb3d_32_oracle, precision):
    spec, Wo, _ = turb3d_32_oracle
    Wg, _, n = gpu_run(spec, precision, 100, **TURB)
    l1 = l1_rho_rel(Wg, Wo, 5)
    assert n == 100 and l1 < 1e-5, l1


def test_3d_256_fp32_forms_against_fp64_after_100_steps():
    """The bench workload at full size: FP32 forms within L1(rho) <= 1e-5 of the FP64 path."""
    spec = inputs.turbulence(256, 3, seed=2132)
    W64, t64, _ = gpu_run(spec, "fp64", 100, **TURB)
    for precision in ("fp32_acc64", "fp32"):
        W32, t32, n = gpu_run(spec, precision, 100, **TURB)
        l1 = l1_rho_rel(W32, W64, 5)
        assert n == 100 and l1 < 1e-5, (precision, l1)
        assert abs(t32 - t64) <= 1e-5 * t64


def test_3d_256_fp64_step_sampled_crops_match_oracle():
    spec = inputs.turbulence(256, 3, seed=2132)
    n = 256
    s = gpu_solver(spec, precision="fp64", **TURB)
    s.set_state(spec["prim"].ravel(), layout="soa_prim")
    s.set_turbulence(spec["f1"].ravel(), spec["f2"].ravel())
    dt = s.compute_dt(0.5)
    s.step(nsteps=1, dt=dt)
    Wg = s.get_state().reshape(5, n, n, n)
    s.close()
    rng = np.random.default_rng(7)
    h = 2 * math.pi / n
    crop = dict(dim=3, n=(9, 9, 9), dx=[np.full(9, h)] * 3, bc=[[0, 0]] * 3)
    c = oracle_case(crop, **TURB)
    prim = spec["prim"]
    for _ in range(12):
        k, j, i = rng.integers(0, n, 3)
        kk, jj, ii = ((np.arange(q - 4, q + 5)) % n for q in (k, j, i))
        sl = np.ix_(kk, jj, ii)
        pc = np.stack([prim[v][sl] for v in range(5)])
        W0 = c.prim_to_cons(pc.ravel())
        Wo, st, _ = c.step(W0, dt, f1=spec["f1"][sl].ravel(), f2=spec["f2"][sl].ravel(), nthreads=CORES)
        wo = Wo.reshape(5, 9, 9, 9)[:, 4, 4, 4]
        w0 = W0.reshape(5, 9, 9, 9)[:, 4, 4, 4]
        wg = Wg[:, k, j, i]
        scale = np.abs(W0.reshape(5, -1)).max(axis=1)
        assert np.all(np.abs(wg - wo) <= 1e-12 * np.maximum(np.abs(wo), 1e-2 * scale)), (wg, wo)
        inc_scale = np.maximum(np.abs(wo - w0), 1e-2 * np.abs(Wo - W0).reshape(5, -1).max(axis=1))
        assert np.all(np.abs(wg - wo) <= 1e-9 * inc_scale), (wg - w0, wo - w0)


@pytest.fixture(scope="module")
def shock_bl_oracle():
    spec = inputs.shock_boundary_layer_crop(16, 48)
    kw = dict(turb_model=3, multid=1, mu=spec["mu"], C_a=0.5)
    c = oracle_case(spec, **kw)
    W0 = c.prim_to_cons(spec["prim"].ravel())
    Wo, t, n, st = c.run(W0, 5000, cfl=0.5, f1=spec["f1"].ravel(), f2=spec["f2"].ravel(), nthreads=CORES)
    assert st == 0 and n == 5000
    return spec, kw, Wo, t


def test_shock_bl_fp64_5000_steps_matches_oracle_elementwise(shock_bl_oracle):
    spec, kw, Wo, to = shock_bl_oracle
    Wg, tg, n = gpu_run(spec, "fp64", 5000, **kw)
    assert n == 5000 and abs(tg - to) <= 1e-11 * to
    err = max_rel_elementwise(Wg, Wo, 4, 1e-2)
    assert np.all(err < 1e-10), err


@pytest.mark.parametrize("precision", ["fp32", "fp32_acc64"])
def test_shock_bl_fp32_forms_meet_the_l1_target_after_5000_steps(shock_bl_oracle, precision):
    spec, kw, Wo, _ = shock_bl_oracle
    Wg, _, n = gpu_run(spec, precision, 5000, **kw)
    l1 = l1_rho_rel(Wg, Wo, 4)
    assert n == 5000 and l1 < 1e-5, l1
