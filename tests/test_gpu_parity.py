"""Parity of the CUDA path (through the C ABI) with the oracle.

Tolerances: the FP64 path matches the oracle to 1e-12 relative per step, element by element
(|a - b| <= 1e-12 max(|b|, 1e-2 max|b_v|) for every cell and variable v; the floor at 1% of the
variable's largest value keeps components that pass through zero, such as a momentum, at the scale
of their variable); interface fluxes to 1e-12 per face.  The FP32 forms are held to L1(rho) <= 1e-5
relative after a run, and their face fluxes to the single-precision accuracy stated in each test.
"""
import math

import numpy as np
import pytest

import oracle
from cases import gpu_solver, max_rel_elementwise, oracle_case, rel_err_per_var
from paper_1302_2132_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_1302_2132_gb300 import gks  # noqa: E402

GAMMA = 1.4


def cons(D, rho, U, p):
    U = np.asarray(U, dtype=float)
    return np.concatenate([[rho], rho * U, [p / (GAMMA - 1.0) + 0.5 * rho * np.dot(U, U)]])


def random_faces(rng, D, n, dt):
    """Random face records (normal frame) and matching oracle faces."""
    nv = D + 2
    L = gks.face_record_len(D)
    recs = np.zeros((n, L))
    faces = []
    for f in range(n):
        wl = cons(D, rng.uniform(0.3, 2.0), rng.uniform(-1.5, 1.5, D), rng.uniform(0.2, 2.0))
        if rng.random() < 0.3:
            wr = wl.copy()  # near-equal states
            wr[0] *= 1 + 1e-6 * rng.normal()
        else:
            wr = cons(D, rng.uniform(0.3, 2.0), rng.uniform(-1.5, 1.5, D), rng.uniform(0.2, 2.0))
        h = rng.uniform(0.002, 0.05)
        sl, sr = rng.normal(size=nv), rng.normal(size=nv)
        cl, cr = wl - 0.5 * h * sl, wr + 0.5 * h * sr
        tl, tr = rng.normal(size=(max(D - 1, 1), nv)), rng.normal(size=(max(D - 1, 1), nv))
        tau_t = rng.choice([0.0, rng.uniform(0, 5) * dt, rng.uniform(0, 1e-3) * dt, rng.uniform(1, 100) * dt])
        parts = [wl, wr, cl, cr, sl, sr] + [tl[k] for k in range(D - 1)] + [tr[k] for k in range(D - 1)]
        recs[f, : 6 * nv + 2 * (D - 1) * nv] = np.concatenate(parts)
        recs[f, -3:] = (0.5 * h, 0.5 * h, tau_t)
        faces.append(oracle.make_face(D, wl, wr, cl, cr, sl, sr, tl[: D - 1], tr[: D - 1], 0.5 * h, 0.5 * h, tau_t))
    return recs, faces


@pytest.mark.parametrize("D,expand,abar", [(1, "directional", "timeint"), (2, "directional", "timeint"),
                                           (2, "multid", "timeint"), (2, "multid", "t0"), (3, "multid", "timeint"),
                                           (3, "directional", "timeint")])
def test_face_flux_fp64_matches_oracle(D, expand, abar):
    rng = np.random.default_rng(1000 + 10 * D + len(expand))
    dt, mu, C_a = 1e-3, 2e-5, 0.4
    recs, faces = random_faces(rng, D, 300, dt)
    F, tau = gks.face_flux(D, torch.tensor(recs, device="cuda"), dt, gamma=GAMMA, mu=mu, C_a=C_a, precision="fp64",
                           expand=expand, abar_mode=abar)
    F, tau = F.cpu().numpy(), tau.cpu().numpy()
    worst = 0.0
    for i, f in enumerate(faces):
        Fo, dg = oracle.face_flux(D, GAMMA, mu, C_a, dt, f, multid=int(expand == "multid"),
                                  abar_mode=int(abar == "t0"), diag=True)
        e = np.linalg.norm(F[i] - Fo) / np.linalg.norm(Fo)
        worst = max(worst, e)
        assert abs(tau[i] - dg.tau) <= 1e-13 * dg.tau
    assert worst < 1e-12, worst


@pytest.mark.parametrize("D", [1, 2, 3])
def test_face_flux_fp32_close_to_oracle(D):
    rng = np.random.default_rng(2000 + D)
    dt = 1e-3
    recs, faces = random_faces(rng, D, 200, dt)
    F, _ = gks.face_flux(D, torch.tensor(recs, device="cuda"), dt, mu=2e-5, C_a=0.4, precision="fp32")
    F = F.cpu().numpy()
    errs = []
    for i, f in enumerate(faces):
        Fo = oracle.face_flux(D, GAMMA, 2e-5, 0.4, dt, f)
        errs.append(np.linalg.norm(F[i] - Fo) / np.linalg.norm(Fo))
    assert np.median(errs) < 2e-6 and max(errs) < 1e-4, (np.median(errs), max(errs))


@pytest.mark.parametrize("D", [1, 2, 3])
@pytest.mark.parametrize("x", [1e-6, 1e-4, 1e-2, 80.0, 300.0])
def test_face_flux_fp32_at_extreme_dt_over_tau(D, x):
    """x = dt/tau at the ends of its range: near-free transport (tau >> dt, the series branch of the
    time coefficients in single precision) and near-equilibrium (tau << dt).  mu = C_a = 0, so tau is
    the face's turbulent relaxation time and x = dt/tau_t exactly."""
    rng = np.random.default_rng(3000 + D + int(1e3 * math.log10(x) + 7000))
    dt = 1e-3
    recs, faces = random_faces(rng, D, 200, dt)
    recs[:, -1] = dt / x
    F, tau = gks.face_flux(D, torch.tensor(recs, device="cuda"), dt, mu=0.0, C_a=0.0, precision="fp32")
    F, tau = F.cpu().numpy(), tau.cpu().numpy()
    errs = []
    for i, f in enumerate(faces):
        f.tau_t = dt / x
        Fo, dg = oracle.face_flux(D, GAMMA, 0.0, 0.0, dt, f, diag=True)
        assert abs(dg.tau - dt / x) <= 1e-15 * dg.tau
        errs.append(np.linalg.norm(F[i] - Fo) / np.linalg.norm(Fo))
    errs = np.array(errs)
    print("D=%d x=%g: median %.2e max %.2e" % (D, x, np.median(errs), errs.max()))
    assert np.median(errs) < 5e-6 and errs.max() < 1e-4, (np.median(errs), errs.max())


def step_both(spec, nsteps=1, cfl=0.5, **kw):
    prec = kw.pop("precision", "fp64")
    s = gpu_solver(spec, precision=prec, **kw)
    c = oracle_case(spec, **kw)
    prim = spec["prim"].ravel()
    s.set_state(prim, layout="soa_prim")
    f1 = spec.get("f1")
    f2 = spec.get("f2")
    if kw.get("turb_model", 0):
        s.set_turbulence(f1.ravel(), None if f2 is None else f2.ravel())
    W = c.prim_to_cons(prim)
    for _ in range(nsteps):
        dt_g = s.compute_dt(cfl)
        dt_o = c.compute_dt(W, cfl)
        assert abs(dt_g - dt_o) <= 1e-14 * dt_o
        s.step(nsteps=1, dt=dt_g)
        W, st, res = c.step(W, dt_g, f1=None if f1 is None else f1.ravel(), f2=None if f2 is None else f2.ravel(),
                            nthreads=8)
        assert st == 0
    Wg = s.get_state()
    return s, c, Wg, W, res


def config_cases():
    sod = inputs.sod_1d(400)
    turb = inputs.turbulence(72, 2, seed=1302)
    turb["n"] = (72, 72)
    sbl = inputs.shock_boundary_layer(70, 45)
    t3 = inputs.turbulence(20, 3, seed=2132)
    quad = inputs.riemann_quadrant(50, seed=4000)
    return {
        "sod_1d_400": (sod, dict(C_a=1.0, limiter=1, mu=1e-5)),
        "turb_2d_72_keps_multid": (turb, dict(turb_model=2, multid=1, mu=1e-5)),
        "shock_bl_70x45_komega": (sbl, dict(turb_model=3, multid=1, mu=sbl["mu"], C_a=0.5)),
        "turb_3d_20_keps": (t3, dict(turb_model=2, multid=1, mu=1e-5)),
        "quadrant_50_directional_minmod": (quad, dict(multid=0, limiter=0, C_a=0.3, mu=1e-4)),
    }


@pytest.mark.parametrize("name", list(config_cases().keys()))
def test_one_step_fp64_matches_oracle(name):
    spec, kw = config_cases()[name]
    s, c, Wg, Wo, res = step_both(spec, nsteps=1, **kw)
    nv = spec["dim"] + 2
    err = max_rel_elementwise(Wg, Wo, nv, 1e-2)
    assert np.all(err < 1e-12), err
    # the increment itself agrees to a few digits fewer than the state (cancellation in W^1 - W^0)
    W0 = c.prim_to_cons(spec["prim"].ravel())
    inc = max_rel_elementwise(Wg - W0, Wo - W0, nv, 1e-2)
    assert np.all(inc < 1e-9), inc
    l2, linf, tot = s.residual()
    assert np.allclose(l2, res[0], rtol=1e-9, atol=1e-300)
    assert np.allclose(linf, res[1], rtol=1e-9, atol=1e-300)
    assert np.allclose(tot, res[2], rtol=1e-12, atol=1e-12 * np.abs(res[2]).max())
    s.close()


def test_sod_full_run_fp64_matches_oracle():
    spec = inputs.sod_1d(400)
    kw = dict(C_a=1.0, limiter=1, mu=1e-5)
    s = gpu_solver(spec, **kw)
    c = oracle_case(spec, **kw)
    s.set_state(spec["prim"].ravel(), layout="soa_prim")
    s.step(nsteps=100000, cfl=0.5, t_end=0.2)
    t, steps = s.time()
    W, to, so, st = c.run(c.prim_to_cons(spec["prim"].ravel()), 100000, cfl=0.5, t_end=0.2, nthreads=8)
    assert abs(t - 0.2) < 1e-14 and abs(to - 0.2) < 1e-14
    err = max_rel_elementwise(s.get_state(), W, 3, 1e-2)
    assert np.all(err < 1e-10), err
    s.close()


@pytest.mark.parametrize("name", ["turb_2d_72_keps_multid", "shock_bl_70x45_komega", "turb_3d_20_keps"])
def test_diagnostics_match_oracle(name):
    spec, kw = config_cases()[name]
    s = gpu_solver(spec, **kw)
    c = oracle_case(spec, **kw)
    s.set_state(spec["prim"].ravel(), layout="soa_prim")
    s.set_turbulence(spec["f1"].ravel(), spec["f2"].ravel())
    W = c.prim_to_cons(spec["prim"].ravel())
    tg, to = s.tau_turb(), c.tau_turb(W, spec["f1"].ravel(), spec["f2"].ravel())
    assert np.max(np.abs(tg - to) / np.maximum(np.abs(to), 1e-300)) < 1e-12
    eg, eo = s.rarefaction(), c.rarefaction(W, spec["f1"].ravel(), spec["f2"].ravel())
    assert np.linalg.norm(eg - eo) <= 1e-12 * np.linalg.norm(eo)
    s.close()


def test_fp32_forms_meet_l1_density_target():
    """2D decaying turbulence, 64^2, 40 steps: the FP32 forms stay within L1(rho) <= 1e-5 of the
    FP64 oracle."""
    spec = inputs.turbulence(64, 2, seed=1302)
    kw = dict(turb_model=2, multid=1, mu=1e-5)
    c = oracle_case(spec, **kw)
    W0 = c.prim_to_cons(spec["prim"].ravel())
    Wo, t, n, st = c.run(W0, 40, cfl=0.5, f1=spec["f1"].ravel(), f2=spec["f2"].ravel(), nthreads=8)
    for prec in ("fp32", "fp32_acc64"):
        s = gpu_solver(spec, precision=prec, **kw)
        s.set_state(spec["prim"].ravel(), layout="soa_prim")
        s.set_turbulence(spec["f1"].ravel(), spec["f2"].ravel())
        s.step(nsteps=40, cfl=0.5)
        Wg = s.get_state().reshape(4, -1)
        l1 = np.sum(np.abs(Wg[0] - Wo.reshape(4, -1)[0])) / np.sum(np.abs(Wo.reshape(4, -1)[0]))
        assert l1 < 1e-5, (prec, l1)
        s.close()


def test_checkpoint_resume_is_bitwise():
    spec = inputs.turbulence(48, 2, seed=3)
    kw = dict(turb_model=2, multid=1, mu=1e-5)
    a = gpu_solver(spec, **kw)
    a.set_state(spec["prim"].ravel(), layout="soa_prim")
    a.set_turbulence(spec["f1"].ravel(), spec["f2"].ravel())
    a.step(nsteps=60, cfl=0.5)
    ta, _ = a.time()
    full = a.get_state()
    b = gpu_solver(spec, **kw)
    b.set_state(spec["prim"].ravel(), layout="soa_prim")
    b.set_turbulence(spec["f1"].ravel(), spec["f2"].ravel())
    b.step(nsteps=25, cfl=0.5)
    chk = b.get_state()
    tb, _ = b.time()
    b.close()
    r = gpu_solver(spec, **kw)
    r.set_state(chk)
    r.set_time(tb)
    r.set_turbulence(spec["f1"].ravel(), spec["f2"].ravel())
    r.step(nsteps=35, cfl=0.5)
    assert np.array_equal(r.get_state(), full)
    assert r.time()[0] == ta
    a.close()
    r.close()


def test_graph_and_eager_paths_agree_bitwise():
    spec = inputs.turbulence(40, 2, seed=5)
    kw = dict(turb_model=2, multid=1, mu=1e-5, precision="fp32")
    out = []
    for timing in (False, True):
        s = gpu_solver(spec, **kw)
        s.set_state(spec["prim"].ravel(), layout="soa_prim")
        s.set_turbulence(spec["f1"].ravel(), spec["f2"].ravel())
        s.enable_timing(timing)
        s.step(nsteps=110, cfl=0.5)
        out.append(s.get_state())
        if timing:
            ms, n = s.kernel_time()
            assert n == 110 and ms > 0
        s.close()
    assert np.array_equal(out[0], out[1])


def test_nonphysical_state_is_reported():
    spec = inputs.sod_1d(64)
    s = gpu_solver(spec, mu=1e-5)
    prim = spec["prim"].copy()
    prim[2, 30] = -1.0  # negative pressure
    s.set_state(prim.ravel(), layout="soa_prim")
    s.step(nsteps=1, dt=1e-4)
    with pytest.raises(gks.GksError) as e:
        s.residual()
    assert e.value.code == gks.ENONPHYS
    s.set_state(spec["prim"].ravel(), layout="soa_prim")  # clears the sticky status
    s.step(nsteps=1, dt=1e-4)
    s.residual()
    s.close()


def test_invalid_arguments_are_rejected():
    spec = inputs.sod_1d(16)
    with pytest.raises(gks.GksError) as e:
        gks.Solver(1, (1,), [["periodic", "periodic"]], dx=[np.ones(1)])
    assert e.value.code == gks.EINVAL
    with pytest.raises(gks.GksError):
        gks.Solver(1, (16,), [["periodic", "wall"]], dx=spec["dx"])
    with pytest.raises(gks.GksError):
        gks.Solver(2, (8, 8), [["dirichlet", "outflow"], ["periodic", "periodic"]], dx=[np.ones(8)] * 2)
    s = gpu_solver(spec)
    with pytest.raises(gks.GksError):
        s.step(nsteps=1)  # no state yet
    s.close()


def test_device_tensors_and_layouts_roundtrip():
    spec = inputs.turbulence(24, 3, seed=11)
    s = gpu_solver(spec, turb_model=2)
    prim = torch.tensor(spec["prim"].ravel(), device="cuda")
    s.set_state(prim, layout="soa_prim")
    back = torch.empty_like(prim)
    s.get_state(layout="soa_prim", out=back)
    assert torch.allclose(back, prim, rtol=1e-14, atol=1e-14)
    W = s.get_state()
    aos = s.get_state(layout="aos_cons")
    assert np.array_equal(aos.reshape(-1, 5).T.ravel(), W)
    s.set_state(aos, layout="aos_cons")
    assert np.array_equal(s.get_state(), W)
    s.close()


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_full_size_2d_turbulence_sampled_cells(prec):
    """Full-size 1024^2 decaying-turbulence step in the bench's launch configuration; sampled cells
    are recomputed by the oracle on a 9x9 crop around each cell with the same dt (the crop's own
    boundary cannot reach the centre cell in one step)."""
    spec = inputs.turbulence(1024, 2, seed=1302)
    kw = dict(turb_model=2, multid=1, mu=1e-5)
    s = gpu_solver(spec, precision=prec, **kw)
    s.set_state(spec["prim"].ravel(), layout="soa_prim")
    s.set_turbulence(spec["f1"].ravel(), spec["f2"].ravel())
    dt = s.compute_dt(0.5)
    s.step(nsteps=1, dt=dt)
    Wg = s.get_state().reshape(4, 1024, 1024)
    tot = s.residual()[2]
    s.close()
    rng = np.random.default_rng(0)
    h = 2 * math.pi / 1024
    prim = spec["prim"]
    errs = []
    for _ in range(24):
        j, i = rng.integers(0, 1024, 2)
        jj = (np.arange(j - 4, j + 5)) % 1024
        ii = (np.arange(i - 4, i + 5)) % 1024
        crop = dict(dim=2, n=(9, 9), dx=[np.full(9, h)] * 2, bc=[[1, 1], [1, 1]])
        c = oracle_case(crop, **kw)
        pc = prim[:, jj][:, :, ii]
        W0 = c.prim_to_cons(pc.ravel())
        f1 = spec["f1"][jj][:, ii].ravel()
        f2 = spec["f2"][jj][:, ii].ravel()
        Wo, st, _ = c.step(W0, dt, f1=f1, f2=f2)
        wo = Wo.reshape(4, 9, 9)[:, 4, 4]
        w0 = W0.reshape(4, 9, 9)[:, 4, 4]
        wg = Wg[:, j, i]
        errs.append(np.abs(wg - wo) / np.maximum(np.abs(wo - w0), 1e-300))
        if prec == "fp64":
            assert np.all(np.abs(wg - wo) <= 1e-12 * np.abs(wo) + 1e-15)
    errs = np.array(errs)
    # FP32 flux: the per-step increment is accurate to about 1e-4 relative
    assert np.median(errs) < (1e-9 if prec == "fp64" else 1e-3), np.median(errs)
    # conservation at full size: total of every variable is unchanged, up to the rounding of the
    # per-cell increments (double, or single precision for the FP32 flux)
    W0 = oracle_case(spec, **kw).prim_to_cons(spec["prim"].ravel()).reshape(4, -1).sum(axis=1) * h * h
    assert np.all(np.abs(tot - W0) <= (1e-11 if prec == "fp64" else 1e-9) * (np.abs(W0) + 1.0))


@pytest.mark.parametrize("precision", ["fp32", "fp32_acc64"])
def test_tile_variants_agree_and_autotuner_picks_one(monkeypatch, precision):
    """The nine 2D single-precision tile shapes (two of them evaluating two faces per thread with
    paired instructions) evaluate the same faces: their results agree to FP32 rounding (different
    compiled kernels), and the autotuner keeps one of them; for the float-pair and the double state."""
    spec = inputs.turbulence(100, 2, seed=8)
    kw = dict(turb_model=2, multid=1, mu=1e-5, precision=precision)
    out = []
    for v in ("0", "1", "2", "3", "4", "5", "6", "7", "8"):
        monkeypatch.setenv("GKS_TILE_VARIANT", v)
        s = gpu_solver(spec, **kw)
        s.set_state(spec["prim"].ravel(), layout="soa_prim")
        s.set_turbulence(spec["f1"].ravel(), spec["f2"].ravel())
        s.step(nsteps=30, cfl=0.5)
        assert s.tile_shape()[0] == int(v)
        out.append(s.get_state())
        s.close()
    for W in out[1:]:
        assert np.all(rel_err_per_var(W, out[0], 4) < 1e-6)
    monkeypatch.delenv("GKS_TILE_VARIANT")
    s = gpu_solver(spec, **kw)
    s.set_state(spec["prim"].ravel(), layout="soa_prim")
    s.set_turbulence(spec["f1"].ravel(), spec["f2"].ravel())
    s.step(nsteps=30, cfl=0.5)
    v = s.tile_shape()
    assert v[0] in range(9) and v[1] * v[2] in (480, 448, 992, 864, 576, 1728, 672)
    assert np.all(rel_err_per_var(s.get_state(), out[0], 4) < 1e-6)
    s.close()


@pytest.mark.parametrize("variant", ["0", "1", "2"])
def test_1d_tile_variants_match_oracle(monkeypatch, variant):
    """Each 1D tile shape (256, 31 and 63 cells per CTA) gives the FP64 Sod step of the oracle."""
    monkeypatch.setenv("GKS_TILE_VARIANT", variant)
    spec = inputs.sod_1d(400)
    s, c, Wg, Wo, res = step_both(spec, nsteps=3, C_a=1.0, limiter=1, mu=1e-5)
    assert s.tile_shape()[:2] == (int(variant), {"0": 256, "1": 31, "2": 63}[variant])
    assert np.all(max_rel_elementwise(Wg, Wo, 3, 1e-2) < 1e-12)
    s.close()


def test_3d_tile_variants_agree(monkeypatch):
    """The four 3D FP32 tile shapes (16x8x4 without the slope table, 16x8x2 and 8x8x4 with it, and
    16x8x2 with two faces per thread) evaluate the same faces: their results agree to FP32 rounding."""
    spec = inputs.turbulence(20, 3, seed=17)
    kw = dict(turb_model=2, multid=1, mu=1e-5, precision="fp32")
    out = []
    for v in ("0", "1", "2", "3"):
        monkeypatch.setenv("GKS_TILE_VARIANT", v)
        s = gpu_solver(spec, **kw)
        s.set_state(spec["prim"].ravel(), layout="soa_prim")
        s.set_turbulence(spec["f1"].ravel(), spec["f2"].ravel())
        s.step(nsteps=10, cfl=0.5)
        assert s.tile_shape()[0] == int(v)
        out.append(s.get_state())
        s.close()
    for W in out[1:]:
        assert np.all(rel_err_per_var(W, out[0], 5) < 1e-6)


def test_steps_continue_after_t_end():
    """A run stopped by t_end (the last steps carry the state over) continues with the CFL time step
    of the stored state: the next step equals the oracle's step from that state."""
    spec = inputs.turbulence(40, 2, seed=17)
    s = gpu_solver(spec, turb_model=2, mu=1e-5)
    c = oracle_case(spec, turb_model=2, mu=1e-5)
    s.set_state(spec["prim"].ravel(), layout="soa_prim")
    s.set_turbulence(spec["f1"].ravel(), spec["f2"].ravel())
    s.step(nsteps=50, cfl=0.5, t_end=0.01)
    t, _ = s.time()
    assert abs(t - 0.01) < 1e-15
    W = s.get_state()
    dt_o = c.compute_dt(W, 0.5)
    assert abs(s.compute_dt(0.5) - dt_o) <= 1e-14 * dt_o
    s.step(nsteps=1, cfl=0.5)
    Wo, st, _ = c.step(W, dt_o, f1=spec["f1"].ravel(), f2=spec["f2"].ravel(), nthreads=8)
    assert st == 0
    assert np.all(max_rel_elementwise(s.get_state(), Wo, 4, 1e-2) < 1e-12)
    s.close()
