"""The rarefaction option on the GPU (gks_turb.rarefaction = GKS_RAR_TAUHAT: the degree of
rarefaction eps = tau/tauhat of Eqs. tautautilde, tautilde, rarefactionkepsilon and epsilonkomega in
place of tau/dt inside alpha and beta, reading G9) against the oracle's option: face fluxes, time
steps on rectilinear and body-fitted grids, and steady multigrid cycles (the paper's solver mode).
FP64 to 1e-12 (faces, per-face norm; states element by element with the 1% floor of each variable);
the FP32 forms within L1(rho) <= 1e-5 after the run."""
import numpy as np
import pytest

import oracle
from cases import gpu_solver, l1_rho_rel, max_rel_elementwise, oracle_case
from paper_1302_2132_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_1302_2132_gb300 import gks  # noqa: E402
from test_gpu_parity import GAMMA, random_faces  # noqa: E402


@pytest.mark.parametrize("D,expand", [(1, "directional"), (2, "directional"), (2, "multid"), (3, "multid"),
                                      (3, "directional")])
def test_face_flux_with_the_option_matches_oracle(D, expand):
    rng = np.random.default_rng(400 + 10 * D + len(expand))
    dt, mu, C_a = 1e-3, 2e-5, 0.4
    recs, faces = random_faces(rng, D, 300, dt)
    multid = int(expand == "multid")
    F, tau = gks.face_flux(D, torch.tensor(recs, device="cuda"), dt, gamma=GAMMA, mu=mu, C_a=C_a, precision="fp64",
                           expand=expand, rarefaction="tauhat")
    F32, _ = gks.face_flux(D, torch.tensor(recs, device="cuda"), dt, gamma=GAMMA, mu=mu, C_a=C_a, precision="fp32",
                           expand=expand, rarefaction="tauhat")
    F, F32 = F.cpu().numpy(), F32.cpu().numpy()
    worst, errs, moved = 0.0, [], 0
    for i, f in enumerate(faces):
        Fo = oracle.face_flux(D, GAMMA, mu, C_a, dt, f, multid=multid, rarefaction=1)
        F0 = oracle.face_flux(D, GAMMA, mu, C_a, dt, f, multid=multid)
        worst = max(worst, np.linalg.norm(F[i] - Fo) / np.linalg.norm(Fo))
        errs.append(np.linalg.norm(F32[i] - Fo) / np.linalg.norm(Fo))
        moved += np.linalg.norm(F0 - Fo) > 1e-8 * np.linalg.norm(Fo)
    assert worst < 1e-12, worst
    assert np.median(errs) < 5e-6 and max(errs) < 2e-4, (np.median(errs), max(errs))
    assert moved > 30  # the option changes the flux of these faces


def step_cases():
    sod = inputs.sod_1d(400)
    turb = inputs.turbulence(72, 2, seed=1302)
    sbl = inputs.shock_boundary_layer(70, 45)
    t3 = inputs.turbulence(20, 3, seed=2132)
    return {
        "sod_1d_400": (sod, dict(C_a=1.0, limiter=1, mu=1e-5, multid=0)),
        "turb_2d_72_keps_multid": (turb, dict(turb_model=2, multid=1, mu=1e-5)),
        "shock_bl_70x45_komega": (sbl, dict(turb_model=3, multid=1, mu=sbl["mu"], C_a=0.5)),
        "turb_3d_20_keps": (t3, dict(turb_model=2, multid=1, mu=1e-5)),
    }


def run_steps(spec, kw, precision, nsteps, rar=1):
    s = gpu_solver(spec, precision=precision, rarefaction=rar, **kw)
    c = oracle_case(spec, rarefaction=rar, **kw)
    s.set_state(spec["prim"].ravel(), layout="soa_prim")
    f1 = None if spec.get("f1") is None else spec["f1"].ravel()
    f2 = None if spec.get("f2") is None else spec["f2"].ravel()
    if kw.get("turb_model", 0):
        s.set_turbulence(f1, f2)
    W = c.prim_to_cons(spec["prim"].ravel())
    for _ in range(nsteps):
        dt = c.compute_dt(W, 0.5)
        s.step(nsteps=1, dt=dt)
        W, st, _ = c.step(W, dt, f1=f1 if kw.get("turb_model", 0) else None,
                          f2=f2 if kw.get("turb_model", 0) else None, nthreads=8)
        assert st == 0
    Wg = s.get_state()
    s.close()
    return Wg, W, c.prim_to_cons(spec["prim"].ravel())


@pytest.mark.parametrize("name", list(step_cases()))
def test_steps_with_the_option_match_oracle(name):
    spec, kw = step_cases()[name]
    nv = spec["dim"] + 2
    Wg, Wo, W0 = run_steps(spec, kw, "fp64", 3)
    err = max_rel_elementwise(Wg, Wo, nv, 1e-2)
    assert np.all(err < 1e-12), err
    inc = max_rel_elementwise(Wg - W0, Wo - W0, nv, 1e-2)
    assert np.all(inc < 1e-9), inc
    # the option changes the step (eps = tau/tauhat differs from tau/dt)
    Wd, _, _ = run_steps(spec, kw, "fp64", 3, rar=0)
    assert np.max(max_rel_elementwise(Wg - W0, Wd - W0, nv, 1e-2)) > 1e-6


@pytest.mark.parametrize("precision", ["fp32", "fp32_acc64"])
@pytest.mark.parametrize("name", ["turb_2d_72_keps_multid", "shock_bl_70x45_komega", "turb_3d_20_keps"])
def test_fp32_forms_with_the_option_meet_the_l1_target(name, precision):
    spec, kw = step_cases()[name]
    Wg, Wo, _ = run_steps(spec, kw, precision, 20)
    l1 = l1_rho_rel(Wg, Wo, spec["dim"] + 2)
    assert l1 < 1e-5, l1


def corner_spec(nx, ny):
    spec = inputs.compression_corner(nx, ny, alpha_deg=24.0)
    spec["dx"] = [np.full(nx, 1.0 / nx), np.full(ny, 1.0 / ny)]
    return spec


@pytest.mark.parametrize("multid", [0, 1])
def test_body_fitted_steps_with_the_option_match_oracle(multid):
    spec = corner_spec(64, 40)
    kw = dict(turb_model=3, multid=multid, C_a=0.5, mu=spec["mu"])
    s = gpu_solver(spec, rarefaction=1, **kw)
    c = oracle_case(spec, rarefaction=1, **kw)
    s.set_nodes(spec["nodes"])
    s.set_state(spec["prim"].ravel(), layout="soa_prim")
    s.set_turbulence(spec["f1"].ravel(), spec["f2"].ravel())
    W = c.prim_to_cons(spec["prim"].ravel())
    for _ in range(3):
        dt = c.compute_dt_curv(spec["nodes"], W, 0.5)
        s.step(nsteps=1, dt=dt)
        W, st = c.step_curv(spec["nodes"], W, dt, f1=spec["f1"].ravel(), f2=spec["f2"].ravel(), nthreads=8)
        assert st == 0
    assert s.tile_shape()[0] == 2
    err = max_rel_elementwise(s.get_state(), W, 4, 1e-2)
    s.close()
    assert np.all(err < 1e-12), err


@pytest.mark.parametrize("levels", [1, 3])
def test_steady_cycles_with_the_option_match_oracle(levels):
    """The paper's solver mode: the residual of every level takes eps = tau/tauhat."""
    spec = inputs.compression_corner(64, 40, alpha_deg=10.0, dy1=0.01, ratio=1.0)
    ny, nx = 40, 64
    prim = np.zeros((4, ny, nx))
    prim[0], prim[1], prim[3] = 1.0, 2.85, 1 / GAMMA
    inflow = np.tile([1.0, 2.85, 0.0, 1 / GAMMA], (ny, 1))
    bc, bc_prim = [[3, 4], [2, 4]], [[inflow, None], [None, None]]
    s = gks.SteadySolver((nx, ny), bc, spec["nodes"], levels=levels, bc_data=bc_prim, gamma=GAMMA, mu=5e-3,
                         T_wall=spec["T_wall"], turb_model=3, C_a=0.5, limiter=0, precision="fp64", lusgs_tile=16,
                         rarefaction="tauhat")
    c = oracle.Case(2, (nx, ny), [np.full(nx, 1.0 / nx), np.full(ny, 1.0 / ny)], bc, gamma=GAMMA, mu=5e-3,
                    T_wall=spec["T_wall"], turb_model=3, multid=0, C_a=0.5, limiter=0, bc_prim=bc_prim, rarefaction=1)
    W = c.prim_to_cons(prim.ravel())
    s.set_state(W)
    f1, f2 = spec["f1"].ravel(), spec["f2"].ravel()
    s.set_turbulence(f1, f2)
    res_g = s.cycles(3, cfl=3.0, cfl_flux=0.5)
    Wo, res_o = W, []
    for _ in range(3):
        Wo, r, st = c.steady_cycle(spec["nodes"], Wo, 3.0, cfl_flux=0.5, levels=levels, tiles=(16, 16), f1=f1, f2=f2,
                                   nthreads=8)
        assert st == 0
        res_o.append(r)
    assert np.allclose(res_g, res_o, rtol=1e-11, atol=0)
    Wg = s.get_state()
    s.close()
    nc = W.size // 4
    for v in range(4):
        a, b = Wg[v * nc:(v + 1) * nc], Wo[v * nc:(v + 1) * nc]
        assert np.abs(a - b).max() < 1e-11 * np.abs(b).max()


def test_unbuilt_combinations_are_rejected():
    spec = inputs.turbulence(24, 2, seed=3)
    with pytest.raises(gks.GksError) as e:
        gpu_solver(spec, turb_model=2, recon=2, rarefaction=1)
    assert e.value.code == gks.EUNSUPPORTED
