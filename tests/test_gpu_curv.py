"""Parity of the CUDA step on body-fitted 2D grids (gks_set_nodes: directional expansion in each
face's frame, the grids of the paper's channel and aerofoil cases, Section 5 Table 2) against the
oracle's curvilinear step."""
import numpy as np
import pytest

from paper_1302_2132_gb300 import inputs
from tests.cases import gpu_solver, max_rel_elementwise, oracle_case

pytestmark = pytest.mark.gpu


def wavy_spec(n0, n1, seed, bc=0, amp=0.04, shear=0.05):
    nodes = inputs.wavy_nodes(n0, n1, amp=amp, shear=shear)
    pts = inputs.cell_points(nodes)
    prim = inputs.smooth_state_at(pts, seed=seed, amp=0.15)
    f1, f2 = inputs.positive_fields_at(pts, seed=seed + 1)
    return dict(dim=2, n=(n0, n1), dx=[np.full(n0, 1.0 / n0), np.full(n1, 1.0 / n1)], bc=[[bc, bc], [bc, bc]],
                prim=prim, f1=f1, f2=f2, nodes=nodes)


def corner_spec(nx, ny, alpha=24.0):
    spec = inputs.compression_corner(nx, ny, alpha_deg=alpha)
    spec["dx"] = [np.full(nx, 1.0 / nx), np.full(ny, 1.0 / ny)]  # unused on a curvilinear grid
    return spec


def curv_both(spec, nsteps, turb_model=0, precision="fp64", cfl=0.5, C_a=0.0, mu=None, check_dt=True, multid=0):
    mu = spec.get("mu", 1e-5) if mu is None else mu
    s = gpu_solver(spec, turb_model=turb_model, multid=multid, precision=precision, C_a=C_a, mu=mu)
    c = oracle_case(spec, turb_model=turb_model, multid=multid, C_a=C_a, mu=mu)
    s.set_nodes(spec["nodes"])
    prim = np.asarray(spec["prim"], dtype=np.float64).ravel()
    s.set_state(prim, layout="soa_prim")
    f1 = np.asarray(spec["f1"], dtype=np.float64).ravel()
    f2 = np.asarray(spec["f2"], dtype=np.float64).ravel()
    if turb_model:
        s.set_turbulence(f1, None if turb_model == 1 else f2)
    W = c.prim_to_cons(prim)
    for _ in range(nsteps):
        dt_o = c.compute_dt_curv(spec["nodes"], W, cfl)
        if check_dt:
            dt_g = s.compute_dt(cfl)
            assert abs(dt_g - dt_o) <= 1e-14 * dt_o
        s.step(nsteps=1, dt=dt_o)
        W, st = c.step_curv(spec["nodes"], W, dt_o, f1=f1 if turb_model else None,
                            f2=f2 if turb_model > 1 else None, nthreads=8)
        assert st == 0
    return s, s.get_state(), W


def cases():
    return {
        "wavy_periodic_keps": (wavy_spec(40, 30, seed=3), dict(turb_model=2, C_a=0.2), 3),
        "wavy_transmissive_komega": (wavy_spec(37, 29, seed=5, bc=1), dict(turb_model=3), 3),
        "wavy_periodic_mut": (wavy_spec(33, 20, seed=7), dict(turb_model=1), 2),
        "wavy_periodic_laminar": (wavy_spec(24, 24, seed=9), dict(turb_model=0, C_a=0.5), 3),
        "corner_komega": (corner_spec(64, 40), dict(turb_model=3, C_a=0.5), 3),
        "corner_laminar": (corner_spec(50, 33, alpha=16.0), dict(turb_model=0, C_a=0.5), 3),
    }


@pytest.mark.parametrize("multid", [0, 1])
@pytest.mark.parametrize("name", list(cases()))
def test_fp64_curvilinear_step_matches_oracle(name, multid):
    spec, kw, steps = cases()[name]
    s, Wg, Wo = curv_both(spec, steps, multid=multid, **kw)
    assert np.all(max_rel_elementwise(Wg, Wo, 4, 1e-2) < 1e-12)
    s.close()


@pytest.mark.parametrize("multid", [0, 1])
@pytest.mark.parametrize("precision", ["fp32", "fp32_acc64"])
def test_fp32_curvilinear_close_to_oracle(precision, multid):
    spec = wavy_spec(64, 48, seed=21)
    s, Wg, Wo = curv_both(spec, 30, turb_model=2, precision=precision, check_dt=False, multid=multid)
    n = Wo.size // 4
    assert np.abs(Wg[:n] - Wo[:n]).sum() / np.abs(Wo[:n]).sum() < 1e-5
    s.close()


def test_fp32_corner_close_to_oracle():
    spec = corner_spec(96, 48)
    s, Wg, Wo = curv_both(spec, 20, turb_model=3, precision="fp32", C_a=0.5, check_dt=False)
    n = Wo.size // 4
    assert np.abs(Wg[:n] - Wo[:n]).sum() / np.abs(Wo[:n]).sum() < 1e-5
    s.close()


def test_full_size_corner_grid_matches_oracle():
    """The 528 x 136 compression-corner grid (the fine grid of the paper's corner cases) at 24
    degrees with k-omega: FP64 two steps element by element, FP32 ten steps in L1."""
    spec = corner_spec(528, 136)
    s, Wg, Wo = curv_both(spec, 2, turb_model=3, C_a=0.5)
    assert np.all(max_rel_elementwise(Wg, Wo, 4, 1e-2) < 1e-12)
    s.close()
    s, Wg, Wo = curv_both(spec, 10, turb_model=3, C_a=0.5, precision="fp32", check_dt=False)
    n = Wo.size // 4
    assert np.abs(Wg[:n] - Wo[:n]).sum() / np.abs(Wo[:n]).sum() < 1e-5
    s.close()


def test_free_stream_is_preserved_on_the_device():
    spec = wavy_spec(45, 31, seed=1, amp=0.05, shear=0.06)
    spec["prim"] = np.zeros((4, 31, 45))
    spec["prim"][0], spec["prim"][1], spec["prim"][2], spec["prim"][3] = 1.1, 0.4, -0.25, 0.7
    s = gpu_solver(spec, turb_model=2, multid=0)
    s.set_nodes(spec["nodes"])
    s.set_state(spec["prim"].ravel(), layout="soa_prim")
    s.set_turbulence(spec["f1"].ravel(), spec["f2"].ravel())
    W0 = s.get_state()
    s.step(nsteps=60, cfl=0.6)
    assert np.abs(s.get_state() - W0).max() < 1e-13
    s.close()


def test_uniform_grid_tau_matches_the_rectilinear_solver():
    """Green-Gauss gradients on a uniform periodic grid are the central differences of the
    rectilinear path: the two handles give the same tau_t field."""
    spec = inputs.turbulence(32, 2, seed=2)
    h = spec["dx"][0][0]
    out = []
    for curv in (False, True):
        s = gpu_solver(spec, turb_model=2, multid=0)
        if curv:
            s.set_nodes(inputs.uniform_nodes(32, 32, 32 * h, 32 * h))
        s.set_state(spec["prim"].ravel(), layout="soa_prim")
        s.set_turbulence(spec["f1"].ravel(), spec["f2"].ravel())
        out.append(s.tau_turb())
        s.close()
    assert np.abs(out[1] - out[0]).max() <= 1e-13 * np.abs(out[0]).max()
    assert out[0].max() > 0


@pytest.mark.parametrize("turb_model", [0, 2, 3])
def test_rarefaction_on_body_fitted_grids_matches_oracle(turb_model):
    """The rarefaction diagnostic (Green-Gauss divergence) on a skewed periodic grid and on the
    corner grid with walls and Dirichlet sides, FP64, against the oracle."""
    for spec, mu in ((wavy_spec(40, 30, seed=5), 2e-3), (corner_spec(64, 40), None)):
        mu = spec["mu"] if mu is None else mu
        s = gpu_solver(spec, turb_model=turb_model, multid=0, mu=mu, C_a=0.5)
        c = oracle_case(spec, turb_model=turb_model, multid=0, mu=mu, C_a=0.5)
        s.set_nodes(spec["nodes"])
        prim = np.asarray(spec["prim"], dtype=np.float64).ravel()
        s.set_state(prim, layout="soa_prim")
        f1 = np.asarray(spec["f1"], dtype=np.float64).ravel()
        f2 = np.asarray(spec["f2"], dtype=np.float64).ravel()
        if turb_model:
            s.set_turbulence(f1, f2)
        eg = s.rarefaction()
        eo = c.rarefaction_curv(spec["nodes"], c.prim_to_cons(prim), f1 if turb_model else None,
                                f2 if turb_model else None)
        assert np.abs(eg - eo).max() <= 1e-12 * np.abs(eo).max()
        assert np.abs(eo).max() > 0
        s.close()


def test_graph_and_eager_curvilinear_steps_are_bitwise_equal():
    spec = corner_spec(80, 44)
    out = []
    for timing in (False, True):
        s = gpu_solver(spec, turb_model=3, multid=0, precision="fp32", C_a=0.5, mu=spec["mu"])
        s.set_nodes(spec["nodes"])
        s.set_state(spec["prim"].ravel(), layout="soa_prim")
        s.set_turbulence(spec["f1"].ravel(), spec["f2"].ravel())
        if timing:
            s.enable_timing(True)
        s.step(nsteps=100, cfl=0.5)
        out.append(s.get_state())
        s.close()
    assert np.array_equal(out[0], out[1])


def test_residual_and_time_end_on_a_curvilinear_grid():
    """t_end stops the march exactly; the residual total is sum(area * W), conserved on a periodic grid."""
    spec = wavy_spec(30, 22, seed=13)
    s = gpu_solver(spec, turb_model=0, multid=0)
    s.set_nodes(spec["nodes"])
    s.set_state(spec["prim"].ravel(), layout="soa_prim")
    s.step(nsteps=1, cfl=0.5)
    _, _, tot0 = s.residual()
    s.step(nsteps=500, cfl=0.5, t_end=0.05)
    t, steps = s.time()
    assert abs(t - 0.05) < 1e-14
    s.step(nsteps=1, cfl=0.5)
    _, _, tot1 = s.residual()
    assert np.all(np.abs(tot1 - tot0) <= 1e-13 * np.abs(tot0).max())
    s.close()


def test_invalid_and_unsupported_grids_are_rejected():
    from paper_1302_2132_gb300 import gks
    spec = wavy_spec(12, 10, seed=1)
    bad = spec["nodes"].copy()
    bad[4, 5] = bad[4, 6] + np.array([0.05, 0.0])
    s = gpu_solver(spec, multid=0)
    with pytest.raises(gks.GksError):
        s.set_nodes(bad)
    s.set_nodes(spec["nodes"])  # the handle stays usable
    s.close()


@pytest.mark.parametrize("variant", ["0", "1", "2"])
def test_every_tile_shape_matches_oracle(monkeypatch, variant):
    """The three tile shapes of the curvilinear step (32 x 15, 16 x 7, 16 x 11; forced instead of
    autotuned) evaluate the same faces: FP64 parity on a corner grid that none of them divides."""
    monkeypatch.setenv("GKS_TILE_VARIANT", variant)
    spec = corner_spec(70, 37)
    s, Wg, Wo = curv_both(spec, 3, turb_model=3, C_a=0.5)
    assert s.tile_shape()[0] == int(variant)
    assert np.all(max_rel_elementwise(Wg, Wo, 4, 1e-2) < 1e-12)
    s.close()
