"""Parity of the CUDA MUSCL-3 and WENO-5 steps on body-fitted grids (index-space reconstruction along
the grid lines in each face's frame) with the oracle."""
import numpy as np
import pytest

import oracle
from paper_1302_2132_gb300 import inputs

pytestmark = pytest.mark.gpu

GAMMA = 1.4
RECON = {"muscl3": oracle.RECON_MUSCL3, "weno5": oracle.RECON_WENO5}


def wavy(n0, n1, seed):
    nodes = inputs.wavy_nodes(n0, n1, amp=0.04, shear=0.05)
    pts = inputs.cell_points(nodes)
    prim = inputs.smooth_state_at(pts, seed=seed, amp=0.15)
    f1, f2 = inputs.positive_fields_at(pts, seed=seed + 1)
    return dict(n=(n0, n1), bc=[[0, 0], [0, 0]], bc_prim=None, nodes=nodes, prim=prim, f1=f1.ravel(),
                f2=f2.ravel(), mu=1e-3, T_wall=1.0, wake_cut=0, turb=2)


def corner(nx, ny):
    sp = inputs.compression_corner(nx, ny, alpha_deg=24.0)
    sp.update(f1=np.ravel(sp["f1"]), f2=np.ravel(sp["f2"]), wake_cut=0, turb=3)
    return sp


def cgrid():
    sp = inputs.naca0012_case(16, 64, 24, mach=0.8, alpha_deg=2.26, Re=2e4)
    f1, f2 = inputs.positive_fields_at(inputs.cell_points(sp["nodes"]), seed=17)
    sp.update(f1=f1.ravel(), f2=f2.ravel(), turb=3)
    return sp


def run_both(sp, recon, nsteps, precision="fp64", expand="directional"):
    from paper_1302_2132_gb300 import gks
    n0, n1 = sp["n"]
    dx = [np.full(n0, 1.0 / n0), np.full(n1, 1.0 / n1)]
    s = gks.Solver(2, sp["n"], sp["bc"], dx=dx, bc_data=sp["bc_prim"], gamma=GAMMA, mu=sp["mu"], T_wall=sp["T_wall"],
                   turb_model=sp["turb"], C_a=0.5, limiter="vanleer", expand=expand, precision=precision,
                   reconstruction=recon, wake_cut=sp["wake_cut"])
    s.set_nodes(sp["nodes"])
    c = oracle.Case(2, sp["n"], dx, sp["bc"], gamma=GAMMA, mu=sp["mu"], T_wall=sp["T_wall"], turb_model=sp["turb"],
                    multid=int(expand == "multid"), C_a=0.5, limiter=oracle.LIM_VANLEER, bc_prim=sp["bc_prim"],
                    wake_cut=sp["wake_cut"], recon=RECON[recon])
    prim = np.asarray(sp["prim"], dtype=np.float64).ravel()
    s.set_state(prim, layout="soa_prim")
    s.set_turbulence(sp["f1"], sp["f2"])
    W = c.prim_to_cons(prim)
    for _ in range(nsteps):
        dt = c.compute_dt_curv(sp["nodes"], W, 0.5)
        s.step(nsteps=1, dt=dt)
        W, st = c.step_curv(sp["nodes"], W, dt, f1=sp["f1"], f2=sp["f2"], nthreads=8)
        assert st == 0
    Wg = s.get_state()
    tile = s.tile_shape()
    s.close()
    return Wg, W, tile


def rel_per_var(a, b):
    a, b = a.reshape(4, -1), b.reshape(4, -1)
    return np.array([np.abs(a[v] - b[v]).max() / np.abs(b[v]).max() for v in range(4)])


@pytest.mark.parametrize("expand", ["directional", "multid"])
@pytest.mark.parametrize("recon", ["muscl3", "weno5"])
@pytest.mark.parametrize("name", ["wavy", "corner", "cgrid"])
def test_fp64_higher_order_on_body_fitted_grids_matches_oracle(name, recon, expand):
    sp = {"wavy": lambda: wavy(40, 30, seed=3), "corner": lambda: corner(70, 37), "cgrid": cgrid}[name]()
    Wg, Wo, _ = run_both(sp, recon, 3, expand=expand)
    assert np.all(rel_per_var(Wg, Wo) < 1e-12)


@pytest.mark.parametrize("variant", ["0", "2"])
@pytest.mark.parametrize("recon", ["muscl3", "weno5"])
def test_both_tile_shapes_match_oracle(monkeypatch, recon, variant):
    monkeypatch.setenv("GKS_TILE_VARIANT", variant)
    Wg, Wo, tile = run_both(corner(70, 37), recon, 2, expand="multid")
    assert tile[0] == int(variant)
    assert np.all(rel_per_var(Wg, Wo) < 1e-12)


@pytest.mark.parametrize("recon", ["muscl3", "weno5"])
def test_fp32_higher_order_close_to_oracle(recon):
    sp = wavy(64, 48, seed=21)
    Wg, Wo, _ = run_both(sp, recon, 20, precision="fp32", expand="multid")
    n = Wo.size // 4
    assert np.abs(Wg[:n] - Wo[:n]).sum() / np.abs(Wo[:n]).sum() < 1e-5
