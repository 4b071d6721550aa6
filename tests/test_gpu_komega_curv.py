"""Parity of the CUDA k-omega transport on body-fitted grids (GKS_TURB_KOMEGA_TRANSPORT with
gks_set_nodes: the flow step in each face's frame, then rho k and rho omega advanced with the face
mass fluxes) with the oracle's curvilinear transport."""
import numpy as np
import pytest

import oracle
from paper_1302_2132_gb300 import inputs

pytestmark = pytest.mark.gpu

GAMMA = 1.4
TRANSPORT = 4


def wavy(n0, n1, seed):
    nodes = inputs.wavy_nodes(n0, n1, amp=0.04, shear=0.05)
    pts = inputs.cell_points(nodes)
    prim = inputs.smooth_state_at(pts, seed=seed, amp=0.15)
    k, om = inputs.positive_fields_at(pts, seed=seed + 1)
    return dict(n=(n0, n1), bc=[[0, 0], [0, 0]], bc_prim=None, nodes=nodes, prim=prim, k=k.ravel(), om=om.ravel(),
                mu=1e-3, T_wall=1.0, wake_cut=0, C_a=0.2)


def corner(nx, ny):
    sp = inputs.compression_corner(nx, ny, alpha_deg=24.0)
    return dict(n=(nx, ny), bc=sp["bc"], bc_prim=sp["bc_prim"], nodes=sp["nodes"], prim=sp["prim"], k=sp["f1"].ravel(),
                om=sp["f2"].ravel(), mu=sp["mu"], T_wall=sp["T_wall"], wake_cut=0, C_a=0.5)


def cgrid():
    sp = inputs.naca0012_case(16, 64, 24, mach=0.8, alpha_deg=2.26, Re=2e4)
    k, om = inputs.positive_fields_at(inputs.cell_points(sp["nodes"]), seed=9)
    return dict(n=sp["n"], bc=sp["bc"], bc_prim=sp["bc_prim"], nodes=sp["nodes"], prim=sp["prim"], k=k.ravel(),
                om=om.ravel(), mu=sp["mu"], T_wall=sp["T_wall"], wake_cut=sp["wake_cut"], C_a=0.5)


def run_both(sp, nsteps, precision="fp64", expand="directional", cfl=0.5, recon="muscl2"):
    from paper_1302_2132_gb300 import gks
    n0, n1 = sp["n"]
    dx = [np.full(n0, 1.0 / n0), np.full(n1, 1.0 / n1)]
    s = gks.Solver(2, sp["n"], sp["bc"], dx=dx, bc_data=sp["bc_prim"], gamma=GAMMA, mu=sp["mu"], T_wall=sp["T_wall"],
                   turb_model=TRANSPORT, C_a=sp["C_a"], limiter="vanleer", expand=expand, precision=precision,
                   wake_cut=sp["wake_cut"], reconstruction=recon)
    s.set_nodes(sp["nodes"])
    c = oracle.Case(2, sp["n"], dx, sp["bc"], gamma=GAMMA, mu=sp["mu"], T_wall=sp["T_wall"],
                    turb_model=oracle.TURB_KOMEGA, multid=int(expand == "multid"), C_a=sp["C_a"],
                    limiter=oracle.LIM_VANLEER, bc_prim=sp["bc_prim"], wake_cut=sp["wake_cut"],
                    recon={"muscl2": 0, "muscl3": 1, "weno5": 2}[recon])
    prim = np.asarray(sp["prim"], dtype=np.float64).ravel()
    s.set_state(prim, layout="soa_prim")
    s.set_turbulence(sp["k"], sp["om"])
    W = c.prim_to_cons(prim)
    nc = n0 * n1
    RK, RW = sp["k"] * W[:nc], sp["om"] * W[:nc]
    for _ in range(nsteps):
        dt = c.compute_dt_curv(sp["nodes"], W, cfl)
        s.step(nsteps=1, dt=dt)
        W, RK, RW, st = c.step_komega_curv(sp["nodes"], W, RK, RW, dt, nthreads=8)
        assert st == 0
    kg, wg = s.get_turbulence()
    Wg = s.get_state()
    s.close()
    return Wg, kg, wg, W, RK / W[:nc], RW / W[:nc]


def relmax(a, b):
    return np.abs(a - b).max() / np.abs(b).max()


@pytest.mark.parametrize("name,expand", [("wavy", "directional"), ("wavy", "multid"), ("corner", "directional"),
                                         ("cgrid", "directional"), ("cgrid", "multid")])
def test_fp64_transport_on_body_fitted_grids_matches_oracle(name, expand):
    sp = {"wavy": lambda: wavy(40, 30, seed=3), "corner": lambda: corner(64, 40), "cgrid": cgrid}[name]()
    Wg, kg, wg, Wo, ko, wo = run_both(sp, 3, expand=expand)
    nc = ko.size
    for v in range(4):
        assert relmax(Wg[v * nc:(v + 1) * nc], Wo[v * nc:(v + 1) * nc]) < 1e-12
    assert relmax(kg, ko) < 1e-12 and relmax(wg, wo) < 1e-12
    assert relmax(ko, sp["k"]) > 1e-8  # the fields moved


def test_fp32_transport_on_a_skewed_grid_close_to_oracle():
    sp = wavy(64, 48, seed=21)
    Wg, kg, wg, Wo, ko, wo = run_both(sp, 30, precision="fp32")
    l1 = lambda a, b: np.abs(a - b).sum() / np.abs(b).sum()
    assert l1(Wg[:ko.size], Wo[:ko.size]) < 1e-5
    assert l1(kg, ko) < 1e-5 and l1(wg, wo) < 1e-5


def naca_fine():
    """The 608 x 160 NACA 0012 C-grid of the paper's fine aerofoil grid size, as benchmarked."""
    sp = inputs.naca0012_case(112, 384, 160, mach=0.8, alpha_deg=2.26, Re=9.0e6, dy1=2e-4, ratio=1.05, R=10.0,
                              x_out=10.0)
    return dict(n=sp["n"], bc=sp["bc"], bc_prim=sp["bc_prim"], nodes=sp["nodes"], prim=sp["prim"],
                k=np.asarray(sp["f1"], dtype=np.float64).ravel(), om=np.asarray(sp["f2"], dtype=np.float64).ravel(),
                mu=sp["mu"], T_wall=sp["T_wall"], wake_cut=sp["wake_cut"], C_a=0.5)


def test_full_size_c_grid_transport_matches_oracle():
    """The benchmarked configuration (608 x 160 C-grid, k and omega from free-stream values): FP64
    parity over two steps and the FP32 form, in the autotuned launch configuration, within 1e-5
    (L1 of rho, k, omega) over ten steps."""
    sp = naca_fine()
    Wg, kg, wg, Wo, ko, wo = run_both(sp, 2)
    nc = ko.size
    for v in range(4):
        assert relmax(Wg[v * nc:(v + 1) * nc], Wo[v * nc:(v + 1) * nc]) < 1e-12
    assert relmax(kg, ko) < 1e-12 and relmax(wg, wo) < 1e-12
    Wg, kg, wg, Wo, ko, wo = run_both(sp, 10, precision="fp32")
    l1 = lambda a, b: np.abs(a - b).sum() / np.abs(b).sum()
    assert l1(Wg[:nc], Wo[:nc]) < 1e-5 and l1(kg, ko) < 1e-5 and l1(wg, wo) < 1e-5


@pytest.mark.parametrize("recon", ["muscl3", "weno5"])
def test_transport_with_higher_order_flow_matches_oracle(recon):
    """The step and transport kernels one after the other (the transport is fused into the MUSCL-2
    step only): WENO-5 / MUSCL-3 flow with transported k, omega on the C-grid, FP64."""
    sp = cgrid()
    Wg, kg, wg, Wo, ko, wo = run_both(sp, 3, recon=recon)
    nc = ko.size
    for v in range(4):
        assert relmax(Wg[v * nc:(v + 1) * nc], Wo[v * nc:(v + 1) * nc]) < 1e-12
    assert relmax(kg, ko) < 1e-12 and relmax(wg, wo) < 1e-12


def test_transport_with_double_state_close_to_oracle():
    """FP32 flux with an IEEE double state (separate transport kernel) on a skewed grid."""
    sp = wavy(64, 48, seed=23)
    Wg, kg, wg, Wo, ko, wo = run_both(sp, 20, precision="fp32_acc64")
    l1 = lambda a, b: np.abs(a - b).sum() / np.abs(b).sum()
    assert l1(Wg[:ko.size], Wo[:ko.size]) < 1e-5
    assert l1(kg, ko) < 1e-5 and l1(wg, wo) < 1e-5


@pytest.mark.parametrize("variant", ["0", "2"])
def test_fused_transport_tile_shapes_match_oracle(monkeypatch, variant):
    monkeypatch.setenv("GKS_TILE_VARIANT", variant)
    sp = corner(70, 37)
    Wg, kg, wg, Wo, ko, wo = run_both(sp, 3, expand="multid")
    nc = ko.size
    for v in range(4):
        assert relmax(Wg[v * nc:(v + 1) * nc], Wo[v * nc:(v + 1) * nc]) < 1e-12
    assert relmax(kg, ko) < 1e-12 and relmax(wg, wo) < 1e-12
