"""Parity of the CUDA steady solver with k-omega transport (GKS_TURB_KOMEGA_TRANSPORT in
gks_steady_*: each cycle one diagonal-implicit k-omega update from the fine residual, then the flow
cycle) with the oracle's composed cycle."""
import numpy as np
import pytest

import oracle
from paper_1302_2132_gb300 import inputs

pytestmark = pytest.mark.gpu

GAMMA = 1.4


def corner(nx, ny):
    sp = inputs.compression_corner(nx, ny, alpha_deg=24.0)
    k, om = inputs.positive_fields_at(inputs.cell_points(sp["nodes"]), seed=13)
    sp["k"], sp["om"], sp["wake_cut"] = 0.05 * k.ravel(), om.ravel(), 0
    return sp


def cgrid(nw=16, ns=64, n1=24, Re=2e4, **kw):
    sp = inputs.naca0012_case(nw, ns, n1, mach=0.8, alpha_deg=2.26, Re=Re, **kw)
    sp["k"], sp["om"] = np.asarray(sp["f1"], dtype=np.float64).ravel(), np.asarray(sp["f2"], dtype=np.float64).ravel()
    return sp


def both(sp, levels, precision="fp64", expand="directional", recon="muscl2"):
    from paper_1302_2132_gb300 import gks
    n0, n1 = sp["n"]
    s = gks.SteadySolver(sp["n"], sp["bc"], sp["nodes"], levels=levels, bc_data=sp["bc_prim"], gamma=GAMMA,
                         mu=sp["mu"], T_wall=sp["T_wall"], turb_model="komega_transport", C_a=0.5, limiter="vanleer",
                         precision=precision, lusgs_tile=16, wake_cut=sp["wake_cut"], expand=expand,
                         reconstruction=recon)
    c = oracle.Case(2, sp["n"], [np.ones(n0), np.ones(n1)], sp["bc"], gamma=GAMMA, mu=sp["mu"], T_wall=sp["T_wall"],
                    turb_model=oracle.TURB_KOMEGA, multid=int(expand == "multid"), C_a=0.5,
                    limiter=oracle.LIM_VANLEER, bc_prim=sp["bc_prim"], wake_cut=sp["wake_cut"],
                    recon={"muscl2": 0, "muscl3": 1, "weno5": 2}[recon])
    W = c.prim_to_cons(np.asarray(sp["prim"], dtype=np.float64).ravel())
    s.set_state(W)
    s.set_turbulence(sp["k"], sp["om"])
    return s, c, W


def oracle_cycles(c, sp, W, levels, cfls, cfl_flux=0.5):
    n = W.size // 4
    RK, RW = sp["k"] * W[:n], sp["om"] * W[:n]
    res = []
    for cfl in cfls:
        W, RK, RW, r, st = c.steady_cycle_komega(sp["nodes"], W, RK, RW, cfl, cfl_flux=cfl_flux, levels=levels,
                                                 tiles=(16, 16), nthreads=8)
        assert st == 0
        res.append(r)
    return W, RK / W[:n], RW / W[:n], np.array(res)


def rel_per_var(a, b, nv=4):
    a, b = a.reshape(nv, -1), b.reshape(nv, -1)
    return np.array([np.abs(a[v] - b[v]).max() / np.abs(b[v]).max() for v in range(nv)])


@pytest.mark.parametrize("name,expand,recon", [("corner", "directional", "muscl2"), ("cgrid", "directional", "muscl2"),
                                               ("cgrid", "multid", "muscl2"), ("cgrid", "multid", "weno5")])
def test_fp64_cycles_with_transport_match_oracle(name, expand, recon):
    sp = corner(64, 32) if name == "corner" else cgrid()
    levels = 3
    s, c, W = both(sp, levels, expand=expand, recon=recon)
    cfls = [1.0, 1.0, 3.0]
    res_g = np.concatenate([s.cycles(2, cfl=1.0), s.cycles(1, cfl=3.0)])
    Wo, ko, wo, res_o = oracle_cycles(c, sp, W, levels, cfls)
    kg, wg = s.get_turbulence()
    assert np.allclose(res_g, res_o, rtol=1e-11, atol=0)
    assert np.all(rel_per_var(s.get_state(), Wo) < 1e-11)
    assert np.abs(kg - ko).max() < 1e-11 * np.abs(ko).max()
    assert np.abs(wg - wo).max() < 1e-11 * np.abs(wo).max()
    assert np.abs(ko - sp["k"]).max() > 1e-6 * np.abs(ko).max()  # the fields moved
    s.close()


def test_fp32_cycles_with_transport_close_to_oracle():
    sp = corner(64, 32)
    s, c, W = both(sp, 3, precision="fp32")
    s.cycles(4, cfl=1.0)
    Wo, ko, wo, _ = oracle_cycles(c, sp, W, 3, [1.0] * 4)
    kg, wg = s.get_turbulence()
    n = ko.size
    l1 = lambda a, b: np.abs(a - b).sum() / np.abs(b).sum()
    assert l1(s.get_state()[:n], Wo[:n]) < 1e-5
    assert l1(kg, ko) < 1e-4 and l1(wg, wo) < 1e-4
    s.close()


def test_full_size_c_grid_cycles_with_transport_match_oracle():
    """The 608 x 160 NACA 0012 C-grid of the steady bench (4 levels, 16 x 16 LU-SGS tiles, k and
    omega from free-stream values): two FP64 cycles element by element."""
    sp = cgrid(112, 384, 160, Re=9.0e6, dy1=2e-4, ratio=1.05, R=10.0, x_out=10.0)
    s, c, W = both(sp, 4)
    res_g = s.cycles(2, cfl=1.0)
    Wo, ko, wo, res_o = oracle_cycles(c, sp, W, 4, [1.0, 1.0])
    kg, wg = s.get_turbulence()
    assert np.allclose(res_g, res_o, rtol=1e-11, atol=0)
    assert np.all(rel_per_var(s.get_state(), Wo) < 1e-11)
    assert np.abs(kg - ko).max() < 1e-11 * np.abs(ko).max()
    assert np.abs(wg - wo).max() < 1e-11 * np.abs(wo).max()
    s.close()


def test_transport_api_rules():
    from paper_1302_2132_gb300 import gks
    sp = corner(32, 16)
    s = gks.SteadySolver(sp["n"], sp["bc"], sp["nodes"], levels=2, bc_data=sp["bc_prim"], mu=sp["mu"],
                         T_wall=sp["T_wall"], turb_model="komega_transport", C_a=0.5)
    with pytest.raises(gks.GksError):  # the fields are stored with the state's density
        s.set_turbulence(sp["k"], sp["om"])
    s.set_state(np.asarray(sp["prim"], dtype=np.float64).ravel(), layout="soa_prim")
    with pytest.raises(gks.GksError):  # cycles need the fields
        s.cycles(1, cfl=1.0)
    s.set_turbulence(sp["k"], sp["om"])
    k, om = s.get_turbulence()
    assert np.allclose(k, sp["k"], rtol=1e-14) and np.allclose(om, sp["om"], rtol=1e-14)
    s.set_komega(sources=0)
    s.cycles(1, cfl=1.0)
    s.close()
    p = gks.SteadySolver(sp["n"], sp["bc"], sp["nodes"], levels=2, bc_data=sp["bc_prim"], mu=sp["mu"],
                         T_wall=sp["T_wall"], turb_model="komega", C_a=0.5)
    with pytest.raises(gks.GksError):
        p.get_turbulence()
    p.close()
