"""Parity of the CUDA steady-state solver (gks_steady_*: local time stepping, LU-SGS smoothing on
32 x 32 or 16 x 16 tiles, FAS multigrid; the paper's solver mode, Section 4) with the oracle."""
import numpy as np
import pytest

import oracle
from paper_1302_2132_gb300 import inputs

pytestmark = pytest.mark.gpu

GAMMA = 1.4


def wavy(n0, n1, seed, turb=0):
    nodes = inputs.wavy_nodes(n0, n1, amp=0.04, shear=0.05)
    pts = inputs.cell_points(nodes)
    prim = inputs.smooth_state_at(pts, seed=seed, amp=0.15)
    f1, f2 = inputs.positive_fields_at(pts, seed=seed + 1)
    return dict(n=(n0, n1), bc=[[0, 0], [0, 0]], bc_prim=None, nodes=nodes, prim=prim, f1=f1.ravel(),
                f2=f2.ravel(), mu=1e-3, T_wall=1.0, turb=turb, C_a=0.2)


def corner(nx, ny, mu=5e-3, turb=0, laminar_start=True):
    spec = inputs.compression_corner(nx, ny, alpha_deg=10.0, dy1=0.01, ratio=1.0)
    prim = np.zeros((4, ny, nx))
    prim[0], prim[1], prim[3] = 1.0, 2.85, 1 / GAMMA
    if not laminar_start:
        prim = spec["prim"]
    inflow = np.tile([1.0, 2.85, 0.0, 1 / GAMMA], (ny, 1))
    return dict(n=(nx, ny), bc=[[3, 4], [2, 4]], bc_prim=[[inflow, None], [None, None]], nodes=spec["nodes"],
                prim=prim, f1=spec["f1"].ravel(), f2=spec["f2"].ravel(), mu=mu, T_wall=spec["T_wall"], turb=turb,
                C_a=0.5)


def both(sp, levels, precision="fp64", limiter=0, tile=32):
    from paper_1302_2132_gb300 import gks
    n0, n1 = sp["n"]
    s = gks.SteadySolver(sp["n"], sp["bc"], sp["nodes"], levels=levels, bc_data=sp["bc_prim"], gamma=GAMMA,
                         mu=sp["mu"], T_wall=sp["T_wall"], turb_model=sp["turb"], C_a=sp["C_a"], limiter=limiter,
                         precision=precision, lusgs_tile=tile)
    c = oracle.Case(2, sp["n"], [np.full(n0, 1.0 / n0), np.full(n1, 1.0 / n1)], sp["bc"], gamma=GAMMA, mu=sp["mu"],
                    T_wall=sp["T_wall"], turb_model=sp["turb"], multid=0, C_a=sp["C_a"], limiter=limiter,
                    bc_prim=sp["bc_prim"])
    W = c.prim_to_cons(np.asarray(sp["prim"], dtype=np.float64).ravel())
    s.set_state(W)
    f1 = f2 = None
    if sp["turb"]:
        f1 = sp["f1"]
        f2 = sp["f2"] if sp["turb"] > 1 else None
        s.set_turbulence(f1, f2)
    return s, c, W, f1, f2


def rel(a, b):
    return np.abs(a - b).max() / np.abs(b).max()


@pytest.mark.parametrize("name,first_order", [("wavy_keps", False), ("wavy_keps", True), ("corner_komega", False),
                                              ("corner_laminar", True)])
def test_residual_matches_oracle(name, first_order):
    sp = {"wavy_keps": lambda: wavy(40, 30, seed=3, turb=2), "corner_komega": lambda: corner(72, 40, turb=3),
          "corner_laminar": lambda: corner(50, 34)}[name]()
    s, c, W, f1, f2 = both(sp, levels=1)
    dt_g, R_g = s.residual(cfl_flux=0.6, first_order=first_order)
    dt_o, R_o = c.steady_residual(sp["nodes"], W, cfl_flux=0.6, first_order=first_order, f1=f1, f2=f2, nthreads=8)
    assert rel(dt_g, dt_o) < 1e-13
    nc = W.size // 4
    for v in range(4):
        assert np.abs(R_g[v * nc:(v + 1) * nc] - R_o[v * nc:(v + 1) * nc]).max() < 1e-12 * np.abs(R_o[v * nc:(v + 1) * nc]).max() + 1e-15
    s.close()


@pytest.mark.parametrize("name,levels,cycles,tile", [("wavy_keps", 1, 2, 32), ("corner_komega", 1, 2, 32),
                                                     ("corner_laminar", 3, 3, 32), ("corner_komega", 4, 2, 32),
                                                     ("wavy_keps", 1, 2, 16), ("corner_komega", 3, 2, 16)])
def test_cycles_match_oracle(name, levels, cycles, tile):
    """LU-SGS on 32 x 32 and 16 x 16 tiles (several tiles and ragged edges) and the multigrid
    transfers: the state after a few cycles equals the oracle's."""
    sp = {"wavy_keps": lambda: wavy(48, 40, seed=5, turb=2), "corner_komega": lambda: corner(72, 40, turb=3),
          "corner_laminar": lambda: corner(64, 40)}[name]()
    s, c, W, f1, f2 = both(sp, levels=levels, tile=tile)
    res_g = s.cycles(cycles, cfl=3.0, cfl_flux=0.5)
    Wo = W
    res_o = []
    for _ in range(cycles):
        Wo, r, st = c.steady_cycle(sp["nodes"], Wo, 3.0, cfl_flux=0.5, levels=levels, tiles=(tile, tile), f1=f1,
                                   f2=f2, nthreads=8)
        assert st == 0
        res_o.append(r)
    assert np.allclose(res_g, res_o, rtol=1e-11, atol=0)
    Wg = s.get_state()
    nc = W.size // 4
    for v in range(4):
        a, b = Wg[v * nc:(v + 1) * nc], Wo[v * nc:(v + 1) * nc]
        assert np.abs(a - b).max() < 1e-11 * np.abs(b).max()
    s.close()


def test_converged_state_matches_oracle_and_fp32_converges():
    """The laminar corner (32 x 16, four levels): the device drives the residual down by more than
    1e5 in 150 cycles and reaches the oracle's steady state; the FP32 solver converges to it within
    single-precision accuracy."""
    sp = corner(32, 16)
    sched = [(1.0 if it < 15 else 10.0) for it in range(150)]
    s, c, W, f1, f2 = both(sp, levels=4)
    hist = np.concatenate([s.cycles(15, cfl=1.0), s.cycles(135, cfl=10.0)])
    assert hist[-1] < 1e-5 * hist[0]
    Wg = s.get_state()
    s.close()
    Wo = W
    for cfl in sched:
        Wo, r, st = c.steady_cycle(sp["nodes"], Wo, cfl, levels=4, tiles=(32, 32), nthreads=8)
        assert st == 0
    assert rel(Wg, Wo) < 1e-8
    s32, _, _, _, _ = both(sp, levels=4, precision="fp32")
    h32 = np.concatenate([s32.cycles(15, cfl=1.0), s32.cycles(135, cfl=10.0)])
    assert h32[-1] < 1e-3 * h32[0]
    assert rel(s32.get_state(), Wo) < 1e-4
    s32.close()


def test_unsupported_and_invalid_options_are_rejected():
    from paper_1302_2132_gb300 import gks
    sp = corner(36, 20)
    with pytest.raises(gks.GksError):  # 36 x 20 is not divisible by 8
        gks.SteadySolver(sp["n"], sp["bc"], sp["nodes"], levels=4, bc_data=sp["bc_prim"])
    with pytest.raises(gks.GksError):
        gks.SteadySolver(sp["n"], sp["bc"], sp["nodes"], levels=1, bc_data=sp["bc_prim"], precision="fp32_acc64")
    bad = sp["nodes"].copy()
    bad[5, 6] = bad[5, 7] + np.array([0.05, 0.0])
    with pytest.raises(gks.GksError):
        gks.SteadySolver(sp["n"], sp["bc"], bad, levels=1, bc_data=sp["bc_prim"])


def test_full_size_steady_corner_matches_oracle():
    """The bench configuration: the 24-degree corner on the 528 x 136 grid with k-omega tau_t, four
    levels, 16 x 16 LU-SGS tiles.  FP64: one cycle element by element; FP32 (the bench's precision):
    five cycles, L1 of the density against the FP64 oracle."""
    spec = inputs.compression_corner(528, 136, alpha_deg=24.0)
    sp = dict(n=spec["n"], bc=spec["bc"], bc_prim=spec["bc_prim"], nodes=spec["nodes"], prim=spec["prim"],
              f1=spec["f1"].ravel(), f2=spec["f2"].ravel(), mu=spec["mu"], T_wall=spec["T_wall"], turb=3, C_a=0.5)
    s, c, W, f1, f2 = both(sp, levels=4, limiter=1, tile=16)
    res_g = s.cycles(1, cfl=1.0, cfl_flux=0.5)
    Wo, r, st = c.steady_cycle(sp["nodes"], W, 1.0, cfl_flux=0.5, levels=4, tiles=(16, 16), f1=f1, f2=f2,
                               nthreads=16)
    assert st == 0
    assert abs(res_g[0] / r - 1.0) < 1e-11
    Wg = s.get_state()
    nc = W.size // 4
    for v in range(4):
        a, b = Wg[v * nc:(v + 1) * nc], Wo[v * nc:(v + 1) * nc]
        assert np.abs(a - b).max() < 1e-11 * np.abs(b).max()
    s.close()
    s32, _, _, _, _ = both(sp, levels=4, limiter=1, tile=16, precision="fp32")
    s32.cycles(5, cfl=1.0, cfl_flux=0.5)
    Wo = W
    for _ in range(5):
        Wo, r, st = c.steady_cycle(sp["nodes"], Wo, 1.0, cfl_flux=0.5, levels=4, tiles=(16, 16), f1=f1, f2=f2,
                                   nthreads=16)
        assert st == 0
    Wg = s32.get_state()
    assert np.abs(Wg[:nc] - Wo[:nc]).sum() / np.abs(Wo[:nc]).sum() < 1e-5
    s32.close()


@pytest.mark.parametrize("recon", ["muscl3", "weno5"])
def test_steady_cycles_with_higher_order_fine_level_match_oracle(recon):
    """MUSCL-3 / WENO-5 on the finest level of the steady solver (coarse levels first order): the
    corner grid with walls, FP64, three cycles against the oracle."""
    from paper_1302_2132_gb300 import gks
    sp = inputs.compression_corner(64, 32, alpha_deg=24.0)
    n0, n1 = sp["n"]
    rc = {"muscl3": oracle.RECON_MUSCL3, "weno5": oracle.RECON_WENO5}[recon]
    s = gks.SteadySolver(sp["n"], sp["bc"], sp["nodes"], levels=3, bc_data=sp["bc_prim"], mu=sp["mu"],
                         T_wall=sp["T_wall"], turb_model="komega", C_a=0.5, limiter="vanleer", precision="fp64",
                         lusgs_tile=16, reconstruction=recon, expand="multid")
    c = oracle.Case(2, sp["n"], [np.ones(n0), np.ones(n1)], sp["bc"], gamma=1.4, mu=sp["mu"], T_wall=sp["T_wall"],
                    turb_model=oracle.TURB_KOMEGA, multid=1, C_a=0.5, limiter=oracle.LIM_VANLEER,
                    bc_prim=sp["bc_prim"], recon=rc)
    f1, f2 = np.ravel(sp["f1"]), np.ravel(sp["f2"])
    W = c.prim_to_cons(np.asarray(sp["prim"], dtype=np.float64).ravel())
    s.set_state(W)
    s.set_turbulence(f1, f2)
    dt_g, R_g = s.residual(cfl_flux=0.5)
    dt_o, R_o = c.steady_residual(sp["nodes"], W, cfl_flux=0.5, f1=f1, f2=f2, nthreads=8)
    assert np.abs(R_g - R_o).max() <= 1e-11 * np.abs(R_o).max()
    res_g = s.cycles(3, cfl=2.0, cfl_flux=0.5)
    res_o = []
    for _ in range(3):
        W, r, st = c.steady_cycle(sp["nodes"], W, 2.0, cfl_flux=0.5, levels=3, tiles=(16, 16), f1=f1, f2=f2,
                                  nthreads=8)
        assert st == 0
        res_o.append(r)
    assert np.allclose(res_g, res_o, rtol=1e-11, atol=0)
    Wg = s.get_state().reshape(4, -1)
    Wo = W.reshape(4, -1)
    for v in range(4):
        assert np.abs(Wg[v] - Wo[v]).max() < 1e-11 * np.abs(Wo[v]).max()
    s.close()
