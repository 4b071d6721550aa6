"""Test helpers: build the GPU solver and the oracle case from one input specification."""
import numpy as np

import oracle

PREC = {"fp64": 0, "fp32": 1, "fp32_acc64": 2}


def oracle_case(spec, turb_model=0, limiter=1, multid=1, abar_mode=0, gamma=1.4, mu=1e-5, C_a=0.0,
                C_mu=0.09, beta_star=0.09, T_wall=None, recon=0, rarefaction=0):
    return oracle.Case(spec["dim"], spec["n"], spec["dx"], spec["bc"], gamma=gamma, mu=mu,
                       T_wall=spec.get("T_wall", 1.0) if T_wall is None else T_wall, turb_model=turb_model,
                       C_mu=C_mu, beta_star=beta_star, C_a=C_a, limiter=limiter, multid=multid,
                       abar_mode=abar_mode, bc_prim=spec.get("bc_prim"), recon=recon, rarefaction=rarefaction)


def gpu_solver(spec, turb_model=0, limiter=1, multid=1, abar_mode=0, gamma=1.4, mu=1e-5, C_a=0.0, C_mu=0.09,
               beta_star=0.09, precision="fp64", T_wall=None, recon=0, rarefaction=0):
    from paper_1302_2132_gb300 import gks
    return gks.Solver(spec["dim"], spec["n"], spec["bc"], dx=spec["dx"], bc_data=spec.get("bc_prim"), gamma=gamma,
                      mu=mu, T_wall=spec.get("T_wall", 1.0) if T_wall is None else T_wall, turb_model=turb_model,
                      C_mu=C_mu, beta_star=beta_star, C_a=C_a, limiter=limiter,
                      expand="multid" if multid else "directional", precision=precision,
                      abar_mode="t0" if abar_mode else "timeint", reconstruction=int(recon),
                      rarefaction="tauhat" if rarefaction else "dt")


def rel_err_per_var(a, b, nv):
    a = a.reshape(nv, -1)
    b = b.reshape(nv, -1)
    return np.array([np.linalg.norm(a[v] - b[v]) / max(np.linalg.norm(b[v]), 1e-300) for v in range(nv)])


def max_rel_elementwise(a, b, nv, floor_frac):
    """Per variable, the largest |a - b| / max(|b|, floor) over the cells, the floor being floor_frac
    times the largest |b| of that variable (so that components that pass through zero, such as a
    momentum, are compared at the scale of the variable)."""
    a = np.asarray(a).reshape(nv, -1)
    b = np.asarray(b).reshape(nv, -1)
    out = np.zeros(nv)
    for v in range(nv):
        floor = floor_frac * max(np.max(np.abs(b[v])), 1e-300)
        out[v] = np.max(np.abs(a[v] - b[v]) / np.maximum(np.abs(b[v]), floor))
    return out


def l1_rho_rel(W, Wref, nv):
    """L1 norm of the density difference relative to the L1 norm of the reference density."""
    r = np.asarray(W).reshape(nv, -1)[0]
    ro = np.asarray(Wref).reshape(nv, -1)[0]
    return float(np.sum(np.abs(r - ro)) / np.sum(np.abs(ro)))
