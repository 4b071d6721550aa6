"""ORACLE — TEST INFRASTRUCTURE, NOT PART OF THE LIBRARY.

ctypes loader for the plain double-precision CPU statement of the turbulent gas-kinetic scheme
(``gks_oracle.cpp``).  Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU baseline
may import this package.  It imports nothing from ``paper_1302_2132_gb300`` and the library
imports nothing from it.

Parity status per function (what pins it, in ``tests/test_oracle_*.py``):
  moments / time coefficients / slope solves / face flux  -- pinned (quadrature, closed forms,
      the compact form with corrected beta, Euler and Navier-Stokes limits)
  whole scheme (MUSCL, update, CFL step, BCs)              -- pinned (Sod exact solution,
      conservation, free-stream preservation)
  turbulent relaxation-time field                           -- pinned for eta = 0 and k-eps/k-omega
      equivalence; the turbulent configurations beyond their invariants are parity unpinned
  k-omega transport (Wilcox 2006 reading)                   -- pinned (homogeneous decay against the
      closed-form ODE solution, uniform-shear production and its limiter, exact discrete diffusion of
      a Fourier mode, advection by a uniform stream, conservation on periodic grids)
  higher-order reconstructions (MUSCL-3, WENO-5)            -- pinned (convergence orders, exact
      quadratics, Sod stability, smooth-wave accuracy)
  body-fitted step, both expansions, C-grid wake cut        -- pinned (equal to the rectilinear step
      on uniform and wall-clustered grids, free stream, rotation, conservation, second-order
      convergence, the cut against a rectilinear strip, symmetry)
  body-fitted MUSCL-3 / WENO-5, rarefaction, transport      -- pinned (rectilinear equivalence, free
      stream, rotation; exact divergence of a linear field; conservation and exact decay)
  steady residual, LU-SGS, multigrid cycle                  -- pinned (time-accurate equivalence of
      the residual, dense solve of the LU-SGS factors, convergence to one steady state)
  steady k-omega update                                     -- pinned (point-implicit closed form at
      rest, free stream, first-order consistency with the time-accurate transport, bounded iteration)
"""
import ctypes
import os
import subprocess
import threading

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "gks_oracle.cpp")
BUILD_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD_DIR, "liboracle.so")

FULL, POS, NEG = 0, 1, 2
BC_PERIODIC, BC_TRANSMISSIVE, BC_WALL, BC_DIRICHLET, BC_OUTFLOW = 0, 1, 2, 3, 4
TURB_NONE, TURB_MUT, TURB_KEPS, TURB_KOMEGA = 0, 1, 2, 3
LIM_MINMOD, LIM_VANLEER = 0, 1
ABAR_TIMEINT, ABAR_T0 = 0, 1
RECON_MUSCL2, RECON_MUSCL3, RECON_WENO5 = 0, 1, 2

_lock = threading.Lock()
_lib = None


def build(force=False):
    """Compile the oracle with the host compiler (no -march=native, no FP contraction)."""
    os.makedirs(BUILD_DIR, exist_ok=True)
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= max(
            os.path.getmtime(SRC), os.path.getmtime(os.path.join(HERE, "gks_oracle.h"))):
        return LIB
    tmp = LIB + ".tmp%d" % os.getpid()
    cmd = ["g++", "-std=c++17", "-O2", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
           "-o", tmp, SRC]
    subprocess.check_call(cmd)
    os.replace(tmp, LIB)
    return LIB


class Problem(ctypes.Structure):
    _fields_ = [
        ("dim", ctypes.c_int),
        ("n", ctypes.c_int * 3),
        ("dx", ctypes.POINTER(ctypes.c_double) * 3),
        ("bc", (ctypes.c_int * 2) * 3),
        ("bc_prim", (ctypes.POINTER(ctypes.c_double) * 2) * 3),
        ("gamma", ctypes.c_double),
        ("mu", ctypes.c_double),
        ("T_wall", ctypes.c_double),
        ("turb_model", ctypes.c_int),
        ("C_mu", ctypes.c_double),
        ("beta_star", ctypes.c_double),
        ("C_a", ctypes.c_double),
        ("limiter", ctypes.c_int),
        ("multid", ctypes.c_int),
        ("abar_mode", ctypes.c_int),
        ("recon", ctypes.c_int),
        ("wake_cut", ctypes.c_int),
        ("rarefaction", ctypes.c_int),
        ("no_fallback", ctypes.c_int),
    ]


class Face(ctypes.Structure):
    _fields_ = [
        ("wl", ctypes.c_double * 5), ("wr", ctypes.c_double * 5),
        ("cl", ctypes.c_double * 5), ("cr", ctypes.c_double * 5),
        ("sl", ctypes.c_double * 5), ("sr", ctypes.c_double * 5),
        ("tl", (ctypes.c_double * 5) * 2), ("tr", (ctypes.c_double * 5) * 2),
        ("dxl", ctypes.c_double), ("dxr", ctypes.c_double), ("tau_t", ctypes.c_double),
    ]


class FaceDiag(ctypes.Structure):
    _fields_ = [
        ("w0", ctypes.c_double * 5), ("al", ctypes.c_double * 5), ("ar", ctypes.c_double * 5),
        ("bl", (ctypes.c_double * 5) * 2), ("br", (ctypes.c_double * 5) * 2),
        ("Al", ctypes.c_double * 5), ("Ar", ctypes.c_double * 5),
        ("abl", ctypes.c_double * 5), ("abr", ctypes.c_double * 5),
        ("bb", (ctypes.c_double * 5) * 2), ("Ab", ctypes.c_double * 5),
        ("tau", ctypes.c_double), ("T", ctypes.c_double * 6), ("tauhat", ctypes.c_double),
    ]


class KOmega(ctypes.Structure):
    _fields_ = [
        ("alpha", ctypes.c_double), ("beta0", ctypes.c_double), ("beta_star", ctypes.c_double),
        ("sigma", ctypes.c_double), ("sigma_star", ctypes.c_double), ("sigma_do", ctypes.c_double),
        ("C_lim", ctypes.c_double), ("omega_floor", ctypes.c_double),
        ("sources", ctypes.c_int), ("diffusion", ctypes.c_int),
    ]


_D = ctypes.c_double
_PD = ctypes.POINTER(ctypes.c_double)
_I = ctypes.c_int


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = ctypes.CDLL(LIB)
            L.orc_umoments.argtypes = [_D, _D, _I, _I, _PD]
            L.orc_ximoments.argtypes = [_D, _D, _I, _PD]
            L.orc_time_coeffs.argtypes = [_D, _D, _PD]
            L.orc_slope.argtypes = [_I, _D, _PD, _PD, _PD]
            L.orc_time_coeffs_hat.argtypes = [_D, _D, _D, _PD]
            L.orc_face_flux.argtypes = [_I, _D, _D, _D, _D, _I, _I, _I, ctypes.POINTER(Face), _PD,
                                        ctypes.POINTER(FaceDiag)]
            L.orc_face_flux_compact.argtypes = [_I, _D, _D, _D, _D, _I, _I, _I, _I, ctypes.POINTER(Face), _PD]
            L.orc_euler_flux.argtypes = [_I, _D, _PD, _PD]
            L.orc_reconstruct.argtypes = [_I, _I, _PD, _PD, _I, _PD, _PD]
            P = ctypes.POINTER(Problem)
            L.orc_prim_to_cons.argtypes = [P, _PD, _PD, ctypes.c_long]
            L.orc_cons_to_prim.argtypes = [P, _PD, _PD, ctypes.c_long]
            L.orc_compute_dt.argtypes = [P, _PD, _D, _PD]
            L.orc_tau_turb.argtypes = [P, _PD, _PD, _PD, _PD]
            L.orc_rarefaction.argtypes = [P, _PD, _PD, _PD, _PD]
            L.orc_step.argtypes = [P, _PD, _PD, _PD, _D, _PD, _I]
            L.orc_fallback_count.argtypes = [P, _PD, _PD, _PD, ctypes.POINTER(ctypes.c_long)]
            L.orc_run.argtypes = [P, _PD, _PD, _PD, _D, _D, _I, _D, _PD, ctypes.POINTER(_I), _I]
            L.orc_step_curv.argtypes = [P, _PD, _PD, _PD, _PD, _D, _I]
            L.orc_compute_dt_curv.argtypes = [P, _PD, _PD, _D, _PD]
            L.orc_rarefaction_curv.argtypes = [P, _PD, _PD, _PD, _PD, _PD]
            L.orc_step_komega_curv.argtypes = [P, _PD, ctypes.POINTER(KOmega), _PD, _PD, _PD, _D, _I]
            L.orc_steady_residual.argtypes = [P, _PD, _PD, _PD, _PD, _D, _I, _PD, _PD, _I]
            L.orc_lusgs.argtypes = [P, _PD, _PD, _PD, _PD, _PD, _PD, _I, _I, _PD]
            L.orc_steady_cycle.argtypes = [P, _PD, _PD, _PD, _PD, _D, _D, _I, _I, _I, _I, _PD]
            L.orc_steady_komega.argtypes = [P, _PD, ctypes.POINTER(KOmega), _PD, _PD, _PD, _D, _D, _I]
            L.orc_komega_defaults.argtypes = [ctypes.POINTER(KOmega)]
            L.orc_step_komega.argtypes = [P, ctypes.POINTER(KOmega), _PD, _PD, _PD, _D, _I]
            _lib = L
    return _lib


def _ptr(a):
    if a is None:
        return None
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(_PD)


# ------------------------------------------------------------------------------------------------
# Point functions
# ------------------------------------------------------------------------------------------------
def umoments(U, lam, region, nmax):
    out = np.zeros(nmax + 1)
    lib().orc_umoments(U, lam, region, nmax, _ptr(out))
    return out


def ximoments(K, lam, lmax):
    out = np.zeros(lmax + 1)
    lib().orc_ximoments(K, lam, lmax, _ptr(out))
    return out


def time_coeffs(dt, tau):
    """T0..T5 and dt^2/2 - T2 of the time integral of Eq. resultingf."""
    out = np.zeros(7)
    lib().orc_time_coeffs(dt, tau, _ptr(out))
    return out


def slope(D, K, w, rhs):
    w = np.ascontiguousarray(w, dtype=np.float64)
    rhs = np.ascontiguousarray(rhs, dtype=np.float64)
    out = np.zeros(D + 2)
    lib().orc_slope(D, K, _ptr(w), _ptr(rhs), _ptr(out))
    return out


def make_face(D, wl, wr, cl=None, cr=None, sl=None, sr=None, tl=None, tr=None, dxl=0.5, dxr=0.5, tau_t=0.0):
    nv = D + 2
    f = Face()
    z = np.zeros(nv)
    for name, val in (("wl", wl), ("wr", wr), ("cl", wl if cl is None else cl),
                      ("cr", wr if cr is None else cr), ("sl", z if sl is None else sl),
                      ("sr", z if sr is None else sr)):
        arr = getattr(f, name)
        for v in range(nv):
            arr[v] = float(val[v])
    for name, val in (("tl", tl), ("tr", tr)):
        arr = getattr(f, name)
        if val is not None:
            for k in range(D - 1):
                for v in range(nv):
                    arr[k][v] = float(val[k][v])
    f.dxl, f.dxr, f.tau_t = dxl, dxr, tau_t
    return f


def time_coeffs_hat(dt, tau, eps):
    """T0..T5 and dt^2/2 - T2 with the degree of rarefaction eps in place of tau/dt."""
    out = np.zeros(7)
    lib().orc_time_coeffs_hat(dt, tau, eps, _ptr(out))
    return out


def face_flux(D, gamma, mu, C_a, dt, face, multid=1, abar_mode=ABAR_TIMEINT, diag=False, rarefaction=0):
    F = np.zeros(D + 2)
    dg = FaceDiag()
    lib().orc_face_flux(D, gamma, mu, C_a, dt, multid, abar_mode, int(rarefaction), ctypes.byref(face), _ptr(F),
                        ctypes.byref(dg))
    if diag:
        return F, dg
    return F


def face_flux_compact(D, gamma, mu, C_a, dt, face, multid=1, abar_mode=ABAR_TIMEINT, printed_beta=False,
                      rarefaction=0):
    F = np.zeros(D + 2)
    lib().orc_face_flux_compact(D, gamma, mu, C_a, dt, multid, abar_mode, int(rarefaction), int(printed_beta),
                                ctypes.byref(face), _ptr(F))
    return F


def reconstruct(recon, v, h=None, limiter=LIM_VANLEER):
    """Face values of a 1D row of cell averages: (wl, wr) with wl[i] the value of cell i at its right
    face and wr[i] at its left face (NaN where the stencil is incomplete)."""
    v = np.ascontiguousarray(v, dtype=np.float64)
    h = np.ascontiguousarray(np.ones_like(v) if h is None else h, dtype=np.float64)
    wl = np.full_like(v, np.nan)
    wr = np.full_like(v, np.nan)
    lib().orc_reconstruct(recon, limiter, _ptr(v), _ptr(h), v.size, _ptr(wl), _ptr(wr))
    return wl, wr


def euler_flux(D, gamma, w):
    w = np.ascontiguousarray(w, dtype=np.float64)
    F = np.zeros(D + 2)
    lib().orc_euler_flux(D, gamma, _ptr(w), _ptr(F))
    return F


# ------------------------------------------------------------------------------------------------
# Grid problems
# ------------------------------------------------------------------------------------------------
class Case:
    """A grid problem for the oracle.  Arrays are kept alive on the instance."""

    def __init__(self, dim, n, dx, bc, gamma=1.4, mu=1e-5, T_wall=1.0, turb_model=TURB_NONE,
                 C_mu=0.09, beta_star=0.09, C_a=0.0, limiter=LIM_VANLEER, multid=1,
                 abar_mode=ABAR_TIMEINT, bc_prim=None, recon=RECON_MUSCL2, wake_cut=0, rarefaction=0):
        self.dim = dim
        self.n = tuple(n)
        self.P = Problem()
        self.P.dim = dim
        self._keep = []
        for d in range(3):
            self.P.n[d] = int(n[d]) if d < dim else 1
        for d in range(dim):
            w = np.ascontiguousarray(np.broadcast_to(np.asarray(dx[d], dtype=np.float64), (n[d],)))
            self._keep.append(w)
            self.P.dx[d] = _ptr(w)
            for s in range(2):
                self.P.bc[d][s] = int(bc[d][s])
                if bc_prim is not None and bc_prim[d][s] is not None:
                    a = np.ascontiguousarray(bc_prim[d][s], dtype=np.float64)
                    self._keep.append(a)
                    self.P.bc_prim[d][s] = _ptr(a)
        self.P.gamma, self.P.mu, self.P.T_wall = gamma, mu, T_wall
        self.P.turb_model, self.P.C_mu, self.P.beta_star, self.P.C_a = turb_model, C_mu, beta_star, C_a
        self.P.limiter, self.P.multid, self.P.abar_mode = limiter, multid, abar_mode
        self.P.recon = recon
        self.P.wake_cut = int(wake_cut)
        self.P.rarefaction = int(rarefaction)
        self.ncell = int(np.prod(n[:dim]))
        self.nv = dim + 2

    def _state(self, W):
        W = np.ascontiguousarray(W, dtype=np.float64)
        assert W.size == self.nv * self.ncell
        return W

    def _field(self, f):
        if f is None:
            return None
        f = np.ascontiguousarray(f, dtype=np.float64)
        assert f.size == self.ncell
        return f

    def prim_to_cons(self, prim):
        prim = self._state(prim)
        W = np.zeros_like(prim)
        lib().orc_prim_to_cons(ctypes.byref(self.P), _ptr(prim), _ptr(W), self.ncell)
        return W

    def cons_to_prim(self, W):
        W = self._state(W)
        prim = np.zeros_like(W)
        lib().orc_cons_to_prim(ctypes.byref(self.P), _ptr(W), _ptr(prim), self.ncell)
        return prim

    def fallback_count(self, W, f1=None, f2=None):
        """Face sides evaluated at first order (reconstructed rho or p not positive) in a step from W."""
        W = self._state(W)
        n = ctypes.c_long()
        lib().orc_fallback_count(ctypes.byref(self.P), _ptr(W), _ptr(self._field(f1)), _ptr(self._field(f2)),
                                 ctypes.byref(n))
        return n.value

    def compute_dt(self, W, cfl):
        W = self._state(W)
        dt = ctypes.c_double()
        lib().orc_compute_dt(ctypes.byref(self.P), _ptr(W), cfl, ctypes.byref(dt))
        return dt.value

    def tau_turb(self, W, f1=None, f2=None):
        W = self._state(W)
        out = np.zeros(self.ncell)
        lib().orc_tau_turb(ctypes.byref(self.P), _ptr(W), _ptr(self._field(f1)), _ptr(self._field(f2)), _ptr(out))
        return out

    def rarefaction(self, W, f1=None, f2=None):
        W = self._state(W)
        out = np.zeros(self.ncell)
        lib().orc_rarefaction(ctypes.byref(self.P), _ptr(W), _ptr(self._field(f1)), _ptr(self._field(f2)),
                              _ptr(out))
        return out

    def step(self, W, dt, f1=None, f2=None, nthreads=1):
        """One step; returns (W_new, status, resid[3, nv] = L2, Linf, total)."""
        W = self._state(W).copy()
        resid = np.zeros(3 * self.nv)
        st = lib().orc_step(ctypes.byref(self.P), _ptr(W), _ptr(self._field(f1)), _ptr(self._field(f2)), dt,
                            _ptr(resid), nthreads)
        return W, st, resid.reshape(3, self.nv)

    def run(self, W, nsteps, cfl=0.5, dt_fixed=0.0, t_end=0.0, t0=0.0, f1=None, f2=None, nthreads=1):
        """Steps until nsteps or t_end; returns (W, t, steps_done, status)."""
        W = self._state(W).copy()
        t = ctypes.c_double(t0)
        done = ctypes.c_int(0)
        st = lib().orc_run(ctypes.byref(self.P), _ptr(W), _ptr(self._field(f1)), _ptr(self._field(f2)),
                           dt_fixed, cfl, nsteps, t_end, ctypes.byref(t), ctypes.byref(done), nthreads)
        return W, t.value, done.value, st

    def step_komega(self, W, RK, RW, dt, coeffs=None, nthreads=1):
        """One flow step plus the k-omega transport step (Wilcox 2006 reading) of RK = rho k and
        RW = rho omega; returns (W, RK, RW, status).  coeffs: a KOmega (default Wilcox's values)."""
        W = self._state(W).copy()
        RK = self._field(RK).copy()
        RW = self._field(RW).copy()
        c = coeffs if coeffs is not None else komega_defaults()
        st = lib().orc_step_komega(ctypes.byref(self.P), ctypes.byref(c), _ptr(W), _ptr(RK), _ptr(RW), dt,
                                   nthreads)
        return W, RK, RW, st


    def _nodes(self, nodes):
        nodes = np.ascontiguousarray(nodes, dtype=np.float64)
        assert self.dim == 2 and nodes.size == 2 * (self.n[0] + 1) * (self.n[1] + 1)
        return nodes

    def step_curv(self, nodes, W, dt, f1=None, f2=None, nthreads=1):
        """One directional step on the curvilinear grid of the node array nodes[n1 + 1, n0 + 1, 2]
        (the problem's dx is not used); returns (W_new, status).  Status 2: a cell that is not a
        convex counter-clockwise quadrilateral."""
        nodes = self._nodes(nodes)
        W = self._state(W).copy()
        st = lib().orc_step_curv(ctypes.byref(self.P), _ptr(nodes), _ptr(W), _ptr(self._field(f1)),
                                 _ptr(self._field(f2)), dt, nthreads)
        return W, st

    def compute_dt_curv(self, nodes, W, cfl):
        nodes = self._nodes(nodes)
        W = self._state(W)
        dt = ctypes.c_double()
        st = lib().orc_compute_dt_curv(ctypes.byref(self.P), _ptr(nodes), _ptr(W), cfl, ctypes.byref(dt))
        assert st == 0
        return dt.value


    def rarefaction_curv(self, nodes, W, f1=None, f2=None):
        """eps = (mu / p + tau_t) |div U| per cell on a curvilinear grid (Green-Gauss divergence)."""
        nodes = self._nodes(nodes)
        W = self._state(W)
        eps = np.zeros(self.ncell)
        st = lib().orc_rarefaction_curv(ctypes.byref(self.P), _ptr(nodes), _ptr(W), _ptr(self._field(f1)),
                                        _ptr(self._field(f2)), _ptr(eps))
        assert st == 0, st
        return eps

    def step_komega_curv(self, nodes, W, RK, RW, dt, coeffs=None, nthreads=1):
        """One flow step plus the k-omega transport step on a curvilinear grid; returns (W, RK, RW,
        status)."""
        nodes = self._nodes(nodes)
        W = self._state(W).copy()
        RK = self._field(RK).copy()
        RW = self._field(RW).copy()
        c = coeffs if coeffs is not None else komega_defaults()
        st = lib().orc_step_komega_curv(ctypes.byref(self.P), _ptr(nodes), ctypes.byref(c), _ptr(W), _ptr(RK),
                                        _ptr(RW), dt, nthreads)
        return W, RK, RW, st

    def steady_residual(self, nodes, W, cfl_flux=0.5, first_order=False, f1=None, f2=None, nthreads=1):
        """Local explicit steps (CFL 1) and the steady residual (flux rates over the face windows
        cfl_flux min(dt_l, dt_r), times face length, outward) on a curvilinear grid: (dt_cell, R)."""
        nodes = self._nodes(nodes)
        W = self._state(W)
        dtc = np.zeros(self.ncell)
        R = np.zeros(self.nv * self.ncell)
        st = lib().orc_steady_residual(ctypes.byref(self.P), _ptr(nodes), _ptr(W), _ptr(self._field(f1)),
                                       _ptr(self._field(f2)), cfl_flux, int(first_order), _ptr(dtc), _ptr(R),
                                       nthreads)
        assert st == 0, st
        return dtc, R

    def lusgs(self, nodes, W, dt_cell, R, tiles=(32, 32), f1=None, f2=None):
        """The LU-SGS increment of residual R with local steps dt_cell, tile by tile."""
        nodes = self._nodes(nodes)
        W = self._state(W)
        dtc = np.ascontiguousarray(dt_cell, dtype=np.float64)
        R = np.ascontiguousarray(R, dtype=np.float64)
        dW = np.zeros(self.nv * self.ncell)
        st = lib().orc_lusgs(ctypes.byref(self.P), _ptr(nodes), _ptr(W), _ptr(self._field(f1)), _ptr(self._field(f2)),
                             _ptr(dtc), _ptr(R), int(tiles[0]), int(tiles[1]), _ptr(dW))
        assert st == 0, st
        return dW

    def steady_cycle(self, nodes, W, cfl, cfl_flux=0.5, levels=4, tiles=(32, 32), f1=None, f2=None, nthreads=1):
        """One FAS multigrid cycle with LU-SGS smoothing (pseudo-time steps cfl times the local explicit
        steps); returns (W, residual before the cycle, status)."""
        nodes = self._nodes(nodes)
        W = self._state(W).copy()
        res = ctypes.c_double()
        st = lib().orc_steady_cycle(ctypes.byref(self.P), _ptr(nodes), _ptr(W), _ptr(self._field(f1)),
                                    _ptr(self._field(f2)), cfl, cfl_flux, int(levels), int(tiles[0]), int(tiles[1]),
                                    nthreads,
                                    ctypes.byref(res))
        return W, res.value, st

    def steady_komega(self, nodes, W, RK, RW, cfl, cfl_flux=0.5, coeffs=None, nthreads=1):
        """The steady k-omega update (one diagonal-implicit step with the flow residual's mass flux
        rates and local steps) of RK, RW for the state W; returns (RK, RW, status)."""
        nodes = self._nodes(nodes)
        W = self._state(W)
        RK = self._field(RK).copy()
        RW = self._field(RW).copy()
        c = coeffs if coeffs is not None else komega_defaults()
        st = lib().orc_steady_komega(ctypes.byref(self.P), _ptr(nodes), ctypes.byref(c), _ptr(W), _ptr(RK), _ptr(RW),
                                     cfl, cfl_flux, nthreads)
        return RK, RW, st

    def steady_cycle_komega(self, nodes, W, RK, RW, cfl, cfl_flux=0.5, levels=4, tiles=(32, 32), coeffs=None,
                            nthreads=1):
        """One steady cycle with k-omega transport: the k-omega update from the cycle's starting state,
        then the flow cycle with the fields k = RK / rho, omega = RW / rho of that state; returns (W,
        RK, RW, flow residual before the cycle, status)."""
        W0 = self._state(W)
        n = self.ncell
        k, om = self._field(RK).ravel() / W0[:n], self._field(RW).ravel() / W0[:n]
        RK, RW, st = self.steady_komega(nodes, W0, RK, RW, cfl, cfl_flux, coeffs, nthreads)
        if st:
            return W0.copy(), RK, RW, float("nan"), st
        W, res, st = self.steady_cycle(nodes, W0, cfl, cfl_flux, levels, tiles, k, om, nthreads)
        return W, RK, RW, res, st


def komega_defaults(**over):
    """Wilcox's 2006 k-omega closure coefficients (and the test switches), optionally overridden."""
    c = KOmega()
    lib().orc_komega_defaults(ctypes.byref(c))
    for k, v in over.items():
        setattr(c, k, v)
    return c
