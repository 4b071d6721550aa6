"""The CUDA library's interface-flux source, compiled for the host by a test harness, agrees with
the oracle to 1e-12 on random faces (checks the hand-expanded algebra without a GPU)."""
import ctypes
import os
import subprocess

import numpy as np
import pytest

import oracle

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
SO = os.path.join(HERE, "_build", "libflux_host.so")


@pytest.fixture(scope="module")
def harness():
    os.makedirs(os.path.dirname(SO), exist_ok=True)
    src = os.path.join(HERE, "flux_host_harness.cpp")
    hdr = os.path.join(ROOT, "paper_1302_2132_gb300", "csrc", "gks_flux.cuh")
    if not os.path.exists(SO) or os.path.getmtime(SO) < max(os.path.getmtime(src), os.path.getmtime(hdr)):
        subprocess.check_call(["g++", "-std=c++17", "-O1", "-fPIC", "-shared", "-ffp-contract=off",
                               "-I", os.path.dirname(hdr), "-o", SO + ".tmp", src])
        os.replace(SO + ".tmp", SO)
    L = ctypes.CDLL(SO)
    P = ctypes.POINTER(ctypes.c_double)
    L.flux_host.argtypes = [ctypes.c_int] * 3 + [ctypes.c_double] * 4 + [P, ctypes.c_long, P, P]
    return L


def cons(D, rho, U, p, g=1.4):
    U = np.asarray(U, dtype=float)
    return np.concatenate([[rho], rho * U, [p / (g - 1.0) + 0.5 * rho * np.dot(U, U)]])


@pytest.mark.parametrize("D,multid,abar", [(1, 0, 0), (2, 0, 0), (2, 1, 0), (2, 1, 1), (3, 0, 0), (3, 1, 0)])
def test_flux_source_matches_oracle(harness, D, multid, abar):
    rng = np.random.default_rng(77 + 10 * D + multid)
    nv = D + 2
    L = 6 * nv + 2 * (D - 1) * nv + 3
    n = 60
    dt, mu, C_a = 1e-3, 2e-5, 0.4
    recs = np.zeros((n, L))
    faces = []
    for f in range(n):
        wl = cons(D, rng.uniform(0.3, 2.0), rng.uniform(-1.5, 1.5, D), rng.uniform(0.2, 2.0))
        wr = cons(D, rng.uniform(0.3, 2.0), rng.uniform(-1.5, 1.5, D), rng.uniform(0.2, 2.0))
        h = rng.uniform(0.002, 0.05)
        sl, sr = rng.normal(size=nv), rng.normal(size=nv)
        cl, cr = wl - 0.5 * h * sl, wr + 0.5 * h * sr
        tl, tr = rng.normal(size=(2, nv)), rng.normal(size=(2, nv))
        tau_t = [0.0, 1e-7, 3e-4, 5e-2][f % 4]
        parts = [wl, wr, cl, cr, sl, sr] + [tl[k] for k in range(D - 1)] + [tr[k] for k in range(D - 1)]
        recs[f, : 6 * nv + 2 * (D - 1) * nv] = np.concatenate(parts)
        recs[f, -3:] = (0.5 * h, 0.5 * h, tau_t)
        faces.append(oracle.make_face(D, wl, wr, cl, cr, sl, sr, tl[: D - 1], tr[: D - 1], 0.5 * h, 0.5 * h, tau_t))
    F = np.zeros((n, nv))
    tau = np.zeros(n)
    P = ctypes.POINTER(ctypes.c_double)
    assert harness.flux_host(D, multid, abar, 1.4, mu, C_a, dt, recs.ctypes.data_as(P), n, F.ctypes.data_as(P),
                             tau.ctypes.data_as(P)) == 0
    for i, f in enumerate(faces):
        Fo = oracle.face_flux(D, 1.4, mu, C_a, dt, f, multid=multid, abar_mode=abar)
        assert np.linalg.norm(F[i] - Fo) <= 1e-12 * np.linalg.norm(Fo), (i, F[i], Fo)
