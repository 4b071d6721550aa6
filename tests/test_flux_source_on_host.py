"""The CUDA library's interface-flux source, compiled for the host by a test harness, agrees with
the oracle to 1e-12 on random faces (checks the hand-expanded algebra without a GPU).  In single
precision, the scalar form and the form that evaluates the two sides of a face on paired lanes (the
FP32 flux of the 1D and 2D kernels, the paired instructions emulated per lane) meet the bar of the
GPU's single-precision face tests, over the whole range of dt/tau."""
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
    f2 = os.path.join(os.path.dirname(hdr), "gks_f2.cuh")
    if not os.path.exists(SO) or os.path.getmtime(SO) < max(os.path.getmtime(p) for p in (src, hdr, f2)):
        subprocess.check_call(["g++", "-std=c++17", "-O1", "-fPIC", "-shared", "-ffp-contract=off",
                               "-I", os.path.dirname(hdr), "-o", SO + ".tmp", src])
        os.replace(SO + ".tmp", SO)
    L = ctypes.CDLL(SO)
    P = ctypes.POINTER(ctypes.c_double)
    L.flux_host.argtypes = [ctypes.c_int] * 3 + [ctypes.c_double] * 4 + [P, ctypes.c_long, P, P]
    L.flux_host_f32.argtypes = [ctypes.c_int] * 4 + [ctypes.c_double] * 4 + [P, ctypes.c_long, P, P]
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


def random_faces(rng, D, n, dt):
    """Face records and the matching oracle faces, drawn as the GPU face tests draw them: 30% of the
    faces with nearly equal states, tau_t from zero to a hundred time steps."""
    nv = D + 2
    L = 6 * nv + 2 * (D - 1) * nv + 3
    recs = np.zeros((n, L))
    faces = []
    for f in range(n):
        wl = cons(D, rng.uniform(0.3, 2.0), rng.uniform(-1.5, 1.5, D), rng.uniform(0.2, 2.0))
        if rng.random() < 0.3:
            wr = wl.copy()
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


def f32_errors(harness, D, multid, paired, recs, faces, dt, mu, C_a, abar=0):
    nv = D + 2
    n = len(faces)
    F = np.zeros((n, nv))
    tau = np.zeros(n)
    P = ctypes.POINTER(ctypes.c_double)
    assert harness.flux_host_f32(D, multid, paired, abar, 1.4, mu, C_a, dt, recs.ctypes.data_as(P), n,
                                 F.ctypes.data_as(P), tau.ctypes.data_as(P)) == 0
    errs = np.array([np.linalg.norm(F[i] - Fo) / np.linalg.norm(Fo) for i, Fo in
                     enumerate(oracle.face_flux(D, 1.4, mu, C_a, dt, f, multid=multid, abar_mode=abar) for f in faces)])
    return errs, F


@pytest.mark.parametrize("D,multid,paired", [(1, 0, 0), (1, 0, 1), (2, 0, 0), (2, 0, 1), (2, 1, 0), (2, 1, 1),
                                             (3, 0, 0), (3, 1, 0)])
def test_f32_flux_source_close_to_oracle(harness, D, multid, paired):
    rng = np.random.default_rng(4000 + 10 * D + 2 * multid + paired)
    dt = 1e-3
    recs, faces = random_faces(rng, D, 200, dt)
    errs, _ = f32_errors(harness, D, multid, paired, recs, faces, dt, 2e-5, 0.4)
    assert np.median(errs) < 2e-6 and errs.max() < 1e-4, (np.median(errs), errs.max())


@pytest.mark.parametrize("D,multid", [(1, 0), (2, 0), (2, 1)])
@pytest.mark.parametrize("x", [1e-6, 1e-4, 1e-2, 0.5, 2.0, 80.0, 300.0])
def test_paired_f32_flux_at_extreme_dt_over_tau(harness, D, multid, x):
    """x = dt/tau from near-free transport to near-equilibrium, on both branches of the paired time
    coefficients (series for x < 1, closed forms above); mu = C_a = 0, so tau = tau_t = dt/x.

    For x <= 1e-4 the flux is a small sum of terms of order tau dt times the slope moments, which
    cancel; single precision (scalar or paired alike) then loses up to about three more digits on
    rare faces: over 3000 faces a median of 5e-7, 0.1% of faces above 1e-4 and a largest error of
    2.6e-4.  There the bar is on the 99th percentile, with a bound on the largest error."""
    rng = np.random.default_rng(5000 + 10 * D + multid + int(1e3 * np.log10(x) + 7000))
    dt = 1e-3
    recs, faces = random_faces(rng, D, 200, dt)
    recs[:, -1] = dt / x
    for f in faces:
        f.tau_t = dt / x
    errs, _ = f32_errors(harness, D, multid, 1, recs, faces, dt, 0.0, 0.0)
    if x >= 1e-2:
        assert np.median(errs) < 5e-6 and errs.max() < 1e-4, (np.median(errs), errs.max())
    else:
        assert np.median(errs) < 5e-6 and np.quantile(errs, 0.99) < 1e-4 and errs.max() < 1e-3, \
            (np.median(errs), np.quantile(errs, 0.99), errs.max())


def test_paired_lanes_are_the_two_sides(harness):
    """Each lane carries one side: the paired flux of a face equals the scalar flux of the same face
    to single-precision rounding, also when the two sides differ strongly (a strong shock and a
    near-vacuum side), so a lane mix-up cannot hide in the average."""
    rng = np.random.default_rng(6000)
    D, nv, dt = 2, 4, 1e-3
    recs, faces = random_faces(rng, D, 100, dt)
    for f in range(0, 100, 2):
        recs[f, nv:2 * nv] = cons(D, 0.05, [-1.0, 0.3], 0.02)  # right side far from the left one
        recs[f, 3 * nv:4 * nv] = recs[f, nv:2 * nv]
        recs[f, 5 * nv:6 * nv] = 0.0
    n = len(faces)
    P = ctypes.POINTER(ctypes.c_double)
    out = []
    for paired in (0, 1):
        F = np.zeros((n, nv))
        tau = np.zeros(n)
        assert harness.flux_host_f32(D, 1, paired, 0, 1.4, 2e-5, 0.4, dt, recs.ctypes.data_as(P), n,
                                     F.ctypes.data_as(P), tau.ctypes.data_as(P)) == 0
        out.append((F, tau))
    (Fs, ts), (Fp, tp) = out
    rel = np.linalg.norm(Fp - Fs, axis=1) / np.linalg.norm(Fs, axis=1)
    assert np.median(rel) < 2e-6 and rel.max() < 1e-4, (np.median(rel), rel.max())
    assert np.allclose(tp, ts, rtol=1e-5, atol=0)


def stress_faces(rng, D, n, dt, mach, jump):
    """Faces with the sides' speeds up to `mach` times their sound speeds in random directions and
    density and pressure ratios across the face up to `jump` either way."""
    nv = D + 2
    L = 6 * nv + 2 * (D - 1) * nv + 3
    recs = np.zeros((n, L))
    faces = []
    for f in range(n):
        rl, pl = rng.uniform(0.5, 2.0), rng.uniform(0.5, 2.0)
        rr, pr = rl * jump ** rng.uniform(-1, 1), pl * jump ** rng.uniform(-1, 1)
        U = []
        for rho, p in ((rl, pl), (rr, pr)):
            u = rng.normal(size=D)
            U.append(u * mach * np.sqrt(1.4 * p / rho) * rng.uniform(0, 1) / np.linalg.norm(u))
        wl, wr = cons(D, rl, U[0], pl), cons(D, rr, U[1], pr)
        h = rng.uniform(0.002, 0.05)
        sl, sr = 0.1 * rng.normal(size=nv) * np.abs(wl), 0.1 * rng.normal(size=nv) * np.abs(wr)
        cl, cr = wl - 0.5 * h * sl, wr + 0.5 * h * sr
        tl, tr = 0.1 * rng.normal(size=(max(D - 1, 1), nv)), 0.1 * rng.normal(size=(max(D - 1, 1), nv))
        tau_t = rng.choice([0.0, rng.uniform(0, 5) * dt, rng.uniform(1, 100) * dt])
        parts = [wl, wr, cl, cr, sl, sr] + [tl[k] for k in range(D - 1)] + [tr[k] for k in range(D - 1)]
        recs[f, : 6 * nv + 2 * (D - 1) * nv] = np.concatenate(parts)
        recs[f, -3:] = (0.5 * h, 0.5 * h, tau_t)
        faces.append(oracle.make_face(D, wl, wr, cl, cr, sl, sr, tl[: D - 1], tr[: D - 1], 0.5 * h, 0.5 * h, tau_t))
    return recs, faces


@pytest.mark.parametrize("D,multid", [(1, 0), (2, 1)])
@pytest.mark.parametrize("paired", [0, 1])
@pytest.mark.parametrize("mach,jump", [(3.0, 10.0), (1.0, 1e3), (5.0, 1e4)])
def test_f32_flux_on_strong_jumps_and_fast_sides(harness, D, multid, paired, mach, jump):
    """Both single-precision forms on faces far from the random faces above: sides up to Mach 5 and
    density and pressure jumps up to 1e4 either way.  Every flux is finite, the median error stays at
    the face tests' level and 99% of faces are within 2e-4.  Up to Mach 3 with jumps of 10 every face
    meets the face tests' 1e-4.  With jumps of 1e3 and 1e4 a few faces in a thousand, whose flux is a
    small difference of large non-equilibrium parts, reach 1e-4 to 1e-2 (measured, scalar and paired
    alike), so there the bar is on the percentile.  Separating sides beyond about Mach 10 leave the
    interface state a near vacuum whose half-space moments underflow in single precision: the FP32
    flux is then not finite, which the update reports as a non-physical state, and the FP64 form
    evaluates those faces."""
    rng = np.random.default_rng(7000 + 10 * D + paired + int(mach) + int(np.log10(jump)))
    dt = 1e-3
    recs, faces = stress_faces(rng, D, 500, dt, mach, jump)
    errs, F = f32_errors(harness, D, multid, paired, recs, faces, dt, 2e-5, 0.4)
    assert np.all(np.isfinite(F))
    assert np.median(errs) < 2e-6 and np.quantile(errs, 0.99) < 2e-4, (np.median(errs), np.quantile(errs, 0.99))
    if mach <= 3.0 and jump <= 10.0:
        assert errs.max() < 1e-4, errs.max()
