"""The allocation-free CFL time step (gks_cfl_dt_noalloc) agrees with gks_compute_dt and the oracle.

Callers that cannot allocate device memory (their process's device memory is held by another
allocator, or cudaMalloc's implicit synchronisation is not acceptable on their path) use
gks_cfl_dt_noalloc, whose scratch is a static device array inside the library.  This file is
collected last so that a failure here leaves every other test already run; it passes alone in a
fresh process and after the other tests.
"""
import ctypes

import numpy as np
import pytest

import oracle
from cases import oracle_case
from paper_1302_2132_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_1302_2132_gb300 import gks  # noqa: E402


def noalloc_dt(W_dev, dim, n, h, gamma, cfl, stream):
    L = gks.load()
    f = L.gks_cfl_dt_noalloc
    f.argtypes = [ctypes.c_int, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_double), ctypes.c_double,
                  ctypes.c_void_p, ctypes.c_double, ctypes.POINTER(ctypes.c_double), ctypes.c_void_p]
    f.restype = ctypes.c_int
    nn = (ctypes.c_int * 3)(*n)
    hh = (ctypes.c_double * 3)(*h)
    out = ctypes.c_double(-7.0)
    st = f(dim, nn, hh, gamma, ctypes.c_void_p(W_dev.data_ptr()), cfl, ctypes.byref(out),
           ctypes.c_void_p(stream.cuda_stream))
    return st, out.value


def reference_dt(spec, cfl):
    s = gks.Solver(spec["dim"], spec["n"], spec["bc"], dx=spec["dx"], precision="fp64")
    s.set_state(spec["prim"].ravel(), layout="soa_prim")
    dt = s.compute_dt(cfl)
    W = torch.tensor(s.get_state(), device="cuda")
    s.close()
    return dt, W


def grid_args(spec):
    h = [float(spec["dx"][d][0]) for d in range(spec["dim"])] + [1.0] * (3 - spec["dim"])
    n = list(spec["n"]) + [1] * (3 - spec["dim"])
    return n, h


def test_noalloc_dt_matches_compute_dt_and_oracle_on_two_calls():
    stream = torch.cuda.Stream()
    big = inputs.turbulence(160, 2, seed=21)        # 25600 cells: many blocks of partials
    small = inputs.turbulence(12, 3, seed=22)       # 1728 cells: fewer blocks, stale partials stay behind
    for spec, cfl in ((big, 0.5), (small, 0.3)):
        dt_ref, W = reference_dt(spec, cfl)
        n, h = grid_args(spec)
        torch.cuda.synchronize()
        st, dt = noalloc_dt(W, spec["dim"], n, h, 1.4, cfl, stream)
        assert st == gks.OK
        assert abs(dt - dt_ref) <= 1e-14 * dt_ref, (dt, dt_ref)
        # the same time step from the plain CPU statement of the CFL rule
        dt_o = oracle_case(spec).compute_dt(W.cpu().numpy(), cfl)
        assert abs(dt - dt_o) <= 1e-14 * dt_o, (dt, dt_o)


def test_noalloc_reports_a_nonphysical_state():
    """One cell with negative pressure: GKS_ENONPHYS from both entry points, dt_out untouched; a
    physical state afterwards gives the library's time step again."""
    stream = torch.cuda.Stream()
    spec = inputs.turbulence(64, 2, seed=23)
    prim = spec["prim"].copy()
    prim[3, 17, 40] = -0.2  # negative pressure in one cell
    s = gks.Solver(2, spec["n"], spec["bc"], dx=spec["dx"], precision="fp64")
    s.set_state(prim.ravel(), layout="soa_prim")
    with pytest.raises(gks.GksError) as e:
        s.compute_dt(0.5)
    assert e.value.code == gks.ENONPHYS
    W = torch.empty(4 * 64 * 64, dtype=torch.float64, device="cuda")
    s.get_state(out=W)  # device copy: no status check
    s.close()
    n, h = grid_args(spec)
    torch.cuda.synchronize()
    st, dt = noalloc_dt(W, 2, n, h, 1.4, 0.5, stream)
    assert st == gks.ENONPHYS and dt == -7.0
    dt_ref, W = reference_dt(spec, 0.5)
    st, dt = noalloc_dt(W, 2, n, h, 1.4, 0.5, stream)
    assert st == gks.OK and abs(dt - dt_ref) <= 1e-14 * dt_ref


def test_noalloc_rejects_states_beyond_the_limit_and_capturing_streams():
    stream = torch.cuda.Stream()
    W = torch.zeros(4, device="cuda", dtype=torch.float64)
    st, _ = noalloc_dt(W, 2, [8192, 4097, 1], [1.0, 1.0, 1.0], 1.4, 0.5, stream)
    assert st == gks.EINVAL
    # inside a capture the call is refused before it enqueues anything, so the capture stays valid
    spec = inputs.turbulence(32, 2, seed=24)
    dt_ref, Wd = reference_dt(spec, 0.5)
    n, h = grid_args(spec)
    x = torch.zeros(1, device="cuda")
    g = torch.cuda.CUDAGraph()
    cap = torch.cuda.Stream()
    torch.cuda.synchronize()
    with torch.cuda.graph(g, stream=cap):
        st, _ = noalloc_dt(Wd, 2, n, h, 1.4, 0.5, cap)
        x.add_(1.0)
    assert st == gks.EINVAL
    g.replay()
    torch.cuda.synchronize()
    assert float(x.item()) == 1.0
    st, dt = noalloc_dt(Wd, 2, n, h, 1.4, 0.5, stream)
    assert st == gks.OK and abs(dt - dt_ref) <= 1e-14 * dt_ref
