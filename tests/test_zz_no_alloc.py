"""The allocation-free CFL time step (gks_cfl_dt_noalloc) agrees with gks_compute_dt.

Callers that cannot allocate device memory (their process's device memory is held by another
allocator, or cudaMalloc's implicit synchronisation is not acceptable on their path) use
gks_cfl_dt_noalloc, whose scratch is a static device array inside the library.  This file is
collected last so that a failure here leaves every other test already run; it passes alone in a
fresh process and after the other tests.
"""
import ctypes

import numpy as np
import pytest

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
    out = ctypes.c_double(0.0)
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


def test_noalloc_dt_matches_compute_dt_on_two_calls():
    stream = torch.cuda.Stream()
    big = inputs.turbulence(160, 2, seed=21)        # 25600 cells: two blocks of partials
    small = inputs.turbulence(12, 3, seed=22)       # 1728 cells: one block, stale partials stay behind
    for spec, cfl in ((big, 0.5), (small, 0.3)):
        dt_ref, W = reference_dt(spec, cfl)
        h = [float(spec["dx"][d][0]) for d in range(spec["dim"])] + [1.0] * (3 - spec["dim"])
        n = list(spec["n"]) + [1] * (3 - spec["dim"])
        torch.cuda.synchronize()
        st, dt = noalloc_dt(W, spec["dim"], n, h, 1.4, cfl, stream)
        assert st == gks.OK
        assert abs(dt - dt_ref) <= 1e-14 * dt_ref, (dt, dt_ref)


def test_noalloc_rejects_states_beyond_the_static_scratch():
    stream = torch.cuda.Stream()
    W = torch.zeros(4, device="cuda", dtype=torch.float64)
    st, _ = noalloc_dt(W, 2, [8192, 4097, 1], [1.0, 1.0, 1.0], 1.4, 0.5, stream)
    assert st == gks.EINVAL
