"""ctypes binding of the serving entry points of libgks.so (gks_server_* in include/gks.h).

A Server keeps a device arena for resident solves; submitted requests are admitted in arrival
order as memory frees up and advance together in batched, graph-captured steps on the GPU (the
C++ worker thread inside the library does the batching).  This module only marshals arguments.
"""
import ctypes

import numpy as np

from . import gks

_D = ctypes.c_double
_I = ctypes.c_int


class _Request(ctypes.Structure):
    _fields_ = [("dim", _I), ("n", _I * 3), ("lo", _D * 3), ("hi", _D * 3), ("bc", (_I * 2) * 3),
                ("gamma", _D), ("mu", _D), ("C_a", _D), ("T_wall", _D), ("cfl", _D),
                ("limiter", _I), ("expand", _I), ("nsteps", _I)]


def _lib():
    L = gks.load()
    if not getattr(L, "_serve_ready", False):
        P = ctypes.c_void_p
        L.gks_server_create.argtypes = [_I, ctypes.c_size_t, ctypes.c_long, _I, P, ctypes.POINTER(P)]
        L.gks_server_submit.argtypes = [P, ctypes.POINTER(_Request), ctypes.POINTER(_D),
                                        ctypes.POINTER(ctypes.c_longlong)]
        L.gks_server_poll.argtypes = [P, ctypes.c_longlong, ctypes.POINTER(_I), ctypes.POINTER(_D),
                                      ctypes.POINTER(_D)]
        L.gks_server_wait_all.argtypes = [P, _D]
        L.gks_server_stats.argtypes = [P, ctypes.POINTER(ctypes.c_longlong), ctypes.POINTER(_D),
                                       ctypes.POINTER(_D), ctypes.POINTER(_D), ctypes.POINTER(_D)]
        L.gks_server_destroy.argtypes = [P]
        L.gks_server_tile_variants.argtypes = [P, ctypes.POINTER(_I)]
        for f in ("gks_server_create", "gks_server_submit", "gks_server_poll", "gks_server_wait_all",
                  "gks_server_stats", "gks_server_destroy", "gks_server_tile_variants"):
            getattr(L, f).restype = _I
        L._serve_ready = True
    return L


class Server:
    def __init__(self, precision="fp32", arena_bytes=8 << 30, max_cells=512 * 512, chunk_steps=24, stream=None):
        L = _lib()
        h = ctypes.c_void_p()
        st = L.gks_server_create(gks.PRECISION[precision], arena_bytes, max_cells, chunk_steps,
                                 ctypes.c_void_p(stream.cuda_stream if stream is not None else 0), ctypes.byref(h))
        if st != gks.OK:
            raise gks.GksError(st, "gks_server_create failed")
        self._h = h
        self._nv = {}

    def submit(self, spec, gamma=1.4, mu=1e-4, C_a=0.5, T_wall=1.0, cfl=0.5, limiter="vanleer", expand="multid"):
        """Queue a request described by an inputs spec (dim, n, lo, hi, bc, prim, nsteps)."""
        q = _Request()
        q.dim = spec["dim"]
        for d in range(3):
            q.n[d] = spec["n"][d] if d < spec["dim"] else 1
            q.lo[d] = spec["lo"][d] if d < spec["dim"] else 0.0
            q.hi[d] = spec["hi"][d] if d < spec["dim"] else 1.0
            for s in range(2):
                q.bc[d][s] = spec["bc"][d][s] if d < spec["dim"] else 0
        q.gamma, q.mu, q.C_a, q.T_wall, q.cfl = gamma, mu, C_a, T_wall, cfl
        q.limiter = gks.LIMITER[limiter]
        q.expand = gks.EXPAND[expand]
        q.nsteps = int(spec["nsteps"])
        prim = np.ascontiguousarray(spec["prim"], dtype=np.float64).ravel()
        rid = ctypes.c_longlong()
        st = _lib().gks_server_submit(self._h, ctypes.byref(q), prim.ctypes.data_as(ctypes.POINTER(_D)),
                                      ctypes.byref(rid))
        if st != gks.OK:
            raise gks.GksError(st, "gks_server_submit failed")
        self._nv[rid.value] = prim.size
        return rid.value

    def poll(self, rid, want_state=True):
        done = _I()
        lat = _D()
        W = np.zeros(self._nv[rid]) if want_state else None
        st = _lib().gks_server_poll(self._h, rid, ctypes.byref(done),
                                    W.ctypes.data_as(ctypes.POINTER(_D)) if W is not None else None, ctypes.byref(lat))
        if st != gks.OK:
            raise gks.GksError(st, "gks_server_poll failed")
        return bool(done.value), (W if done.value else None), lat.value

    def wait_all(self, timeout=600.0):
        st = _lib().gks_server_wait_all(self._h, timeout)
        if st != gks.OK:
            raise gks.GksError(st, "gks_server_wait_all failed")

    def stats(self):
        c = ctypes.c_longlong()
        p50, p99, sps, busy = _D(), _D(), _D(), _D()
        _lib().gks_server_stats(self._h, ctypes.byref(c), ctypes.byref(p50), ctypes.byref(p99), ctypes.byref(sps),
                                ctypes.byref(busy))
        return {"completed": c.value, "p50_s": p50.value, "p99_s": p99.value, "solves_per_s": sps.value,
                "gpu_busy_s": busy.value}

    def tile_variants(self):
        """Tile shape (gks_tile_shape variant) of each group's batch kernel: 1D, 2D, 2D multi-D."""
        v = (_I * 3)()
        _lib().gks_server_tile_variants(self._h, v)
        return list(v)

    def close(self):
        if self._h is not None:
            _lib().gks_server_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
