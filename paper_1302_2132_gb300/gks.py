"""ctypes binding of libgks.so (C ABI in include/gks.h): argument marshalling only.

Every step of the scheme runs in the library's CUDA kernels; this module converts Python/torch
arguments into the C structures and pointers.  PyTorch provides device memory for the caller's
tensors and the CUDA stream the library works on.  If the library cannot be loaded the import
fails: there is no other implementation behind this module.
"""
import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libgks.so")

OK, EINVAL, ENOMEM, ECUDA, ENONPHYS, ETIMEOUT, EUNSUPPORTED = range(7)
BC = {"periodic": 0, "transmissive": 1, "wall": 2, "dirichlet": 3, "outflow": 4}
TURB = {"none": 0, "mut": 1, "keps": 2, "komega": 3, "komega_transport": 4}
LIMITER = {"minmod": 0, "vanleer": 1}
EXPAND = {"directional": 0, "multid": 1}
PRECISION = {"fp64": 0, "fp32": 1, "fp32_acc64": 2}
ABAR = {"timeint": 0, "t0": 1}
RAREFACTION = {"dt": 0, "tauhat": 1}
RECON = {"muscl2": 0, "muscl3": 1, "weno5": 2}
LAYOUT = {"soa_cons": 0, "aos_cons": 1, "soa_prim": 2}
MEM_HOST, MEM_DEVICE = 0, 1
F64, F32 = 0, 1

_D = ctypes.c_double
_PD = ctypes.POINTER(ctypes.c_double)
_I = ctypes.c_int
_V = ctypes.c_void_p


class GksError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("gks error %d: %s" % (code, msg))
        self.code = code


class _Grid(ctypes.Structure):
    _fields_ = [("dim", _I), ("n", _I * 3), ("lo", _D * 3), ("hi", _D * 3), ("dx", _PD * 3),
                ("bc", (_I * 2) * 3), ("bc_data", (_PD * 2) * 3), ("wake_cut", _I)]


class _Gas(ctypes.Structure):
    _fields_ = [("gamma", _D), ("mu", _D), ("prandtl", _D), ("T_wall", _D)]


class _Turb(ctypes.Structure):
    _fields_ = [("model", _I), ("C_mu", _D), ("beta_star", _D), ("C_a", _D), ("rarefaction", _I)]


class _Num(ctypes.Structure):
    _fields_ = [("limiter", _I), ("expand", _I), ("precision", _I), ("abar_mode", _I), ("reconstruction", _I)]


_lib = None


def load():
    """Load libgks.so (built in-tree by paper_1302_2132_gb300.build)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError("libgks.so not built: run paper_1302_2132_gb300.build.build() first (%s)" % LIB_PATH)
    L = ctypes.CDLL(LIB_PATH)
    H = _V
    L.gks_create.argtypes = [ctypes.POINTER(_Grid), ctypes.POINTER(_Gas), ctypes.POINTER(_Turb),
                             ctypes.POINTER(_Num), _V, ctypes.POINTER(H)]
    L.gks_set_state.argtypes = [H, _V, _I, _I, _I]
    L.gks_get_state.argtypes = [H, _V, _I, _I, _I]
    L.gks_set_turbulence.argtypes = [H, _V, _V, _I, _I]
    L.gks_set_nodes.argtypes = [H, _V, _I]
    L.gks_steady_create.argtypes = [ctypes.POINTER(_Grid), ctypes.POINTER(_Gas), ctypes.POINTER(_Turb),
                                    ctypes.POINTER(_Num), _PD, _I, _I, _V, ctypes.POINTER(_V)]
    L.gks_steady_set_state.argtypes = [_V, _V, _I, _I, _I]
    L.gks_steady_set_turbulence.argtypes = [_V, _V, _V, _I, _I]
    L.gks_steady_cycles.argtypes = [_V, _I, _D, _D, _PD]
    L.gks_steady_get_turbulence.argtypes = [_V, _V, _V, _I, _I]
    L.gks_steady_residual.argtypes = [_V, _D, _I, _PD, _PD]
    L.gks_steady_get_state.argtypes = [_V, _V, _I, _I, _I]
    L.gks_steady_destroy.argtypes = [_V]
    L.gks_steady_last_error.argtypes = [_V]
    L.gks_steady_last_error.restype = ctypes.c_char_p
    for name in ("gks_steady_create", "gks_steady_set_state", "gks_steady_set_turbulence", "gks_steady_cycles",
                 "gks_steady_residual", "gks_steady_get_state", "gks_steady_destroy", "gks_set_nodes",
                 "gks_steady_set_komega", "gks_steady_get_turbulence"):
        getattr(L, name).restype = _I
    L.gks_compute_dt.argtypes = [H, _D, _PD]
    L.gks_step.argtypes = [H, _D, _D, _I, _D]
    L.gks_get_time.argtypes = [H, _PD, ctypes.POINTER(ctypes.c_longlong)]
    L.gks_set_time.argtypes = [H, _D]
    L.gks_residual.argtypes = [H, _PD, _PD, _PD]
    L.gks_status_word.argtypes = [H, ctypes.POINTER(ctypes.c_uint), _PD]
    L.gks_get_rarefaction.argtypes = [H, _V, _I, _I]
    L.gks_get_tau_turb.argtypes = [H, _V, _I, _I]
    L.gks_komega_defaults.argtypes = [ctypes.POINTER(KOmega)]
    L.gks_set_komega.argtypes = [H, ctypes.POINTER(KOmega)]
    L.gks_get_turbulence.argtypes = [H, _V, _V, _I, _I]
    L.gks_steady_set_komega.argtypes = [_V, ctypes.POINTER(KOmega)]
    L.gks_enable_timing.argtypes = [H, _I]
    L.gks_kernel_time.argtypes = [H, _PD, ctypes.POINTER(ctypes.c_longlong)]
    L.gks_destroy.argtypes = [H]
    L.gks_last_error.argtypes = [H]
    L.gks_last_error.restype = ctypes.c_char_p
    L.gks_face_record_len.argtypes = [_I]
    L.gks_tile_shape.argtypes = [H, ctypes.POINTER(_I), ctypes.POINTER(_I), ctypes.POINTER(_I), ctypes.POINTER(_I)]
    L.gks_tile_shape.restype = _I
    L.gks_probe_alu.argtypes = [_PD, _PD]
    L.gks_probe_alu.restype = _I
    L.gks_probe_alu_packed.argtypes = [_PD]
    L.gks_probe_alu_packed.restype = _I
    L.gks_probe_cvt.argtypes = [_PD, _PD]
    L.gks_probe_cvt.restype = _I
    L.gks_face_op_count.argtypes = [_I, _I, _I, ctypes.POINTER(ctypes.c_longlong)]
    L.gks_face_op_count.restype = _I
    L.gks_cell_op_count.argtypes = [_I, ctypes.POINTER(ctypes.c_longlong)]
    L.gks_cell_op_count.restype = _I
    L.gks_recon_op_count.argtypes = [_I, _I, ctypes.POINTER(ctypes.c_longlong)]
    L.gks_recon_op_count.restype = _I
    L.gks_face_flux.argtypes = [_I, _I, _I, _I, _I, _D, _D, _D, _D, _V, ctypes.c_long, _V, _V, _V]
    for name in ("gks_create", "gks_set_state", "gks_get_state", "gks_set_turbulence", "gks_compute_dt",
                 "gks_step", "gks_get_time", "gks_set_time", "gks_residual", "gks_status_word",
                 "gks_get_rarefaction", "gks_get_tau_turb", "gks_enable_timing", "gks_kernel_time",
                 "gks_destroy", "gks_face_flux", "gks_komega_defaults", "gks_set_komega", "gks_get_turbulence"):
        getattr(L, name).restype = _I
    _lib = L
    return L


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _is_torch(x):
    return type(x).__module__.startswith("torch")


class KOmega(ctypes.Structure):
    """gks_komega: closure coefficients of the k-omega transport (Wilcox 2006 defaults)."""
    _fields_ = [("alpha", ctypes.c_double), ("beta0", ctypes.c_double), ("sigma", ctypes.c_double),
                ("sigma_star", ctypes.c_double), ("sigma_do", ctypes.c_double), ("C_lim", ctypes.c_double),
                ("omega_floor", ctypes.c_double), ("sources", ctypes.c_int), ("diffusion", ctypes.c_int)]


def komega_defaults(**over):
    c = KOmega()
    load().gks_komega_defaults(ctypes.byref(c))
    for k, v in over.items():
        setattr(c, k, v)
    return c


def _structs(dim, n, bc, dx, lo, hi, bc_data, gamma, mu, T_wall, turb_model, C_mu, beta_star, C_a, limiter, expand,
             precision, abar_mode, reconstruction, wake_cut=0, rarefaction="dt"):
    """gks_grid, gks_gas, gks_turb, gks_numerics and the arrays they point to."""
    keep = []
    g = _Grid()
    g.dim = dim
    g.wake_cut = int(wake_cut)
    for d in range(3):
        g.n[d] = n[d] if d < dim else 1
        g.lo[d] = lo[d] if lo is not None and d < dim else 0.0
        g.hi[d] = hi[d] if hi is not None and d < dim else 1.0
    for d in range(dim):
        if dx is not None and dx[d] is not None:
            w = _f64(np.broadcast_to(np.asarray(dx[d], dtype=np.float64), (n[d],)))
            keep.append(w)
            g.dx[d] = w.ctypes.data_as(_PD)
        for s in range(2):
            code = bc[d][s]
            g.bc[d][s] = BC[code] if isinstance(code, str) else int(code)
            if bc_data is not None and bc_data[d][s] is not None:
                a = _f64(bc_data[d][s])
                keep.append(a)
                g.bc_data[d][s] = a.ctypes.data_as(_PD)
    gas = _Gas(gamma, mu, 1.0, T_wall)
    tm = TURB[turb_model] if isinstance(turb_model, str) else int(turb_model)
    turb = _Turb(tm, C_mu, beta_star, C_a,
                 RAREFACTION[rarefaction] if isinstance(rarefaction, str) else int(rarefaction))
    num = _Num(LIMITER[limiter] if isinstance(limiter, str) else int(limiter),
               EXPAND[expand] if isinstance(expand, str) else int(expand),
               PRECISION[precision] if isinstance(precision, str) else int(precision),
               ABAR[abar_mode] if isinstance(abar_mode, str) else int(abar_mode),
               RECON[reconstruction] if isinstance(reconstruction, str) else int(reconstruction))
    return g, gas, turb, num, keep


class Solver:
    """One grid problem on one GPU (see gks_create in include/gks.h for the meaning of each field).

    Arrays passed in may be numpy arrays (host memory) or torch tensors (host or CUDA)."""

    def __init__(self, dim, n, bc, dx=None, lo=None, hi=None, bc_data=None, gamma=1.4, mu=1e-5, T_wall=1.0,
                 turb_model="none", C_mu=0.09, beta_star=0.09, C_a=0.0, limiter="vanleer", expand="multid",
                 precision="fp64", abar_mode="timeint", reconstruction="muscl2", wake_cut=0, stream=None,
                 rarefaction="dt"):
        import torch
        L = load()
        self.dim, self.nv = dim, dim + 2
        self.n = tuple(int(v) for v in n[:dim])
        self.ncell = int(np.prod(self.n))
        g, gas, turb, num, self._keep = _structs(dim, self.n, bc, dx, lo, hi, bc_data, gamma, mu, T_wall, turb_model,
                                                 C_mu, beta_star, C_a, limiter, expand, precision, abar_mode,
                                                 reconstruction, wake_cut, rarefaction)
        self.precision = num.precision
        self.stream = stream if stream is not None else torch.cuda.Stream()
        h = _V()
        st = L.gks_create(ctypes.byref(g), ctypes.byref(gas), ctypes.byref(turb), ctypes.byref(num),
                          _V(self.stream.cuda_stream), ctypes.byref(h))
        self._h = h
        if st != OK:
            msg = L.gks_last_error(h).decode() if h.value else "gks_create failed"
            if h.value:
                L.gks_destroy(h)
            self._h = None
            raise GksError(st, msg)

    # -- helpers -----------------------------------------------------------------------------------
    def _check(self, st):
        if st != OK:
            raise GksError(st, load().gks_last_error(self._h).decode())

    def _ptr(self, x, writable=False):
        """(pointer, memspace, dtype) of a numpy array or torch tensor; keeps a reference."""
        if _is_torch(x):
            import torch
            assert x.is_contiguous()
            dt = {torch.float64: F64, torch.float32: F32}[x.dtype]
            mem = MEM_DEVICE if x.is_cuda else MEM_HOST
            if x.is_cuda:
                self.stream.wait_stream(torch.cuda.current_stream(x.device))
            return _V(x.data_ptr()), mem, dt
        a = np.asarray(x)
        if not writable:
            a = np.ascontiguousarray(a)
        dt = {np.dtype(np.float64): F64, np.dtype(np.float32): F32}[a.dtype]
        self._keep_tmp = a
        return _V(a.ctypes.data), MEM_HOST, dt

    def _after_device_write(self, x):
        if _is_torch(x) and x.is_cuda:
            import torch
            torch.cuda.current_stream(x.device).wait_stream(self.stream)

    # -- API ---------------------------------------------------------------------------------------
    def set_state(self, W, layout="soa_cons"):
        p, mem, dt = self._ptr(W)
        self._check(load().gks_set_state(self._h, p, LAYOUT[layout], mem, dt))
        if mem == MEM_HOST:
            self.stream.synchronize()  # the host buffer may be reused by the caller

    def set_turbulence(self, f1, f2=None):
        p1, mem, dt = self._ptr(f1)
        keep = self._keep_tmp if not _is_torch(f1) else f1
        p2 = None
        if f2 is not None:
            p2, mem2, dt2 = self._ptr(f2)
            assert (mem2, dt2) == (mem, dt)
        self._check(load().gks_set_turbulence(self._h, p1, p2, mem, dt))
        del keep
        self.stream.synchronize()

    def set_nodes(self, nodes):
        """Make the grid body-fitted: nodes[(n1 + 1), (n0 + 1), 2] = (x, y), double, host array or
        CUDA tensor (2D, directional expansion, MUSCL2)."""
        if _is_torch(nodes):
            assert nodes.dtype.is_floating_point and nodes.element_size() == 8
        else:
            nodes = np.ascontiguousarray(nodes, dtype=np.float64)
        p, mem, dt = self._ptr(nodes)
        assert dt == F64
        n0, n1 = self.n[0], self.n[1]
        assert int(np.prod(nodes.shape)) == 2 * (n0 + 1) * (n1 + 1)
        self._check(load().gks_set_nodes(self._h, p, mem))
        self.stream.synchronize()

    def get_state(self, layout="soa_cons", out=None, dtype=np.float64):
        if out is None:
            out = np.zeros(self.nv * self.ncell, dtype=dtype)
        p, mem, dt = self._ptr(out, writable=True)
        self._check(load().gks_get_state(self._h, p, LAYOUT[layout], mem, dt))
        self._after_device_write(out)
        return out

    def compute_dt(self, cfl):
        v = _D()
        self._check(load().gks_compute_dt(self._h, cfl, ctypes.byref(v)))
        return v.value

    def step(self, nsteps=1, dt=0.0, cfl=0.5, t_end=0.0):
        self._check(load().gks_step(self._h, dt, cfl, int(nsteps), t_end))

    def time(self):
        t, s = _D(), ctypes.c_longlong()
        self._check(load().gks_get_time(self._h, ctypes.byref(t), ctypes.byref(s)))
        return t.value, s.value

    def set_time(self, t):
        self._check(load().gks_set_time(self._h, t))

    def residual(self):
        l2, li, tot = (np.zeros(self.nv) for _ in range(3))
        self._check(load().gks_residual(self._h, l2.ctypes.data_as(_PD), li.ctypes.data_as(_PD),
                                        tot.ctypes.data_as(_PD)))
        return l2, li, tot

    def status_word(self):
        b, d = ctypes.c_uint(), _D()
        self._check(load().gks_status_word(self._h, ctypes.byref(b), ctypes.byref(d)))
        return b.value, d.value

    def rarefaction(self, out=None):
        if out is None:
            out = np.zeros(self.ncell)
        p, mem, dt = self._ptr(out, writable=True)
        self._check(load().gks_get_rarefaction(self._h, p, mem, dt))
        self._after_device_write(out)
        return out

    def set_komega(self, **coeffs):
        """Closure coefficients of the k-omega transport (keywords of gks_komega)."""
        self._check(load().gks_set_komega(self._h, ctypes.byref(komega_defaults(**coeffs))))

    def get_turbulence(self, k_out=None, omega_out=None):
        """Transported k and omega (k-omega transport handles)."""
        if k_out is None:
            k_out = np.zeros(self.ncell)
        if omega_out is None:
            omega_out = np.zeros(self.ncell)
        pk, mem, dt = self._ptr(k_out, writable=True)
        pw, mem2, dt2 = self._ptr(omega_out, writable=True)
        assert (mem, dt) == (mem2, dt2)
        self._check(load().gks_get_turbulence(self._h, pk, pw, mem, dt))
        self._after_device_write(k_out)
        self._after_device_write(omega_out)
        return k_out, omega_out

    def tau_turb(self, out=None):
        if out is None:
            out = np.zeros(self.ncell)
        p, mem, dt = self._ptr(out, writable=True)
        self._check(load().gks_get_tau_turb(self._h, p, mem, dt))
        self._after_device_write(out)
        return out

    def enable_timing(self, on=True):
        self._check(load().gks_enable_timing(self._h, int(on)))

    def kernel_time(self):
        ms, n = _D(), ctypes.c_longlong()
        self._check(load().gks_kernel_time(self._h, ctypes.byref(ms), ctypes.byref(n)))
        return ms.value, n.value

    def tile_shape(self):
        """(variant, tx, ty, tz) of the step kernel's tile (2D FP32: chosen by the autotuner)."""
        v, x, y, z = _I(), _I(), _I(), _I()
        self._check(load().gks_tile_shape(self._h, ctypes.byref(v), ctypes.byref(x), ctypes.byref(y), ctypes.byref(z)))
        return v.value, x.value, y.value, z.value

    def close(self):
        if self._h is not None:
            load().gks_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def probe_alu():
    """Measured FP32 and FP64 FMA throughput of the current device, TFLOP/s."""
    a, b = _D(), _D()
    st = load().gks_probe_alu(ctypes.byref(a), ctypes.byref(b))
    if st != OK:
        raise GksError(st, "gks_probe_alu failed")
    return a.value, b.value


def probe_alu_packed():
    """Measured throughput of the paired FP32 FMA (two FMAs per thread instruction), TFLOP/s."""
    a = _D()
    st = load().gks_probe_alu_packed(ctypes.byref(a))
    if st != OK:
        raise GksError(st, "gks_probe_alu_packed failed")
    return a.value

def probe_cvt():
    """(double -> float, float -> double) conversions per second of the current device, in 1e9/s."""
    a, b = ctypes.c_double(), ctypes.c_double()
    st = load().gks_probe_cvt(ctypes.byref(a), ctypes.byref(b))
    if st != OK:
        raise GksError(st, "gks_probe_cvt failed")
    return a.value, b.value


def face_op_count(dim, expand=True, with_recon=True):
    """Static per-face operation count of the flux code: (add, mul, div, sqrt, exp, erfc)."""
    c = (ctypes.c_longlong * 6)()
    load().gks_face_op_count(dim, int(expand), int(with_recon), c)
    return tuple(c)


def cell_op_count(dim):
    """Static per-cell operation count of the reconstruction slopes: (add, mul, div, sqrt, exp, erfc)."""
    c = (ctypes.c_longlong * 6)()
    load().gks_cell_op_count(dim, c)
    return tuple(c)


def recon_op_count(dim, reconstruction):
    """Static per-face operation count of a higher-order reconstruction's face values and slopes."""
    c = (ctypes.c_longlong * 6)()
    r = RECON[reconstruction] if isinstance(reconstruction, str) else int(reconstruction)
    if r == 0:
        return (0,) * 6
    load().gks_recon_op_count(dim, r, c)
    return tuple(c)


def face_record_len(dim):
    return load().gks_face_record_len(dim)


def face_flux(dim, faces, dt, gamma=1.4, mu=1e-5, C_a=0.0, precision="fp64", expand="multid",
              abar_mode="timeint", stream=None, rarefaction="dt"):
    """Evaluate interface fluxes for face records held in a CUDA float64 tensor
    [nfaces, face_record_len(dim)]; returns (F [nfaces, dim+2], tau [nfaces]) as CUDA tensors."""
    import torch
    assert faces.is_cuda and faces.dtype == torch.float64 and faces.is_contiguous()
    nf = faces.shape[0]
    F = torch.empty((nf, dim + 2), dtype=torch.float64, device=faces.device)
    tau = torch.empty((nf,), dtype=torch.float64, device=faces.device)
    s = stream if stream is not None else torch.cuda.current_stream(faces.device)
    st = load().gks_face_flux(dim, PRECISION[precision], EXPAND[expand], ABAR[abar_mode], RAREFACTION[rarefaction],
                              gamma, mu, C_a, dt,
                              _V(faces.data_ptr()), nf, _V(F.data_ptr()), _V(tau.data_ptr()),
                              _V(s.cuda_stream))
    if st != OK:
        raise GksError(st, "gks_face_flux failed")
    return F, tau


class SteadySolver:
    """Steady-state solver on a body-fitted 2D grid: local time stepping, LU-SGS smoothing and FAS
    multigrid (gks_steady_* in include/gks.h).  nodes[(n1 + 1), (n0 + 1), 2] (host)."""

    def __init__(self, n, bc, nodes, levels=4, bc_data=None, gamma=1.4, mu=1e-5, T_wall=1.0, turb_model="none",
                 C_mu=0.09, beta_star=0.09, C_a=0.0, limiter="vanleer", precision="fp64", lusgs_tile=16, wake_cut=0,
                 expand="directional", stream=None, reconstruction="muscl2", rarefaction="dt"):
        import torch
        L = load()
        self.n = (int(n[0]), int(n[1]))
        self.nv = 4
        self.ncell = self.n[0] * self.n[1]
        dx = [np.ones(self.n[0]), np.ones(self.n[1])]
        g, gas, turb, num, self._keep = _structs(2, self.n, bc, dx, None, None, bc_data, gamma, mu, T_wall, turb_model,
                                                 C_mu, beta_star, C_a, limiter, expand, precision, "timeint",
                                                 reconstruction, wake_cut, rarefaction)
        nodes = _f64(nodes)
        assert nodes.size == 2 * (self.n[0] + 1) * (self.n[1] + 1)
        self.stream = stream if stream is not None else torch.cuda.Stream()
        h = _V()
        st = L.gks_steady_create(ctypes.byref(g), ctypes.byref(gas), ctypes.byref(turb), ctypes.byref(num),
                                 nodes.ctypes.data_as(_PD), int(levels), int(lusgs_tile), _V(self.stream.cuda_stream),
                                 ctypes.byref(h))
        self._h = h if st == OK else None
        if st != OK:
            raise GksError(st, "gks_steady_create failed")

    def _check(self, st):
        if st != OK:
            raise GksError(st, load().gks_steady_last_error(self._h).decode())

    def set_state(self, W, layout="soa_cons"):
        """W: numpy array or torch tensor (host or CUDA, float64 or float32)."""
        if _is_torch(W):
            import torch
            assert W.is_contiguous()
            dt = {torch.float64: F64, torch.float32: F32}[W.dtype]
            if W.is_cuda:
                self.stream.wait_stream(torch.cuda.current_stream(W.device))
            self._check(load().gks_steady_set_state(self._h, _V(W.data_ptr()), LAYOUT[layout],
                                                    MEM_DEVICE if W.is_cuda else MEM_HOST, dt))
            return
        a = _f64(W)
        self._check(load().gks_steady_set_state(self._h, _V(a.ctypes.data), LAYOUT[layout], MEM_HOST, F64))
        self.stream.synchronize()

    def set_turbulence(self, f1, f2=None):
        """f1, f2: numpy arrays or torch tensors (host or CUDA, float64), one value per cell."""
        if _is_torch(f1):
            import torch
            assert f1.dtype == torch.float64 and (f2 is None or f2.dtype == torch.float64)
            if f1.is_cuda:
                self.stream.wait_stream(torch.cuda.current_stream(f1.device))
            self._check(load().gks_steady_set_turbulence(self._h, _V(f1.data_ptr()),
                                                         _V(f2.data_ptr()) if f2 is not None else None,
                                                         MEM_DEVICE if f1.is_cuda else MEM_HOST, F64))
            return
        a = _f64(f1)
        b = _f64(f2) if f2 is not None else None
        self._check(load().gks_steady_set_turbulence(self._h, _V(a.ctypes.data), _V(b.ctypes.data) if b is not None
                                                     else None, MEM_HOST, F64))

    def set_komega(self, **coeffs):
        """Closure coefficients of the steady k-omega transport (keywords of gks_komega)."""
        self._check(load().gks_steady_set_komega(self._h, ctypes.byref(komega_defaults(**coeffs))))

    def get_turbulence(self):
        """k and omega of the current state (k-omega transport handles), host float64."""
        k, om = np.zeros(self.ncell), np.zeros(self.ncell)
        self._check(load().gks_steady_get_turbulence(self._h, _V(k.ctypes.data), _V(om.ctypes.data), MEM_HOST, F64))
        return k, om

    def cycles(self, ncycles, cfl, cfl_flux=0.5):
        """Run ncycles multigrid cycles; returns the fine residual norm before each."""
        res = np.zeros(max(int(ncycles), 1))
        self._check(load().gks_steady_cycles(self._h, int(ncycles), cfl, cfl_flux, res.ctypes.data_as(_PD)))
        return res[:ncycles]

    def residual(self, cfl_flux=0.5, first_order=False):
        dt = np.zeros(self.ncell)
        R = np.zeros(4 * self.ncell)
        self._check(load().gks_steady_residual(self._h, cfl_flux, int(first_order), dt.ctypes.data_as(_PD),
                                               R.ctypes.data_as(_PD)))
        return dt, R

    def get_state(self, layout="soa_cons"):
        out = np.zeros(4 * self.ncell)
        self._check(load().gks_steady_get_state(self._h, _V(out.ctypes.data), LAYOUT[layout], MEM_HOST, F64))
        return out

    def close(self):
        if self._h is not None:
            load().gks_steady_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
