"""The C ABI library loads and exports every entry point declared in include/gks.h (no GPU)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            text = open(os.path.join(ROOT, "include", fn)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names.update(re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\*?\s*(gks_[a-z0-9_]+)\s*\(", text, re.M))
    return sorted(names)


def test_header_declares_the_boundary():
    names = declared_symbols()
    for n in ("gks_create", "gks_set_state", "gks_compute_dt", "gks_step", "gks_get_state", "gks_residual",
              "gks_set_turbulence", "gks_get_rarefaction", "gks_destroy", "gks_last_error", "gks_face_flux"):
        assert n in names


def test_library_exports_every_declared_symbol():
    from paper_1302_2132_gb300 import build
    lib = build.build()
    L = ctypes.CDLL(lib)
    missing = [n for n in declared_symbols() if not hasattr(L, n)]
    assert not missing, missing


def test_binding_fails_loudly_without_library(tmp_path, monkeypatch):
    from paper_1302_2132_gb300 import gks
    monkeypatch.setattr(gks, "LIB_PATH", str(tmp_path / "missing.so"))
    monkeypatch.setattr(gks, "_lib", None)
    with pytest.raises(ImportError):
        gks.load()


def test_face_record_length():
    from paper_1302_2132_gb300 import build, gks
    build.build()
    gks.load()
    assert [gks.face_record_len(d) for d in (1, 2, 3)] == [21, 35, 53]


def test_null_handles_are_rejected_without_touching_the_device():
    """Entry points of the steady solver, the k-omega transport and the body-fitted grids return
    GKS_EINVAL for null handles or arguments before any CUDA call (so this runs without a GPU)."""
    from paper_1302_2132_gb300 import build
    L = ctypes.CDLL(build.build())
    EINVAL = 1
    V = ctypes.c_void_p
    L.gks_steady_set_komega.argtypes = [V, V]
    L.gks_steady_get_turbulence.argtypes = [V, V, V, ctypes.c_int, ctypes.c_int]
    L.gks_steady_cycles.argtypes = [V, ctypes.c_int, ctypes.c_double, ctypes.c_double, V]
    L.gks_steady_residual.argtypes = [V, ctypes.c_double, ctypes.c_int, V, V]
    L.gks_set_nodes.argtypes = [V, V, ctypes.c_int]
    L.gks_get_turbulence.argtypes = [V, V, V, ctypes.c_int, ctypes.c_int]
    L.gks_komega_defaults.argtypes = [V]
    assert L.gks_steady_set_komega(None, None) == EINVAL
    assert L.gks_steady_get_turbulence(None, None, None, 0, 0) == EINVAL
    assert L.gks_steady_cycles(None, 1, 1.0, 0.5, None) == EINVAL
    assert L.gks_steady_residual(None, 0.5, 0, None, None) == EINVAL
    assert L.gks_set_nodes(None, None, 0) == EINVAL
    assert L.gks_get_turbulence(None, None, None, 0, 0) == EINVAL
    assert L.gks_komega_defaults(None) == EINVAL


def test_create_rejects_bad_sizes_before_touching_the_device():
    """gks_create refuses a grid of more than GKS_MAX_CELLS cells (among them one whose cell count
    would wrap a 64-bit product) and an axis of fewer than two cells, with a message, before any
    CUDA call (so this runs without a GPU); the returned handle is released by gks_destroy."""
    from paper_1302_2132_gb300 import build, gks
    build.build()
    L = gks.load()
    EINVAL = 1
    cases = [((1 << 22, 1 << 22, 1 << 21), "GKS_MAX_CELLS"),   # 2^65 cells: wraps to 0 in 64 bits
             ((1 << 30, 1 << 30, 16), "GKS_MAX_CELLS"),
             ((1 << 17, 1 << 17, 2), "GKS_MAX_CELLS"),        # 2^35
             ((1 << 17, 1 << 16, 1), "two cells")]            # third axis active with one cell
    for n, msg in cases:
        g = gks._Grid()
        g.dim = 3
        for d in range(3):
            g.n[d] = n[d]
            g.lo[d], g.hi[d] = 0.0, 1.0
        gas = gks._Gas(1.4, 1e-5, 1.0, 1.0)
        turb = gks._Turb(0, 0.09, 0.09, 0.0, 0)
        num = gks._Num(1, 1, 0, 0, 0)
        h = ctypes.c_void_p()
        st = L.gks_create(ctypes.byref(g), ctypes.byref(gas), ctypes.byref(turb), ctypes.byref(num), None,
                          ctypes.byref(h))
        assert st == EINVAL and h.value
        assert msg in L.gks_last_error(h).decode()
        assert L.gks_destroy(h) == 0
    header = open(os.path.join(ROOT, "include", "gks.h")).read()
    assert "#define GKS_MAX_CELLS (1LL << 34)" in header


def comment_before(text, pos):
    """The last /* ... */ block that ends before pos."""
    end = text.rfind("*/", 0, pos)
    start = text.rfind("/*", 0, end)
    return text[start:end + 2] if start >= 0 and end >= 0 else ""


def test_every_call_cites_its_passage_or_has_no_counterpart():
    """Each declaration's comment names the section or equation of the paper that defines the
    operation, or says that the paper has no counterpart (resource management, diagnostics)."""
    text = open(os.path.join(ROOT, "include", "gks.h")).read()
    bad = []
    for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\*?\s*(gks_[a-z0-9_]+)\s*\(", text, re.M):
        c = re.sub(r"\s*\n\s*\*?\s*", " ", comment_before(text, m.start()))
        if not re.search(r"Section \d|Eqs?\. [a-z]|Table \d|no paper counterpart|paper has no counterpart", c, re.I):
            bad.append(m.group(1))
    assert not bad, bad


def test_binding_structs_match_the_header_layout(tmp_path):
    """Offsets and sizes of the boundary's structs, compiled from include/gks.h with the host compiler,
    equal those of the ctypes binding (gks_turb carries the rarefaction option)."""
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no host C compiler")
    from paper_1302_2132_gb300 import gks
    fields = {"gks_turb": (gks._Turb, ["model", "C_mu", "beta_star", "C_a", "rarefaction"]),
              "gks_gas": (gks._Gas, ["gamma", "mu", "prandtl", "T_wall"]),
              "gks_numerics": (gks._Num, ["limiter", "expand", "precision", "abar_mode", "reconstruction"]),
              "gks_grid": (gks._Grid, ["dim", "n", "lo", "hi", "dx", "bc", "bc_data", "wake_cut"])}
    src = ['#include <stdio.h>', '#include <stddef.h>', '#include "gks.h"', "int main(void) {"]
    for st, (_, names) in fields.items():
        src.append('printf("%s %%zu\\n", sizeof(%s));' % (st, st))
        for n in names:
            src.append('printf("%s.%s %%zu\\n", offsetof(%s, %s));' % (st, n, st, n))
    src.append('printf("GKS_RAR_TAUHAT %d\\n", GKS_RAR_TAUHAT); return 0; }')
    c = tmp_path / "layout.c"
    c.write_text("\n".join(src))
    exe = tmp_path / "layout"
    subprocess.check_call([cc, "-I", os.path.join(ROOT, "include"), str(c), "-o", str(exe)])
    out = dict(line.split() for line in subprocess.check_output([str(exe)], text=True).splitlines())
    for st, (cls, names) in fields.items():
        assert int(out[st]) == ctypes.sizeof(cls), st
        for n in names:
            assert int(out["%s.%s" % (st, n)]) == getattr(cls, n).offset, (st, n)
    assert int(out["GKS_RAR_TAUHAT"]) == gks.RAREFACTION["tauhat"]
