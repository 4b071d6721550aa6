"""Stored expected values under tests/golden/: the number the paper prints for the hot path (C_mu),
checked against the defaults of the library's binding and of the oracle, and the FP64 oracle's fluxes
of fixed faces (written by tests/golden/make_golden.py, which calls only the oracle), recomputed so
that any later change to the oracle's arithmetic shows here."""
import importlib.util
import inspect
import json
import os

import numpy as np
import pytest

import oracle

GOLD = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def load_maker():
    spec = importlib.util.spec_from_file_location("make_golden", os.path.join(GOLD, "make_golden.py"))
    m = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(m)
    return m


def golden_faces():
    with open(os.path.join(GOLD, "oracle_face_flux.jsonl")) as f:
        return [json.loads(line) for line in f if line.strip() and not line.startswith("#")]


def paper_constants():
    out = {}
    with open(os.path.join(GOLD, "paper_constants.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                name, value = line.split()[:2]
                out[name] = float(value)
    return out


def test_paper_constants_are_the_defaults():
    from paper_1302_2132_gb300 import gks
    c = paper_constants()
    assert c == {"C_mu": 0.09}
    for fn in (gks.Solver.__init__, gks.SteadySolver.__init__, oracle.Case.__init__):
        assert inspect.signature(fn).parameters["C_mu"].default == c["C_mu"]


def test_golden_file_covers_every_dimension_expansion_and_regime():
    recs = golden_faces()
    assert len(recs) == 25
    seen = {(r["D"], r["multid"], r["tau_t"]) for r in recs}
    for D in (1, 2, 3):
        for multid in ((0,) if D == 1 else (0, 1)):
            for tau_t in (0.0, 1e-7, 3e-4, 5e-2, 1e3):
                assert (D, multid, tau_t) in seen


@pytest.mark.parametrize("i", range(25))
def test_oracle_reproduces_the_stored_fluxes(i):
    rec = golden_faces()[i]
    maker = load_maker()
    F, dg = oracle.face_flux(rec["D"], rec["gamma"], rec["mu"], rec["C_a"], rec["dt"], maker.face_of(rec),
                             multid=rec["multid"], abar_mode=rec["abar_mode"], diag=True)
    Fs = np.asarray(rec["F"])
    assert np.linalg.norm(np.asarray(F) - Fs) <= 1e-12 * np.linalg.norm(Fs), (F, Fs)
    assert abs(dg.tau - rec["tau"]) <= 1e-14 * rec["tau"]
