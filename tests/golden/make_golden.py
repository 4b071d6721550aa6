"""Writes oracle_face_flux.jsonl: the FP64 oracle's time-integrated interface flux (Eqs. resultingf,
fluxesf; relaxation time of Eqs. relaxation time and taua) of fixed faces in 1D, 2D and 3D, both
expansions, the relaxation time from equilibrium (tau_t = 0) to near-free transport.  The paper prints
no worked example of the flux, so these values are the oracle's, kept so that a later change to the
oracle's arithmetic shows in test_golden.py.  Calls only the oracle.  From the repository root:

    python tests/golden/make_golden.py
"""
import json
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))
import oracle  # noqa: E402

GAMMA, MU, C_A, DT = 1.4, 2e-5, 0.4, 1e-3


def cons(D, rho, U, p):
    U = np.asarray(U, dtype=float)
    return np.concatenate([[rho], rho * U, [p / (GAMMA - 1.0) + 0.5 * rho * np.dot(U, U)]])


def cases():
    rng = np.random.default_rng(1302)
    for D in (1, 2, 3):
        nv = D + 2
        for multid in ((0,) if D == 1 else (0, 1)):
            for tau_t in (0.0, 1e-7, 3e-4, 5e-2, 1e3):
                wl = cons(D, rng.uniform(0.3, 2.0), rng.uniform(-1.5, 1.5, D), rng.uniform(0.2, 2.0))
                wr = cons(D, rng.uniform(0.3, 2.0), rng.uniform(-1.5, 1.5, D), rng.uniform(0.2, 2.0))
                h = rng.uniform(0.002, 0.05)
                sl, sr = rng.normal(size=nv), rng.normal(size=nv)
                cl, cr = wl - 0.5 * h * sl, wr + 0.5 * h * sr
                tl, tr = rng.normal(size=(D - 1, nv)), rng.normal(size=(D - 1, nv))
                yield dict(D=D, multid=multid, abar_mode=0, gamma=GAMMA, mu=MU, C_a=C_A, dt=DT, wl=wl, wr=wr,
                           cl=cl, cr=cr, sl=sl, sr=sr, tl=tl, tr=tr, dxl=0.5 * h, dxr=0.5 * h, tau_t=tau_t)


def face_of(c):
    return oracle.make_face(c["D"], np.asarray(c["wl"]), np.asarray(c["wr"]), np.asarray(c["cl"]),
                            np.asarray(c["cr"]), np.asarray(c["sl"]), np.asarray(c["sr"]),
                            np.asarray(c["tl"], dtype=float).reshape(c["D"] - 1, c["D"] + 2),
                            np.asarray(c["tr"], dtype=float).reshape(c["D"] - 1, c["D"] + 2),
                            c["dxl"], c["dxr"], c["tau_t"])


def main():
    path = os.path.join(HERE, "oracle_face_flux.jsonl")
    with open(path, "w") as f:
        f.write("# FP64 oracle interface fluxes (Eqs. resultingf, fluxesf), written by make_golden.py; one face per\n"
                "# line: inputs in the face frame (conservative states, cell averages, normal and tangential\n"
                "# slopes, centre-to-face distances, tau_t) and the flux F with the face relaxation time tau.\n")
        for c in cases():
            F, dg = oracle.face_flux(c["D"], c["gamma"], c["mu"], c["C_a"], c["dt"], face_of(c), multid=c["multid"],
                                     abar_mode=c["abar_mode"], diag=True)
            rec = {k: (v.tolist() if isinstance(v, np.ndarray) else v) for k, v in c.items()}
            rec["F"] = np.asarray(F).tolist()
            rec["tau"] = float(dg.tau)
            f.write(json.dumps(rec) + "\n")
    print("wrote", path)


if __name__ == "__main__":
    main()
