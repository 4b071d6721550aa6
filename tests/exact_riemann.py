"""Exact solution of the 1D Riemann problem for an ideal gas (test pin, not part of the library).

Textbook construction (Toro, "Riemann Solvers and Numerical Methods for Fluid Dynamics", ch. 4):
the star pressure solves f_L(p) + f_R(p) + (u_R - u_L) = 0, with f_K the shock (Rankine-Hugoniot)
or rarefaction (isentropic) branch, found by Newton's method; the solution is then sampled on x/t.
"""
import numpy as np


def _fK(p, rho, pK, cK, g):
    if p > pK:  # shock
        A = 2.0 / ((g + 1.0) * rho)
        B = (g - 1.0) / (g + 1.0) * pK
        s = np.sqrt(A / (p + B))
        f = (p - pK) * s
        df = s * (1.0 - 0.5 * (p - pK) / (B + p))
    else:  # rarefaction
        f = 2.0 * cK / (g - 1.0) * ((p / pK) ** ((g - 1.0) / (2.0 * g)) - 1.0)
        df = 1.0 / (rho * cK) * (p / pK) ** (-(g + 1.0) / (2.0 * g))
    return f, df


def star_state(left, right, g=1.4, tol=1e-15):
    rL, uL, pL = left
    rR, uR, pR = right
    cL, cR = np.sqrt(g * pL / rL), np.sqrt(g * pR / rR)
    p = max(tol, 0.5 * (pL + pR))
    for _ in range(200):
        fL, dL = _fK(p, rL, pL, cL, g)
        fR, dR = _fK(p, rR, pR, cR, g)
        dp = (fL + fR + uR - uL) / (dL + dR)
        pn = max(tol, p - dp)
        if abs(pn - p) < tol * 0.5 * (pn + p):
            p = pn
            break
        p = pn
    fL, _ = _fK(p, rL, pL, cL, g)
    fR, _ = _fK(p, rR, pR, cR, g)
    u = 0.5 * (uL + uR) + 0.5 * (fR - fL)
    return p, u


def sample(left, right, xi, g=1.4):
    """Primitive (rho, u, p) at similarity coordinates xi = (x - x0)/t."""
    rL, uL, pL = left
    rR, uR, pR = right
    cL, cR = np.sqrt(g * pL / rL), np.sqrt(g * pR / rR)
    ps, us = star_state(left, right, g)
    out = np.zeros((3, len(xi)))
    for i, s in enumerate(xi):
        if s <= us:  # left of contact
            if ps > pL:
                SL = uL - cL * np.sqrt((g + 1) / (2 * g) * ps / pL + (g - 1) / (2 * g))
                if s <= SL:
                    out[:, i] = (rL, uL, pL)
                else:
                    r = rL * (ps / pL + (g - 1) / (g + 1)) / ((g - 1) / (g + 1) * ps / pL + 1)
                    out[:, i] = (r, us, ps)
            else:
                SHL = uL - cL
                csL = cL * (ps / pL) ** ((g - 1) / (2 * g))
                STL = us - csL
                if s <= SHL:
                    out[:, i] = (rL, uL, pL)
                elif s >= STL:
                    out[:, i] = (rL * (ps / pL) ** (1 / g), us, ps)
                else:
                    u = 2 / (g + 1) * (cL + (g - 1) / 2 * uL + s)
                    c = 2 / (g + 1) * (cL + (g - 1) / 2 * (uL - s))
                    r = rL * (c / cL) ** (2 / (g - 1))
                    out[:, i] = (r, u, pL * (c / cL) ** (2 * g / (g - 1)))
        else:
            if ps > pR:
                SR = uR + cR * np.sqrt((g + 1) / (2 * g) * ps / pR + (g - 1) / (2 * g))
                if s >= SR:
                    out[:, i] = (rR, uR, pR)
                else:
                    r = rR * (ps / pR + (g - 1) / (g + 1)) / ((g - 1) / (g + 1) * ps / pR + 1)
                    out[:, i] = (r, us, ps)
            else:
                SHR = uR + cR
                csR = cR * (ps / pR) ** ((g - 1) / (2 * g))
                STR = us + csR
                if s >= SHR:
                    out[:, i] = (rR, uR, pR)
                elif s <= STR:
                    out[:, i] = (rR * (ps / pR) ** (1 / g), us, ps)
                else:
                    u = 2 / (g + 1) * (-cR + (g - 1) / 2 * uR + s)
                    c = 2 / (g + 1) * (cR - (g - 1) / 2 * (uR - s))
                    r = rR * (c / cR) ** (2 / (g - 1))
                    out[:, i] = (r, u, pR * (c / cR) ** (2 * g / (g - 1)))
    return out


def cell_average(left, right, edges, t, x0=0.5, g=1.4, sub=64):
    """Cell averages of the exact primitive solution over cells [edges[i], edges[i+1]]."""
    n = len(edges) - 1
    out = np.zeros((3, n))
    gx, gw = np.polynomial.legendre.leggauss(8)
    for i in range(n):
        a, b = edges[i], edges[i + 1]
        h = (b - a) / sub
        xs, ws = [], []
        for k in range(sub):
            lo = a + k * h
            xs.append(lo + 0.5 * h * (gx + 1))
            ws.append(0.5 * h * gw)
        xs = np.concatenate(xs)
        ws = np.concatenate(ws)
        vals = sample(left, right, (xs - x0) / t, g)
        out[:, i] = vals @ ws / (b - a)
    return out
