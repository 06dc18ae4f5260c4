"""Exact solution of the Riemann problem for the ideal-gas Euler equations.

Test helper, independent of the oracle: the star pressure solves
f_L(p) + f_R(p) + (u_R - u_L) = 0 (shock branch from the Rankine-Hugoniot
relations, rarefaction branch from the isentropic Riemann invariants), and the
solution is sampled along x/t (textbook construction, e.g. Toro, 'Riemann Solvers
and Numerical Methods for Fluid Dynamics', ch. 4).
"""
from __future__ import annotations

import math

import numpy as np


def _f_and_df(p, rho, pK, cK, g):
    if p > pK:   # shock
        A = 2.0 / ((g + 1.0) * rho)
        B = (g - 1.0) / (g + 1.0) * pK
        s = math.sqrt(A / (p + B))
        return (p - pK) * s, s * (1.0 - 0.5 * (p - pK) / (p + B))
    # rarefaction
    e = (g - 1.0) / (2.0 * g)
    f = 2.0 * cK / (g - 1.0) * ((p / pK) ** e - 1.0)
    df = 1.0 / (rho * cK) * (p / pK) ** (-(g + 1.0) / (2.0 * g))
    return f, df


def star_state(rL, uL, pL, rR, uR, pR, g):
    """(p*, u*) of the Riemann problem."""
    cL, cR = math.sqrt(g * pL / rL), math.sqrt(g * pR / rR)
    p = max(1e-12, 0.5 * (pL + pR))
    # two-rarefaction guess is robust for all three classical tubes
    e = (g - 1.0) / (2.0 * g)
    num = cL + cR - 0.5 * (g - 1.0) * (uR - uL)
    if num > 0:
        p = (num / (cL / pL ** e + cR / pR ** e)) ** (1.0 / e)
    for _ in range(200):
        fL, dL = _f_and_df(p, rL, pL, cL, g)
        fR, dR = _f_and_df(p, rR, pR, cR, g)
        f = fL + fR + uR - uL
        dp = f / (dL + dR)
        pn = max(p - dp, 1e-14 * p)
        if abs(pn - p) <= 1e-15 * (pn + p):
            p = pn
            break
        p = pn
    fL, _ = _f_and_df(p, rL, pL, cL, g)
    fR, _ = _f_and_df(p, rR, pR, cR, g)
    return p, 0.5 * (uL + uR) + 0.5 * (fR - fL)


def sample(S, rL, uL, pL, rR, uR, pR, g):
    """Density, velocity and pressure at similarity coordinates S = (x - x0)/t."""
    ps, us = star_state(rL, uL, pL, rR, uR, pR, g)
    cL, cR = math.sqrt(g * pL / rL), math.sqrt(g * pR / rR)
    gm, gp = (g - 1.0) / (g + 1.0), (g + 1.0) / (2.0 * g)
    S = np.asarray(S, dtype=np.float64)
    rho, u, p = np.empty_like(S), np.empty_like(S), np.empty_like(S)
    for idx, s in np.ndenumerate(S):
        if s <= us:   # left of the contact
            if ps > pL:
                rs = rL * (ps / pL + gm) / (gm * ps / pL + 1.0)
                SL = uL - cL * math.sqrt(gp * ps / pL + (g - 1.0) / (2.0 * g))
                val = (rL, uL, pL) if s < SL else (rs, us, ps)
            else:
                rs = rL * (ps / pL) ** (1.0 / g)
                cs = cL * (ps / pL) ** ((g - 1.0) / (2.0 * g))
                if s < uL - cL:
                    val = (rL, uL, pL)
                elif s > us - cs:
                    val = (rs, us, ps)
                else:
                    c = 2.0 / (g + 1.0) * (cL + 0.5 * (g - 1.0) * (uL - s))
                    uu = 2.0 / (g + 1.0) * (cL + 0.5 * (g - 1.0) * uL + s)
                    val = (rL * (c / cL) ** (2.0 / (g - 1.0)), uu, pL * (c / cL) ** (2.0 * g / (g - 1.0)))
        else:         # right of the contact
            if ps > pR:
                rs = rR * (ps / pR + gm) / (gm * ps / pR + 1.0)
                SR = uR + cR * math.sqrt(gp * ps / pR + (g - 1.0) / (2.0 * g))
                val = (rR, uR, pR) if s > SR else (rs, us, ps)
            else:
                rs = rR * (ps / pR) ** (1.0 / g)
                cs = cR * (ps / pR) ** ((g - 1.0) / (2.0 * g))
                if s > uR + cR:
                    val = (rR, uR, pR)
                elif s < us + cs:
                    val = (rs, us, ps)
                else:
                    c = 2.0 / (g + 1.0) * (cR - 0.5 * (g - 1.0) * (uR - s))
                    uu = 2.0 / (g + 1.0) * (-cR + 0.5 * (g - 1.0) * uR + s)
                    val = (rR * (c / cR) ** (2.0 / (g - 1.0)), uu, pR * (c / cR) ** (2.0 * g / (g - 1.0)))
        rho[idx], u[idx], p[idx] = val
    return rho, u, p
