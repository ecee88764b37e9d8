"""Exact solution of the 1D Riemann problem for an ideal gas (test infrastructure).

Used to compare shock-tube runs with the analytic solution, as the paper does
for its Sod test (Sec. 3.2).  Written from the gas dynamics of the problem:
the star pressure p* solves f_L(p) + f_R(p) + (u_R - u_L) = 0, where f_K is the
shock (Rankine-Hugoniot) branch for p > p_K and the rarefaction (isentropic
Riemann-invariant) branch otherwise; the star velocity, star densities and
wave speeds follow, and the self-similar profile is sampled at x/t.
"""
from __future__ import annotations

import math

import numpy as np


def _fk(p, rho, pk, ck, g):
    if p > pk:
        A = 2.0 / ((g + 1.0) * rho)
        B = (g - 1.0) / (g + 1.0) * pk
        f = (p - pk) * math.sqrt(A / (p + B))
        df = math.sqrt(A / (B + p)) * (1.0 - 0.5 * (p - pk) / (B + p))
    else:
        f = 2.0 * ck / (g - 1.0) * ((p / pk) ** ((g - 1.0) / (2.0 * g)) - 1.0)
        df = 1.0 / (rho * ck) * (p / pk) ** (-(g + 1.0) / (2.0 * g))
    return f, df


def star_state(rhoL, uL, pL, rhoR, uR, pR, gamma):
    """Return dict(p, u, rhoL, rhoR, SL_head, SL_tail, SR) of the star region."""
    g = gamma
    cL = math.sqrt(g * pL / rhoL)
    cR = math.sqrt(g * pR / rhoR)
    if 2.0 * (cL + cR) / (g - 1.0) <= uR - uL:
        raise ValueError("vacuum is generated")
    p = max(1e-12, 0.5 * (pL + pR))
    for _ in range(200):
        fL, dL = _fk(p, rhoL, pL, cL, g)
        fR, dR = _fk(p, rhoR, pR, cR, g)
        pn = p - (fL + fR + uR - uL) / (dL + dR)
        pn = max(pn, 1e-14)
        if abs(pn - p) < 1e-15 * (pn + p):
            p = pn
            break
        p = pn
    fL, _ = _fk(p, rhoL, pL, cL, g)
    fR, _ = _fk(p, rhoR, pR, cR, g)
    u = 0.5 * (uL + uR) + 0.5 * (fR - fL)
    gr = (g - 1.0) / (g + 1.0)
    out = {"p": p, "u": u}
    if p > pL:
        out["rhoL"] = rhoL * (p / pL + gr) / (gr * p / pL + 1.0)
        SL = uL - cL * math.sqrt((g + 1.0) / (2 * g) * p / pL + (g - 1.0) / (2 * g))
        out["SL_head"] = out["SL_tail"] = SL
    else:
        out["rhoL"] = rhoL * (p / pL) ** (1.0 / g)
        cs = cL * (p / pL) ** ((g - 1.0) / (2 * g))
        out["SL_head"] = uL - cL
        out["SL_tail"] = u - cs
    if p > pR:
        out["rhoR"] = rhoR * (p / pR + gr) / (gr * p / pR + 1.0)
        SR = uR + cR * math.sqrt((g + 1.0) / (2 * g) * p / pR + (g - 1.0) / (2 * g))
        out["SR_head"] = out["SR_tail"] = SR
    else:
        out["rhoR"] = rhoR * (p / pR) ** (1.0 / g)
        cs = cR * (p / pR) ** ((g - 1.0) / (2 * g))
        out["SR_head"] = uR + cR
        out["SR_tail"] = u + cs
    out["SR"] = out["SR_head"]
    return out


def sample(xi, rhoL, uL, pL, rhoR, uR, pR, gamma):
    """Density, velocity and pressure at the similarity coordinates xi = x/t."""
    g = gamma
    s = star_state(rhoL, uL, pL, rhoR, uR, pR, gamma)
    cL = math.sqrt(g * pL / rhoL)
    cR = math.sqrt(g * pR / rhoR)
    xi = np.atleast_1d(np.asarray(xi, dtype=np.float64))
    rho = np.empty_like(xi)
    u = np.empty_like(xi)
    p = np.empty_like(xi)
    for k, x in enumerate(xi):
        if x <= s["u"]:
            if x <= s["SL_head"]:
                rho[k], u[k], p[k] = rhoL, uL, pL
            elif x >= s["SL_tail"]:
                rho[k], u[k], p[k] = s["rhoL"], s["u"], s["p"]
            else:  # inside the left rarefaction fan
                c = 2.0 / (g + 1.0) * (cL + 0.5 * (g - 1.0) * (uL - x))
                u[k] = 2.0 / (g + 1.0) * (cL + 0.5 * (g - 1.0) * uL + x)
                rho[k] = rhoL * (c / cL) ** (2.0 / (g - 1.0))
                p[k] = pL * (c / cL) ** (2.0 * g / (g - 1.0))
        else:
            if x >= s["SR_head"]:
                rho[k], u[k], p[k] = rhoR, uR, pR
            elif x <= s["SR_tail"]:
                rho[k], u[k], p[k] = s["rhoR"], s["u"], s["p"]
            else:  # inside a right rarefaction fan
                c = 2.0 / (g + 1.0) * (cR - 0.5 * (g - 1.0) * (uR - x))
                u[k] = 2.0 / (g + 1.0) * (-cR + 0.5 * (g - 1.0) * uR + x)
                rho[k] = rhoR * (c / cR) ** (2.0 / (g - 1.0))
                p[k] = pR * (c / cR) ** (2.0 * g / (g - 1.0))
    return rho, u, p
