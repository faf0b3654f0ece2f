"""Exact solution of the Riemann problem for the 1D Euler equations (ideal gas).

Written from the mathematics of the two-shock/two-rarefaction wave curves
(Toro, "Riemann Solvers and Numerical Methods for Fluid Dynamics", Ch. 4):
the star pressure solves f_L(p) + f_R(p) + (u_R - u_L) = 0, where f_K is the
shock (Rankine-Hugoniot) branch for p > p_K and the isentropic rarefaction
branch otherwise; the solution is then sampled on rays x/t.

Used only as an independent pin of the oracle (its own numerics, no code in
common with the oracle or the CUDA path).
"""
from __future__ import annotations

import math

import numpy as np


def _fK(p, rho, pK, g):
    c = math.sqrt(g * pK / rho)
    if p > pK:
        A = 2.0 / ((g + 1.0) * rho)
        B = (g - 1.0) / (g + 1.0) * pK
        f = (p - pK) * math.sqrt(A / (p + B))
        df = math.sqrt(A / (B + p)) * (1.0 - (p - pK) / (2.0 * (B + p)))
    else:
        f = 2.0 * c / (g - 1.0) * ((p / pK) ** ((g - 1.0) / (2.0 * g)) - 1.0)
        df = 1.0 / (rho * c) * (p / pK) ** (-(g + 1.0) / (2.0 * g))
    return f, df


def star_state(rhoL, uL, pL, rhoR, uR, pR, g=1.4, tol=1e-15):
    """Return (p*, u*, rho*_L, rho*_R)."""
    cL, cR = math.sqrt(g * pL / rhoL), math.sqrt(g * pR / rhoR)
    # two-rarefaction guess
    z = (g - 1.0) / (2.0 * g)
    p = ((cL + cR - 0.5 * (g - 1.0) * (uR - uL)) / (cL / pL ** z + cR / pR ** z)) ** (1.0 / z)
    p = max(p, 1e-12)
    for _ in range(200):
        fL, dL = _fK(p, rhoL, pL, g)
        fR, dR = _fK(p, rhoR, pR, g)
        pn = p - (fL + fR + uR - uL) / (dL + dR)
        pn = max(pn, 1e-14)
        if abs(pn - p) / (0.5 * (pn + p)) < tol:
            p = pn
            break
        p = pn
    fL, _ = _fK(p, rhoL, pL, g)
    fR, _ = _fK(p, rhoR, pR, g)
    u = 0.5 * (uL + uR) + 0.5 * (fR - fL)
    gm = (g - 1.0) / (g + 1.0)

    def rho_star(rhoK, pK):
        if p > pK:
            return rhoK * (p / pK + gm) / (gm * p / pK + 1.0)
        return rhoK * (p / pK) ** (1.0 / g)

    return p, u, rho_star(rhoL, pL), rho_star(rhoR, pR)


def sample(xi, rhoL, uL, pL, rhoR, uR, pR, g=1.4):
    """Exact (rho, u, p) at similarity coordinates xi = (x - x0) / t (array)."""
    ps, us, rsL, rsR = star_state(rhoL, uL, pL, rhoR, uR, pR, g)
    xi = np.asarray(xi, dtype=np.float64)
    rho = np.empty_like(xi)
    u = np.empty_like(xi)
    p = np.empty_like(xi)
    cL, cR = math.sqrt(g * pL / rhoL), math.sqrt(g * pR / rhoR)
    for idx, s in np.ndenumerate(xi):
        if s <= us:  # left of contact
            if ps > pL:
                SL = uL - cL * math.sqrt((g + 1) / (2 * g) * ps / pL + (g - 1) / (2 * g))
                r, v, q = (rhoL, uL, pL) if s <= SL else (rsL, us, ps)
            else:
                SHL = uL - cL
                cs = cL * (ps / pL) ** ((g - 1) / (2 * g))
                STL = us - cs
                if s <= SHL:
                    r, v, q = rhoL, uL, pL
                elif s > STL:
                    r, v, q = rsL, us, ps
                else:
                    f = 2 / (g + 1) + (g - 1) / ((g + 1) * cL) * (uL - s)
                    r = rhoL * f ** (2 / (g - 1))
                    v = 2 / (g + 1) * (cL + (g - 1) / 2 * uL + s)
                    q = pL * f ** (2 * g / (g - 1))
        else:  # right of contact
            if ps > pR:
                SR = uR + cR * math.sqrt((g + 1) / (2 * g) * ps / pR + (g - 1) / (2 * g))
                r, v, q = (rhoR, uR, pR) if s >= SR else (rsR, us, ps)
            else:
                SHR = uR + cR
                cs = cR * (ps / pR) ** ((g - 1) / (2 * g))
                STR = us + cs
                if s >= SHR:
                    r, v, q = rhoR, uR, pR
                elif s <= STR:
                    r, v, q = rsR, us, ps
                else:
                    f = 2 / (g + 1) - (g - 1) / ((g + 1) * cR) * (uR - s)
                    r = rhoR * f ** (2 / (g - 1))
                    v = 2 / (g + 1) * (-cR + (g - 1) / 2 * uR + s)
                    q = pR * f ** (2 * g / (g - 1))
        rho[idx], u[idx], p[idx] = r, v, q
    return rho, u, p


def cell_average(x_lo, x_hi, t, x0, states, g=1.4, sub=64):
    """Exact cell averages of (rho, u, p) over cells [x_lo, x_hi) (midpoint sub-sampling)."""
    x_lo = np.asarray(x_lo, float)
    x_hi = np.asarray(x_hi, float)
    fr = (np.arange(sub) + 0.5) / sub
    xs = x_lo[:, None] + (x_hi - x_lo)[:, None] * fr[None, :]
    r, u, p = sample((xs - x0) / t, *states, g=g)
    return r.mean(axis=1), u.mean(axis=1), p.mean(axis=1)
