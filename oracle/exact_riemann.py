"""Exact Riemann solver for a polytropic gas, used with gamma = 3 as the analytic
solution of the one-dimensional collisionless moment equations.

Test infrastructure only.  Sec. 4 ("Tests") shows that for a 1D flow along x the moment
equations reduce to classic hydrodynamics with pressure P = rho sigma_xx^2 and gamma = 3,
and Sec. 4.1 uses Sod's (1978) standard solution procedure for the shock tube.  This
module writes that procedure from the mathematics (two-shock/two-rarefaction pressure
function, root for p*, self-similar sampling); it follows the presentation in Toro,
"Riemann Solvers and Numerical Methods for Fluid Dynamics", ch. 4.

The transverse moments are passive in this flow: with v = w = 0 and P_xy = P_xz = 0, the
equations for E_yy, E_zz, E_yz have the same conservative form as the continuity
equation, so P_yy/rho, P_zz/rho and P_yz/rho are constant along particle paths and
continuous across shocks: they take the value of the material's side of the contact.
"""
from __future__ import annotations

import math

import numpy as np
from scipy.optimize import brentq


def _fk(p, rho, pk, ck, g):
    """Velocity change across the left/right wave as a function of the star pressure."""
    if p > pk:  # shock: Rankine-Hugoniot
        A = 2.0 / ((g + 1.0) * rho)
        B = (g - 1.0) / (g + 1.0) * pk
        return (p - pk) * math.sqrt(A / (p + B))
    # rarefaction: isentropic
    return 2.0 * ck / (g - 1.0) * ((p / pk) ** ((g - 1.0) / (2.0 * g)) - 1.0)


def star_state(rhoL, uL, pL, rhoR, uR, pR, gamma=3.0):
    """Return (p*, u*, rho*_L, rho*_R)."""
    g = gamma
    cL, cR = math.sqrt(g * pL / rhoL), math.sqrt(g * pR / rhoR)
    f = lambda p: _fk(p, rhoL, pL, cL, g) + _fk(p, rhoR, pR, cR, g) + (uR - uL)
    pmax = max(pL, pR)
    hi = 10.0 * pmax
    while f(hi) < 0:
        hi *= 10.0
    ps = brentq(f, 1e-14 * min(pL, pR), hi, xtol=1e-15, rtol=1e-15, maxiter=500)
    us = 0.5 * (uL + uR) + 0.5 * (_fk(ps, rhoR, pR, cR, g) - _fk(ps, rhoL, pL, cL, g))

    def rho_star(rho, pk):
        if ps > pk:
            r = ps / pk
            q = (g - 1.0) / (g + 1.0)
            return rho * (r + q) / (q * r + 1.0)
        return rho * (ps / pk) ** (1.0 / g)

    return ps, us, rho_star(rhoL, pL), rho_star(rhoR, pR)


def wave_speeds(rhoL, uL, pL, rhoR, uR, pR, gamma=3.0):
    """Dict with the characteristic speeds of the solution fan."""
    g = gamma
    ps, us, rsL, rsR = star_state(rhoL, uL, pL, rhoR, uR, pR, g)
    cL, cR = math.sqrt(g * pL / rhoL), math.sqrt(g * pR / rhoR)
    out = {"p_star": ps, "u_star": us, "rho_star_L": rsL, "rho_star_R": rsR, "contact": us}
    if ps > pL:
        out["left_shock"] = uL - cL * math.sqrt((g + 1) / (2 * g) * ps / pL + (g - 1) / (2 * g))
    else:
        out["left_head"] = uL - cL
        out["left_tail"] = us - cL * (ps / pL) ** ((g - 1) / (2 * g))
    if ps > pR:
        out["right_shock"] = uR + cR * math.sqrt((g + 1) / (2 * g) * ps / pR + (g - 1) / (2 * g))
    else:
        out["right_head"] = uR + cR
        out["right_tail"] = us + cR * (ps / pR) ** ((g - 1) / (2 * g))
    return out


def sample(xi, rhoL, uL, pL, rhoR, uR, pR, gamma=3.0):
    """(rho, u, p, side) at similarity coordinates xi = (x - x0)/t; side = 0 for material
    from the left state, 1 for the right."""
    g = gamma
    xi = np.asarray(xi, dtype=np.float64)
    ps, us, rsL, rsR = star_state(rhoL, uL, pL, rhoR, uR, pR, g)
    cL, cR = math.sqrt(g * pL / rhoL), math.sqrt(g * pR / rhoR)
    rho = np.empty_like(xi)
    u = np.empty_like(xi)
    p = np.empty_like(xi)
    side = (xi > us).astype(np.int64)
    for i, s in enumerate(xi.ravel()):
        if s <= us:  # left of contact
            if ps > pL:
                SL = uL - cL * math.sqrt((g + 1) / (2 * g) * ps / pL + (g - 1) / (2 * g))
                st = (rhoL, uL, pL) if s <= SL else (rsL, us, ps)
            else:
                head = uL - cL
                tail = us - cL * (ps / pL) ** ((g - 1) / (2 * g))
                if s <= head:
                    st = (rhoL, uL, pL)
                elif s >= tail:
                    st = (rsL, us, ps)
                else:
                    c = 2.0 / (g + 1) * (cL + (g - 1) / 2 * (uL - s))
                    st = (rhoL * (c / cL) ** (2 / (g - 1)), 2 / (g + 1) * (cL + (g - 1) / 2 * uL + s),
                          pL * (c / cL) ** (2 * g / (g - 1)))
        else:  # right of contact
            if ps > pR:
                SR = uR + cR * math.sqrt((g + 1) / (2 * g) * ps / pR + (g - 1) / (2 * g))
                st = (rhoR, uR, pR) if s >= SR else (rsR, us, ps)
            else:
                head = uR + cR
                tail = us + cR * (ps / pR) ** ((g - 1) / (2 * g))
                if s >= head:
                    st = (rhoR, uR, pR)
                elif s <= tail:
                    st = (rsR, us, ps)
                else:
                    c = 2.0 / (g + 1) * (cR - (g - 1) / 2 * (uR - s))
                    st = (rhoR * (c / cR) ** (2 / (g - 1)), 2 / (g + 1) * (-cR + (g - 1) / 2 * uR + s),
                          pR * (c / cR) ** (2 * g / (g - 1)))
        rho.flat[i], u.flat[i], p.flat[i] = st
    return rho, u, p, side


def bme_sod_solution(x, t, x0, left, right):
    """Analytic primitive state (10 x len(x)) of a 1D moment-equation Riemann problem with
    v = w = 0 and diagonal P.  left/right: dicts with rho, u, Pxx, Pyy, Pzz."""
    x = np.asarray(x, dtype=np.float64)
    rho, u, p, side = sample((x - x0) / t, left["rho"], left["u"], left["Pxx"],
                             right["rho"], right["u"], right["Pxx"], 3.0)
    W = np.zeros((10, x.size))
    W[0], W[1], W[4] = rho, u, p
    for comp, key in ((7, "Pyy"), (9, "Pzz")):
        sL = left[key] / left["rho"]
        sR = right[key] / right["rho"]
        W[comp] = rho * np.where(side == 0, sL, sR)
    return W
