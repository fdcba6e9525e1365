"""Exact Riemann solver for the ideal-gas Euler equations (test helper).

Textbook construction (Toro, Riemann Solvers and Numerical Methods for Fluid
Dynamics, ch. 4): the star pressure solves f_L(p) + f_R(p) + (u_R - u_L) = 0,
with f_K the shock (Rankine-Hugoniot) branch for p > p_K and the isentropic
rarefaction branch otherwise; the solution is then sampled in x/t.
Independent of the oracle: it is a pin for the oracle's Sod runs.
"""
import math

import numpy as np
from scipy.optimize import brentq


def _fK(p, rho, pK, c, g):
    if p > pK:
        A = 2.0 / ((g + 1.0) * rho)
        B = (g - 1.0) / (g + 1.0) * pK
        return (p - pK) * math.sqrt(A / (p + B))
    return 2.0 * c / (g - 1.0) * ((p / pK) ** ((g - 1.0) / (2.0 * g)) - 1.0)


def star_state(rhoL, uL, pL, rhoR, uR, pR, g):
    cL = math.sqrt(g * pL / rhoL)
    cR = math.sqrt(g * pR / rhoR)
    F = lambda p: _fK(p, rhoL, pL, cL, g) + _fK(p, rhoR, pR, cR, g) + (uR - uL)
    p = brentq(F, 1e-12, 10.0 * max(pL, pR), xtol=1e-15, rtol=1e-15, maxiter=500)
    u = 0.5 * (uL + uR) + 0.5 * (_fK(p, rhoR, pR, cR, g) - _fK(p, rhoL, pL, cL, g))

    def rho_star(rho, pK):
        if p > pK:
            r = (g - 1.0) / (g + 1.0)
            return rho * (p / pK + r) / (r * p / pK + 1.0)
        return rho * (p / pK) ** (1.0 / g)
    return p, u, rho_star(rhoL, pL), rho_star(rhoR, pR)


def sample(xi, rhoL, uL, pL, rhoR, uR, pR, g):
    """Density, velocity, pressure at similarity coordinates xi = (x - x0)/t (array)."""
    p, u, rLs, rRs = star_state(rhoL, uL, pL, rhoR, uR, pR, g)
    cL = math.sqrt(g * pL / rhoL)
    cR = math.sqrt(g * pR / rhoR)
    xi = np.asarray(xi, float)
    rho = np.empty_like(xi)
    vel = np.empty_like(xi)
    pre = np.empty_like(xi)
    for n, s in enumerate(xi.flat):
        if s <= u:  # left of contact
            if p > pL:
                S = uL - cL * math.sqrt((g + 1) / (2 * g) * p / pL + (g - 1) / (2 * g))
                st = (rhoL, uL, pL) if s < S else (rLs, u, p)
            else:
                cs = cL * (p / pL) ** ((g - 1) / (2 * g))
                head, tail = uL - cL, u - cs
                if s < head:
                    st = (rhoL, uL, pL)
                elif s > tail:
                    st = (rLs, u, p)
                else:
                    c = 2 / (g + 1) * (cL + (g - 1) / 2 * (uL - s))
                    v = 2 / (g + 1) * (cL + (g - 1) / 2 * uL + s)
                    st = (rhoL * (c / cL) ** (2 / (g - 1)), v, pL * (c / cL) ** (2 * g / (g - 1)))
        else:
            if p > pR:
                S = uR + cR * math.sqrt((g + 1) / (2 * g) * p / pR + (g - 1) / (2 * g))
                st = (rhoR, uR, pR) if s > S else (rRs, u, p)
            else:
                cs = cR * (p / pR) ** ((g - 1) / (2 * g))
                head, tail = uR + cR, u + cs
                if s > head:
                    st = (rhoR, uR, pR)
                elif s < tail:
                    st = (rRs, u, p)
                else:
                    c = 2 / (g + 1) * (cR - (g - 1) / 2 * (uR - s))
                    v = 2 / (g + 1) * (-cR + (g - 1) / 2 * uR + s)
                    st = (rhoR * (c / cR) ** (2 / (g - 1)), v, pR * (c / cR) ** (2 * g / (g - 1)))
        rho.flat[n], vel.flat[n], pre.flat[n] = st
    return rho, vel, pre


def shock_speed(rhoR, uR, pR, p_star, g):
    cR = math.sqrt(g * pR / rhoR)
    return uR + cR * math.sqrt((g + 1) / (2 * g) * p_star / pR + (g - 1) / (2 * g))
