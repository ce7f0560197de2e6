"""Exact solution of the Riemann problem of the 1-D Euler equations for an
ideal gas (Toro, Riemann Solvers and Numerical Methods for Fluid Dynamics,
Ch. 4): the star pressure is the root of f_L(p) + f_R(p) + u_R - u_L = 0,
with f_K the shock (Rankine-Hugoniot) or rarefaction (isentropic) relation
of side K, and the solution is self-similar in x/t.  Test infrastructure:
an independent reference for the hydrodynamic oracle."""
import numpy as np
from scipy.optimize import brentq


def _f(p, rho, pk, a, g):
    if p > pk:  # shock
        A = 2.0 / ((g + 1.0) * rho)
        B = (g - 1.0) / (g + 1.0) * pk
        return (p - pk) * np.sqrt(A / (p + B))
    return 2.0 * a / (g - 1.0) * ((p / pk) ** ((g - 1.0) / (2.0 * g)) - 1.0)


def star(WL, WR, g):
    """(p*, u*) of the left and right primitive states (rho, u, p)."""
    rL, uL, pL = WL
    rR, uR, pR = WR
    aL, aR = np.sqrt(g * pL / rL), np.sqrt(g * pR / rR)
    fun = lambda p: _f(p, rL, pL, aL, g) + _f(p, rR, pR, aR, g) + uR - uL
    lo, hi = 1e-14 * min(pL, pR), 10.0 * max(pL, pR)
    while fun(hi) < 0:
        hi *= 10.0
    ps = brentq(fun, lo, hi, xtol=1e-15, rtol=1e-15, maxiter=500)
    us = 0.5 * (uL + uR) + 0.5 * (_f(ps, rR, pR, aR, g) - _f(ps, rL, pL, aL, g))
    return ps, us


def sample(WL, WR, g, xi):
    """(rho, u, p) at the similarity coordinates xi = (x - x0)/t."""
    rL, uL, pL = WL
    rR, uR, pR = WR
    aL, aR = np.sqrt(g * pL / rL), np.sqrt(g * pR / rR)
    ps, us = star(WL, WR, g)
    gm = (g - 1.0) / (g + 1.0)
    out = np.zeros((3, len(xi)))
    for i, s in enumerate(np.asarray(xi, dtype=float)):
        if s <= us:
            if ps > pL:
                SL = uL - aL * np.sqrt((g + 1) / (2 * g) * ps / pL + (g - 1) / (2 * g))
                W = (rL, uL, pL) if s <= SL else \
                    (rL * (ps / pL + gm) / (gm * ps / pL + 1.0), us, ps)
            else:
                SH = uL - aL
                ast = aL * (ps / pL) ** ((g - 1) / (2 * g))
                ST = us - ast
                if s <= SH:
                    W = (rL, uL, pL)
                elif s >= ST:
                    W = (rL * (ps / pL) ** (1.0 / g), us, ps)
                else:
                    u = 2.0 / (g + 1) * (aL + 0.5 * (g - 1) * uL + s)
                    a = 2.0 / (g + 1) * (aL + 0.5 * (g - 1) * (uL - s))
                    W = (rL * (a / aL) ** (2 / (g - 1)), u, pL * (a / aL) ** (2 * g / (g - 1)))
        else:
            if ps > pR:
                SR = uR + aR * np.sqrt((g + 1) / (2 * g) * ps / pR + (g - 1) / (2 * g))
                W = (rR, uR, pR) if s >= SR else \
                    (rR * (ps / pR + gm) / (gm * ps / pR + 1.0), us, ps)
            else:
                SH = uR + aR
                ast = aR * (ps / pR) ** ((g - 1) / (2 * g))
                ST = us + ast
                if s >= SH:
                    W = (rR, uR, pR)
                elif s <= ST:
                    W = (rR * (ps / pR) ** (1.0 / g), us, ps)
                else:
                    u = 2.0 / (g + 1) * (-aR + 0.5 * (g - 1) * uR + s)
                    a = 2.0 / (g + 1) * (aR - 0.5 * (g - 1) * (uR - s))
                    W = (rR * (a / aR) ** (2 / (g - 1)), u, pR * (a / aR) ** (2 * g / (g - 1)))
        out[:, i] = W
    return out
