"""Exact solution of the Riemann problem of the 1D Euler equations for an ideal gas.

TEST INFRASTRUCTURE ONLY (pins the oracle's shock capturing against the shock-tube tests of
Sec. 5.1 / Table Test1D).

Method (Godunov's exact solver as described by Toro, "Riemann Solvers and Numerical Methods for
Fluid Dynamics", Ch. 4): the star-region pressure p* is the root of
    f_L(p) + f_R(p) + (u_R - u_L) = 0,
where for side K the wave is a shock when p > p_K,
    f_K(p) = (p - p_K) sqrt(A_K / (p + B_K)),  A_K = 2 / ((g+1) rho_K),  B_K = (g-1)/(g+1) p_K,
and a rarefaction otherwise,
    f_K(p) = 2 c_K / (g-1) ((p / p_K)^((g-1)/(2g)) - 1).
f is monotone in p, so the root is bracketed and found with Brent's method. The star velocity is
u* = (u_L + u_R)/2 + (f_R(p*) - f_L(p*))/2, and the self-similar solution is sampled at x/t.
"""
from __future__ import annotations

import math

import numpy as np
from scipy.optimize import brentq


def _fk(p, rho, pk, gamma):
    ck = math.sqrt(gamma * pk / rho)
    if p > pk:
        A = 2.0 / ((gamma + 1.0) * rho)
        B = (gamma - 1.0) / (gamma + 1.0) * pk
        return (p - pk) * math.sqrt(A / (p + B))
    return 2.0 * ck / (gamma - 1.0) * ((p / pk) ** ((gamma - 1.0) / (2.0 * gamma)) - 1.0)


def star_state(left, right, gamma=1.4):
    """(p*, u*) of the Riemann problem with primitive states left/right = (rho, u, p)."""
    rl, ul, pl = left
    rr, ur, pr = right
    cl, cr = math.sqrt(gamma * pl / rl), math.sqrt(gamma * pr / rr)
    if 2.0 / (gamma - 1.0) * (cl + cr) <= ur - ul:
        raise ValueError("initial data generate vacuum")

    def f(p):
        return _fk(p, rl, pl, gamma) + _fk(p, rr, pr, gamma) + (ur - ul)

    lo, hi = 1e-14 * min(pl, pr), 10.0 * max(pl, pr)
    while f(hi) < 0.0:
        hi *= 10.0
    ps = brentq(f, lo, hi, xtol=1e-15 * hi, rtol=1e-15, maxiter=500)
    us = 0.5 * (ul + ur) + 0.5 * (_fk(ps, rr, pr, gamma) - _fk(ps, rl, pl, gamma))
    return ps, us


def star_densities(left, right, ps, gamma=1.4):
    """Densities just left and right of the contact in the star region."""
    out = []
    for (rk, uk, pk) in (left, right):
        if ps > pk:  # shock: Rankine-Hugoniot density ratio
            g = (gamma - 1.0) / (gamma + 1.0)
            out.append(rk * (ps / pk + g) / (g * ps / pk + 1.0))
        else:  # rarefaction: isentropic
            out.append(rk * (ps / pk) ** (1.0 / gamma))
    return tuple(out)


def sample(left, right, x, t, x0, gamma=1.4):
    """Exact (rho, u, p) at positions x (array) and time t > 0, discontinuity initially at x0."""
    rl, ul, pl = left
    rr, ur, pr = right
    ps, us = star_state(left, right, gamma)
    rsl, rsr = star_densities(left, right, ps, gamma)
    cl, cr = math.sqrt(gamma * pl / rl), math.sqrt(gamma * pr / rr)
    g1 = (gamma - 1.0) / (2.0 * gamma)
    xi = (np.asarray(x, dtype=np.float64) - x0) / t
    rho = np.empty_like(xi)
    u = np.empty_like(xi)
    p = np.empty_like(xi)
    for k, s in enumerate(xi):
        if s <= us:  # left of the contact
            if ps > pl:
                SL = ul - cl * math.sqrt((gamma + 1.0) / (2.0 * gamma) * ps / pl + g1)
                rho[k], u[k], p[k] = (rl, ul, pl) if s <= SL else (rsl, us, ps)
            else:
                SHL = ul - cl
                STL = us - cl * (ps / pl) ** g1
                if s <= SHL:
                    rho[k], u[k], p[k] = rl, ul, pl
                elif s >= STL:
                    rho[k], u[k], p[k] = rsl, us, ps
                else:
                    base = 2.0 / (gamma + 1.0) + (gamma - 1.0) / ((gamma + 1.0) * cl) * (ul - s)
                    rho[k] = rl * base ** (2.0 / (gamma - 1.0))
                    u[k] = 2.0 / (gamma + 1.0) * (cl + (gamma - 1.0) / 2.0 * ul + s)
                    p[k] = pl * base ** (2.0 * gamma / (gamma - 1.0))
        else:  # right of the contact
            if ps > pr:
                SR = ur + cr * math.sqrt((gamma + 1.0) / (2.0 * gamma) * ps / pr + g1)
                rho[k], u[k], p[k] = (rr, ur, pr) if s >= SR else (rsr, us, ps)
            else:
                SHR = ur + cr
                STR = us + cr * (ps / pr) ** g1
                if s >= SHR:
                    rho[k], u[k], p[k] = rr, ur, pr
                elif s <= STR:
                    rho[k], u[k], p[k] = rsr, us, ps
                else:
                    base = 2.0 / (gamma + 1.0) - (gamma - 1.0) / ((gamma + 1.0) * cr) * (ur - s)
                    rho[k] = rr * base ** (2.0 / (gamma - 1.0))
                    u[k] = 2.0 / (gamma + 1.0) * (-cr + (gamma - 1.0) / 2.0 * ur + s)
                    p[k] = pr * base ** (2.0 * gamma / (gamma - 1.0))
    return rho, u, p


def wave_speeds(left, right, gamma=1.4):
    """Speeds of the left wave (shock speed, or head/tail of the fan), the contact and the right wave."""
    rl, ul, pl = left
    rr, ur, pr = right
    ps, us = star_state(left, right, gamma)
    cl, cr = math.sqrt(gamma * pl / rl), math.sqrt(gamma * pr / rr)
    g1 = (gamma - 1.0) / (2.0 * gamma)
    if ps > pl:
        lw = (ul - cl * math.sqrt((gamma + 1.0) / (2.0 * gamma) * ps / pl + g1),)
    else:
        lw = (ul - cl, us - cl * (ps / pl) ** g1)
    if ps > pr:
        rw = (ur + cr * math.sqrt((gamma + 1.0) / (2.0 * gamma) * ps / pr + g1),)
    else:
        rw = (us + cr * (ps / pr) ** g1, ur + cr)
    return lw, us, rw
