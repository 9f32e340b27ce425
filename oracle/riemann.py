"""Exact Riemann solver for the 1D Euler equations of an ideal gas.

TEST INFRASTRUCTURE ONLY (pin P9: convergence of the compact GKS to the exact
solution of two-state problems such as the paper's shock tubes, Sec. 6.5).

Written from the wave relations: across a shock the Rankine-Hugoniot
conditions give the velocity jump f_K(p) = (p - p_K) sqrt(A_K / (p + B_K)),
A_K = 2 / ((g+1) rho_K), B_K = (g-1)/(g+1) p_K; across a rarefaction the
isentropic relation gives f_K(p) = 2 c_K / (g-1) ((p/p_K)^((g-1)/(2g)) - 1).
The star pressure solves f_L(p) + f_R(p) + u_R - u_L = 0 (monotone in p, so
a bracketing root finder is used), u* = (u_L + u_R + f_R - f_L) / 2.
"""
from __future__ import annotations

import math

import numpy as np
from scipy.optimize import brentq


def _f(p, rho, pk, gamma):
    c = math.sqrt(gamma * pk / rho)
    if p > pk:
        A = 2.0 / ((gamma + 1.0) * rho)
        B = (gamma - 1.0) / (gamma + 1.0) * pk
        return (p - pk) * math.sqrt(A / (p + B))
    return 2.0 * c / (gamma - 1.0) * ((p / pk) ** ((gamma - 1.0) / (2.0 * gamma)) - 1.0)


def star_state(L, R, gamma=1.4):
    """(p*, u*) for primitive states L = (rho, u, p), R = (rho, u, p)."""
    rl, ul, pl = L
    rr, ur, pr = R
    cl = math.sqrt(gamma * pl / rl)
    cr = math.sqrt(gamma * pr / rr)
    if ur - ul >= 2.0 * (cl + cr) / (gamma - 1.0):
        raise ValueError("vacuum is generated")
    g = lambda p: _f(p, rl, pl, gamma) + _f(p, rr, pr, gamma) + ur - ul
    lo, hi = 1e-14, max(pl, pr)
    while g(hi) < 0.0:
        hi *= 2.0
    ps = brentq(g, lo, hi, xtol=1e-15, rtol=1e-15, maxiter=500)
    us = 0.5 * (ul + ur) + 0.5 * (_f(ps, rr, pr, gamma) - _f(ps, rl, pl, gamma))
    return ps, us


def sample(L, R, xi, gamma=1.4):
    """Primitive state (rho, u, p) of the self-similar solution at xi = x/t (arrays)."""
    rl, ul, pl = L
    rr, ur, pr = R
    ps, us = star_state(L, R, gamma)
    gm = (gamma - 1.0) / (gamma + 1.0)
    xi = np.asarray(xi, dtype=np.float64)
    rho = np.empty_like(xi)
    u = np.empty_like(xi)
    p = np.empty_like(xi)
    for idx, s in np.ndenumerate(xi):
        if s <= us:  # left of the contact
            c = math.sqrt(gamma * pl / rl)
            if ps > pl:  # left shock
                S = ul - c * math.sqrt((gamma + 1) / (2 * gamma) * ps / pl + (gamma - 1) / (2 * gamma))
                if s <= S:
                    st = (rl, ul, pl)
                else:
                    st = (rl * (ps / pl + gm) / (gm * ps / pl + 1), us, ps)
            else:  # left rarefaction
                cs = c * (ps / pl) ** ((gamma - 1) / (2 * gamma))
                if s <= ul - c:
                    st = (rl, ul, pl)
                elif s >= us - cs:
                    st = (rl * (ps / pl) ** (1 / gamma), us, ps)
                else:
                    uu = 2 / (gamma + 1) * (c + (gamma - 1) / 2 * ul + s)
                    cc = 2 / (gamma + 1) * (c + (gamma - 1) / 2 * (ul - s))
                    st = (rl * (cc / c) ** (2 / (gamma - 1)), uu, pl * (cc / c) ** (2 * gamma / (gamma - 1)))
        else:  # right of the contact
            c = math.sqrt(gamma * pr / rr)
            if ps > pr:  # right shock
                S = ur + c * math.sqrt((gamma + 1) / (2 * gamma) * ps / pr + (gamma - 1) / (2 * gamma))
                if s >= S:
                    st = (rr, ur, pr)
                else:
                    st = (rr * (ps / pr + gm) / (gm * ps / pr + 1), us, ps)
            else:  # right rarefaction
                cs = c * (ps / pr) ** ((gamma - 1) / (2 * gamma))
                if s >= ur + c:
                    st = (rr, ur, pr)
                elif s <= us + cs:
                    st = (rr * (ps / pr) ** (1 / gamma), us, ps)
                else:
                    uu = 2 / (gamma + 1) * (-c + (gamma - 1) / 2 * ur + s)
                    cc = 2 / (gamma + 1) * (c - (gamma - 1) / 2 * (ur - s))
                    st = (rr * (cc / c) ** (2 / (gamma - 1)), uu, pr * (cc / c) ** (2 * gamma / (gamma - 1)))
        rho[idx], u[idx], p[idx] = st
    return rho, u, p


def cell_averages(L, R, n, t, x0=0.5, gamma=1.4, sub=64):
    """Cell averages of the conservative variables on [0, 1] (n cells) at time t,
    by midpoint sampling with `sub` points per cell."""
    h = 1.0 / n
    xs = (np.arange(n * sub) + 0.5) * (h / sub)
    rho, u, p = sample(L, R, (xs - x0) / t, gamma)
    W = np.stack([rho, rho * u, p / (gamma - 1) + 0.5 * rho * u * u])
    return W.reshape(3, n, sub).mean(axis=2)
