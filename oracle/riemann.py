"""Exact solution of the 1D Riemann problem of an ideal gas (gamma-law), the
reference for the Sod shock tube and the blast wave tests (Sect. 4.1-4.2).

TEST INFRASTRUCTURE ONLY (used by the test suite, never by the product).

Two uniform states (rho, u, p) meet at x0 at t = 0.  The solution is
self-similar in xi = (x - x0) / t: a left wave (shock or rarefaction), a
contact moving at u*, a right wave, with the star-region pressure p* the
root of

    f_L(p) + f_R(p) + (u_R - u_L) = 0,

where, for side K with sound speed c_K = sqrt(gamma p_K / rho_K),

    shock (p > p_K):        f_K = (p - p_K) sqrt(A_K / (p + B_K)),
                            A_K = 2 / ((gamma + 1) rho_K), B_K = p_K (gamma - 1) / (gamma + 1)
    rarefaction (p <= p_K): f_K = 2 c_K / (gamma - 1) ((p / p_K)^((gamma - 1) / (2 gamma)) - 1)

(the velocity jump across each wave: the Rankine-Hugoniot conditions for a
shock, the constancy of the Riemann invariant u +- 2 c / (gamma - 1) and of
the entropy p / rho^gamma through a rarefaction), and u* = (u_L + u_R) / 2 +
(f_R(p*) - f_L(p*)) / 2.  The root is bracketed and found with a library
root finder (scipy's brentq).
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np
from scipy.optimize import brentq


@dataclass
class State:
    rho: float
    u: float
    p: float


@dataclass
class Star:
    p: float
    u: float
    rho_l: float
    rho_r: float


def _sound(s: State, gamma: float) -> float:
    return float(np.sqrt(gamma * s.p / s.rho))


def _f(p: float, s: State, gamma: float) -> float:
    if p > s.p:
        A = 2.0 / ((gamma + 1.0) * s.rho)
        B = s.p * (gamma - 1.0) / (gamma + 1.0)
        return (p - s.p) * np.sqrt(A / (p + B))
    c = _sound(s, gamma)
    return 2.0 * c / (gamma - 1.0) * ((p / s.p) ** ((gamma - 1.0) / (2.0 * gamma)) - 1.0)


def _rho_star(p: float, s: State, gamma: float) -> float:
    r = p / s.p
    if p > s.p:                      # behind a shock (Rankine-Hugoniot)
        g = (gamma - 1.0) / (gamma + 1.0)
        return s.rho * (r + g) / (g * r + 1.0)
    return s.rho * r ** (1.0 / gamma)  # isentropic


def star_state(left: State, right: State, gamma: float) -> Star:
    """p*, u* and the densities on both sides of the contact."""
    g = lambda p: _f(p, left, gamma) + _f(p, right, gamma) + (right.u - left.u)
    lo, hi = 1e-14 * min(left.p, right.p), max(left.p, right.p)
    while g(hi) < 0.0:
        hi *= 2.0
    if g(lo) > 0.0:
        raise ValueError("the states do not meet (vacuum forms)")
    p = brentq(g, lo, hi, xtol=1e-16 * hi, rtol=1e-15, maxiter=500)
    u = 0.5 * (left.u + right.u) + 0.5 * (_f(p, right, gamma) - _f(p, left, gamma))
    return Star(p, u, _rho_star(p, left, gamma), _rho_star(p, right, gamma))


def _side(xi, s: State, star: Star, gamma: float, m: float):
    """(rho, u, p) at speeds xi on one side of the contact: m = +1 for the
    left side; m = -1 for the right side, which is the left side mirrored
    (x -> -x, u -> -u), so one set of left-wave formulas serves both."""
    c = _sound(s, gamma)
    us, u0 = m * star.u, m * s.u
    x = m * xi
    rho_s = star.rho_l if m > 0 else star.rho_r
    if star.p > s.p:                      # shock, moving to -x in the (mirrored) frame
        S = u0 - c * np.sqrt((gamma + 1.0) / (2.0 * gamma) * star.p / s.p + (gamma - 1.0) / (2.0 * gamma))
        pre = x < S
        rho = np.where(pre, s.rho, rho_s)
        u = np.where(pre, u0, us)
        p = np.where(pre, s.p, star.p)
    else:                                 # rarefaction fan between head and tail
        cs = c * (star.p / s.p) ** ((gamma - 1.0) / (2.0 * gamma))
        head, tail = u0 - c, us - cs
        uf = 2.0 / (gamma + 1.0) * (c + 0.5 * (gamma - 1.0) * u0 + x)
        cf = np.maximum(2.0 / (gamma + 1.0) * (c + 0.5 * (gamma - 1.0) * (u0 - x)), 0.0)
        fan = (x >= head) & (x <= tail)
        rho = np.where(x < head, s.rho, np.where(fan, s.rho * (cf / c) ** (2.0 / (gamma - 1.0)), rho_s))
        u = np.where(x < head, u0, np.where(fan, uf, us))
        p = np.where(x < head, s.p, np.where(fan, s.p * (cf / c) ** (2.0 * gamma / (gamma - 1.0)), star.p))
    return rho, m * u, p


def sample(x, t: float, x0: float, left: State, right: State, gamma: float):
    """(rho, u, p) of the exact solution at positions x and time t > 0."""
    x = np.asarray(x, np.float64)
    xi = (x - x0) / t
    star = star_state(left, right, gamma)
    rl, ul, pl = _side(xi, left, star, gamma, 1.0)
    rr, ur, pr = _side(xi, right, star, gamma, -1.0)
    lft = xi < star.u
    return np.where(lft, rl, rr), np.where(lft, ul, ur), np.where(lft, pl, pr)


def wave_speeds(left: State, right: State, gamma: float):
    """(left head, left tail, contact, right tail, right head) speeds; for a
    shock head = tail = the shock speed."""
    star = star_state(left, right, gamma)
    out = []
    for s, m in ((left, 1.0), (right, -1.0)):
        c = _sound(s, gamma)
        u0, us = m * s.u, m * star.u
        if star.p > s.p:
            S = u0 - c * np.sqrt((gamma + 1.0) / (2.0 * gamma) * star.p / s.p + (gamma - 1.0) / (2.0 * gamma))
            out.append((m * S, m * S))
        else:
            cs = c * (star.p / s.p) ** ((gamma - 1.0) / (2.0 * gamma))
            out.append((m * (u0 - c), m * (us - cs)))
    (lh, lt), (rh, rt) = out
    return lh, lt, star.u, rt, rh
