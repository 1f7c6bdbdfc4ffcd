"""Seeded synthetic inputs shaped like the paper's tests (Sect. 4).

This module only draws initial conditions; it contains none of the SPH
method's arithmetic (no density, force or integration).  Both the CUDA path's
tests and the oracle-based tests take their inputs from here, so the two sides
always see the same float32 arrays.  Every generator uses
``numpy.random.Generator(PCG64(seed))``.

Array conventions (the library's layout):
  pos  float32 [n, 4]  = (x, y, z, m)
  vel  float32 [n, 4]  = (vx, vy, vz, u)
  h    float32 [n]     initial smoothing-length guess from an estimated density
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

HFACT = 1.2


@dataclass
class Workload:
    name: str
    pos: np.ndarray
    vel: np.ndarray
    h: np.ndarray
    meta: dict = field(default_factory=dict)

    @property
    def n(self) -> int:
        return int(self.pos.shape[0])


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def _pack(x, m, v, u):
    n = x.shape[0]
    pos = np.empty((n, 4), np.float32)
    vel = np.empty((n, 4), np.float32)
    pos[:, :3] = x
    pos[:, 3] = m
    vel[:, :3] = v
    vel[:, 3] = u
    return pos, vel


def unit_sphere(n: int = 8192, seed: int = 1, sigma_v: float = 0.1, u0: float = 0.05,
                hfact: float = HFACT) -> Workload:
    """n equal-mass (m = 1/n) particles uniform in the unit sphere (rejection
    sampling), Gaussian velocities (sigma per component), uniform u.
    Initial h from the mean density 3/(4 pi)."""
    g = _rng(seed)
    pts = np.empty((0, 3))
    while pts.shape[0] < n:
        c = g.uniform(-1.0, 1.0, size=(2 * n + 16, 3))
        c = c[np.einsum("ij,ij->i", c, c) < 1.0]
        pts = np.concatenate([pts, c])
    x = pts[:n]
    v = g.normal(0.0, sigma_v, size=(n, 3))
    m = np.full(n, 1.0 / n)
    u = np.full(n, u0)
    pos, vel = _pack(x, m, v, u)
    rho_est = 3.0 / (4.0 * np.pi)
    h = np.full(n, hfact * (1.0 / n / rho_est) ** (1.0 / 3.0), np.float32)
    return Workload("unit_sphere", pos, vel, h, {"seed": seed, "rho_est": rho_est})


def _bspline_shape(q):
    """Cubic B-spline profile used to spread the blast energy (initial condition)."""
    q = np.asarray(q, np.float64)
    return np.where(q < 1.0, 1.0 - 1.5 * q * q + 0.75 * q ** 3,
                    np.where(q < 2.0, 0.25 * (2.0 - q) ** 3, 0.0))


def sedov_lattice(side: int = 128, seed: int = 2, jitter: float = 0.1, E: float = 1.0,
                  u_bg: float = 1e-6, hfact: float = HFACT) -> Workload:
    """Sedov-Taylor blast on a jittered cubic lattice in the unit box.

    side^3 particles at ((i + 1/2) + U(-jitter, jitter)) * dx, dx = 1/side;
    m = 1/side^3 so rho0 = 1; zero velocity; u = u_bg plus the blast energy E
    spread over the particles within 2.4 dx of the box centre with B-spline
    weights w_j = f(|r_j - c| / (hfact dx)): u_j += E w_j / (m sum_k w_k).
    Open (vacuum) boundaries."""
    g = _rng(seed)
    dx = 1.0 / side
    n = side ** 3
    i = np.arange(side, dtype=np.float64)
    X, Y, Z = np.meshgrid(i, i, i, indexing="ij")
    lat = np.stack([X.ravel(), Y.ravel(), Z.ravel()], axis=1)
    x = (lat + 0.5 + g.uniform(-jitter, jitter, size=(n, 3))) * dx
    m = np.full(n, 1.0 / n)
    u = np.full(n, u_bg)
    # energy deposit: the IC spreads E with a smooth compact profile
    x32 = x.astype(np.float32).astype(np.float64)
    centre = np.array([0.5, 0.5, 0.5])
    hc = hfact * dx
    w = _bspline_shape(np.linalg.norm(x32 - centre, axis=1) / hc)
    sel = w > 0
    u[sel] += E * w[sel] / (m[sel] * w.sum())
    pos, vel = _pack(x, m, np.zeros((n, 3)), u)
    h = np.full(n, hfact * dx, np.float32)
    return Workload("sedov_lattice", pos, vel, h,
                    {"seed": seed, "side": side, "E": E, "centre": centre.tolist(),
                     "rho0": 1.0, "n_deposit": int(sel.sum())})


def shock_tube(nx_left: int, n_left: int, rho: tuple, P: tuple, gamma: float,
               hfact: float = 1.0, x_range: tuple = (-0.5, 0.5), name: str = "shock_tube") -> Workload:
    """A two-state shock tube in a box periodic on every axis (Sect. 4.1-4.2).

    The left state fills [x0, xm) with a cubic lattice of nx_left x n_left x
    n_left particles, spacing dx_L = (xm - x0) / nx_left, xm the midpoint of
    x_range; the right state fills [xm, x1) with a lattice of spacing
    dx_R = dx_L (rho_L / rho_R)^(1/3) (equal masses m = rho_L dx_L^3), the
    cross-section L_yz = n_left dx_L the same for both (so rho_L / rho_R must
    make n_left dx_L / dx_R a whole number).  Zero velocity,
    u = P / ((gamma - 1) rho).  Periodic in x too, the tube holds a second
    interface at x0 = x1 (the same problem mirrored), whose waves start at the
    tube's ends.  meta: box_lo, box_len and the two states."""
    x0, x1 = x_range
    xm = 0.5 * (x0 + x1)
    dxl = (xm - x0) / nx_left
    ratio = (rho[0] / rho[1]) ** (1.0 / 3.0)
    dxr = dxl * ratio
    Lyz = n_left * dxl
    n_right = int(round(Lyz / dxr))
    nx_right = int(round((x1 - xm) / dxr))
    assert abs(n_right * dxr - Lyz) < 1e-9 * Lyz and abs(nx_right * dxr - (x1 - xm)) < 1e-9
    parts = []
    for (nx, ny, dx, xa) in ((nx_left, n_left, dxl, x0), (nx_right, n_right, dxr, xm)):
        i, j, k = np.meshgrid(np.arange(nx), np.arange(ny), np.arange(ny), indexing="ij")
        parts.append(np.stack([xa + (i.ravel() + 0.5) * dx, (j.ravel() + 0.5) * dx,
                               (k.ravel() + 0.5) * dx], axis=1))
    x = np.concatenate(parts)
    nl = parts[0].shape[0]
    n = x.shape[0]
    m = np.full(n, rho[0] * dxl ** 3)
    rh = np.where(np.arange(n) < nl, rho[0], rho[1])
    u = np.where(np.arange(n) < nl, P[0], P[1]) / ((gamma - 1.0) * rh)
    pos, vel = _pack(x, m, np.zeros((n, 3)), u)
    h = (hfact * (m / rh) ** (1.0 / 3.0)).astype(np.float32)
    box_lo = (float(x0), 0.0, 0.0)
    box_len = (float(x1 - x0), float(Lyz), float(Lyz))
    return Workload(name, pos, vel, h,
                    {"box_lo": box_lo, "box_len": box_len, "gamma": gamma, "x_mid": xm,
                     "left": (rho[0], 0.0, P[0]), "right": (rho[1], 0.0, P[1]),
                     "dx": (dxl, dxr)})


def sod_tube(nx_left: int = 256, n_left: int = 24, hfact: float = 1.0) -> Workload:
    """Sod's shock tube as in Sect. 4.1: [rho, P] = [1, 1] left with
    256 x 24 x 24 particles, [0.125, 0.1] right with 128 x 12 x 12, gamma =
    5/3, in [-0.5, 0.5) x L_yz^2."""
    return shock_tube(nx_left, n_left, (1.0, 0.125), (1.0, 0.1), 5.0 / 3.0, hfact, name="sod_tube")


def blast_tube(nx_left: int = 400, n_left: int = 12, hfact: float = 1.0) -> Workload:
    """The blast wave of Sect. 4.2: [rho, P] = [1, 1000] left and [1, 0.1]
    right, 400 x 12 x 12 particles each, gamma = 7/5, in [-0.5, 0.5) x L_yz^2."""
    return shock_tube(nx_left, n_left, (1.0, 1.0), (1000.0, 0.1), 1.4, hfact, name="blast_tube")


def plummer(n: int = 1 << 24, seed: int = 3, a: float = 0.1, rmax: float = 1.0,
            hfact: float = HFACT) -> Workload:
    """Plummer gas sphere (scale a, truncated at rmax), m = 1/n, v = 0,
    u = 1/(6 sqrt(r^2 + a^2)) (G = M = 1); h from the analytic density."""
    g = _rng(seed)
    mmax = rmax ** 3 / (rmax * rmax + a * a) ** 1.5
    X = g.uniform(0.0, mmax, size=n)
    X = np.maximum(X, 1e-300)
    r = a / np.sqrt(X ** (-2.0 / 3.0) - 1.0)
    d = g.normal(size=(n, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    x = d * r[:, None]
    m = np.full(n, 1.0 / n)
    u = 1.0 / (6.0 * np.sqrt(r * r + a * a))
    pos, vel = _pack(x, m, np.zeros((n, 3)), u)
    rho = 3.0 / (4.0 * np.pi * a ** 3) * (1.0 + r * r / (a * a)) ** -2.5 / mmax
    h = (hfact * (m / rho) ** (1.0 / 3.0)).astype(np.float32)
    return Workload("plummer", pos, vel, h, {"seed": seed, "a": a, "rmax": rmax})


def batch_sizes(n_inst: int = 512, seed: int = 4, nmin: int = 4096, nmax: int = 262144):
    """Instance sides s_k = round(n_k^(1/3)), n_k log-uniform in [nmin, nmax]."""
    g = _rng(seed)
    nk = np.exp(g.uniform(np.log(nmin), np.log(nmax), size=n_inst))
    return np.rint(nk ** (1.0 / 3.0)).astype(np.int64)


def sedov_batch(n_inst: int = 512, seed: int = 4, only=None, **kw):
    """Independent Sedov blasts of uneven sizes, packed back to back.
    ``only``: indices of the instances to generate (a rank's share).
    Returns (Workload with those particles, offsets[len + 1])."""
    sides = batch_sizes(n_inst, seed, **kw)
    ks = range(n_inst) if only is None else only
    parts = [sedov_lattice(int(sides[k]), seed=seed * 100003 + k) for k in ks]
    off = np.zeros(len(parts) + 1, np.int64)
    off[1:] = np.cumsum([p.n for p in parts])
    pos = np.concatenate([p.pos for p in parts])
    vel = np.concatenate([p.vel for p in parts])
    h = np.concatenate([p.h for p in parts])
    return Workload("sedov_batch", pos, vel, h, {"seed": seed, "sides": [int(sides[k]) for k in ks]}), off


def probe_indices(n: int, k: int = 1024, seed: int = 5) -> np.ndarray:
    """Seeded probe particles (by original index) for the rollout loss."""
    return np.sort(_rng(seed).choice(n, size=k, replace=False)).astype(np.int64)
