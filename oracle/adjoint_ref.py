"""FP64 PyTorch (CPU) reference for the differentiable rollout.

TEST INFRASTRUCTURE ONLY (used by the test suite): a plain restatement of
Eqs. 1-15 and the kick-drift-kick step (Eqs. 5-7) in torch float64, so that
torch autograd gives the reference gradient of a rollout loss.  Particles keep
their input order (no tree).  Pair sums run over an explicit list of all
pairs within a generous reach, recomputed each step without gradient; terms
beyond the kernel support are exactly zero, so the list only has to be a
superset of the interacting pairs (checked).  The smoothing length is the
Newton fixed point of Eq. 2, unrolled with autograd: the derivative of the
converged iterate is the implicit-function derivative, obtained here without
writing it down (the CUDA adjoint writes it down; this checks it).

The per-step dt sequence is an input (held fixed, no gradient through the
Courant minimum).
"""
from __future__ import annotations

import numpy as np
import torch

C_NORM = 1.0 / np.pi
T = torch.float64


def m4(q):
    """f(q), f'(q) of the M4 cubic spline (support q < 2)."""
    t = torch.clamp(2.0 - q, min=0.0)
    inner = q < 1.0
    f = torch.where(inner, 1.0 - 1.5 * q * q + 0.75 * q ** 3, 0.25 * t ** 3)
    df = torch.where(inner, -3.0 * q + 2.25 * q * q, -0.75 * t * t)
    return f, df


@torch.no_grad()
def pair_list(x, h, reach=1.3):
    """All ordered pairs i != j with |x_i - x_j| < 2 max(h_i, h_j) * reach."""
    n = x.shape[0]
    ii, jj = [], []
    for a in range(0, n, 1024):
        d = torch.cdist(x[a:a + 1024], x)
        R = 2.0 * torch.maximum(h[a:a + 1024, None], h[None, :]) * reach
        ok = d < R
        ok[torch.arange(ok.shape[0]), torch.arange(a, a + ok.shape[0])] = False
        i, j = torch.nonzero(ok, as_tuple=True)
        ii.append(i + a)
        jj.append(j)
    return torch.cat(ii), torch.cat(jj)


def _r(x, i, j):
    dx = x[i] - x[j]
    r = torch.sqrt((dx * dx).sum(1))
    return dx, r


def density(x, m, h0, i, j, hfact=1.2, iters=12):
    """Unrolled Newton on g(h) = sum_j m_j W(r_ij, h) - m (hfact/h)^3 (Eqs. 1-2),
    then rho = m (hfact/h)^3 and Omega (Eq. 4)."""
    n = x.shape[0]
    dx, r = _r(x, i, j)
    M = m * hfact ** 3
    h = h0.detach().clone()
    for _ in range(iters):
        q = r / h[i]
        f, df = m4(q)
        s0 = m + torch.zeros(n, dtype=T).index_add(0, i, m[j] * f)        # self term f(0) = 1
        s1 = 3.0 * m + torch.zeros(n, dtype=T).index_add(0, i, m[j] * (3 * f + q * df))
        gt = C_NORM * s0 - M
        gp = 3.0 * M - C_NORM * s1
        h = h * torch.clamp(1.0 - gt / gp, 0.5, 2.0)   # inactive once converged
    q = r / h[i]
    f, df = m4(q)
    s1 = 3.0 * m + torch.zeros(n, dtype=T).index_add(0, i, m[j] * (3 * f + q * df))
    rho = M / h ** 3
    omega = 1.0 - C_NORM * s1 / (3.0 * M)
    return h, rho, omega


def force(x, v, u, m, h, rho, omega, i, j, gamma=5 / 3, alpha=1.0, beta=2.0, alpha_u=1.0):
    """Accelerations and du/dt (Eqs. 9-15) summed over the pair list."""
    n = x.shape[0]
    dx, r = _r(x, i, j)
    rhat = dx / r[:, None]
    hi, hj = h[i], h[j]
    _, dfi = m4(r / hi)
    _, dfj = m4(r / hj)
    Fi = C_NORM * dfi / hi ** 4
    Fj = C_NORM * dfj / hj ** 4
    P = (gamma - 1.0) * rho * u
    c = torch.sqrt(gamma * P / rho)
    vr = ((v[i] - v[j]) * rhat).sum(1)
    app = vr < 0
    vsi = alpha * c[i] + beta * vr.abs()
    vsj = alpha * c[j] + beta * vr.abs()
    qi = torch.where(app, -0.5 * rho[i] * vsi * vr, torch.zeros_like(vr))
    qj = torch.where(app, -0.5 * rho[j] * vsj * vr, torch.zeros_like(vr))
    Ai = 1.0 / (rho[i] * omega[i])
    Aj = 1.0 / (rho[j] * omega[j])
    coef = m[j] * ((P[i] + qi) / (rho[i] ** 2 * omega[i]) * Fi + (P[j] + qj) / (rho[j] ** 2 * omega[j]) * Fj)
    acc = -torch.zeros((n, 3), dtype=T).index_add(0, i, coef[:, None] * rhat)
    du_p = torch.zeros(n, dtype=T).index_add(0, i, m[j] * vr * Fi)
    du_av = torch.zeros(n, dtype=T).index_add(
        0, i, torch.where(app, m[j] * 0.5 * vsi * vr * vr * Fi, torch.zeros_like(vr)))
    vsu = torch.sqrt((P[i] - P[j]).abs() / (0.5 * (rho[i] + rho[j])))
    du_c = torch.zeros(n, dtype=T).index_add(0, i, m[j] * alpha_u * vsu * (u[i] - u[j]) * 0.5 * (Fi * Ai + Fj * Aj))
    dudt = P / (rho ** 2 * omega) * du_p - du_av / (rho * omega) + du_c
    return acc, dudt


def courant(h, x, v, u, rho, i, j, gamma=5 / 3, alpha=1.0, beta=2.0, c_cour=0.3):
    """C_cour min h / vsigmax over the force sets (Eq. 8), no gradient."""
    with torch.no_grad():
        dx, r = _r(x, i, j)
        inset = r < 2.0 * torch.maximum(h[i], h[j])
        c = torch.sqrt(gamma * (gamma - 1.0) * u)
        vr = ((v[i] - v[j]) * dx).sum(1) / r
        vs = torch.where(inset, alpha * c[i] + beta * vr.abs(), torch.zeros_like(vr))
        vmax = torch.maximum(alpha * c, torch.zeros_like(c).index_reduce(0, i, vs, "amax"))
        return float(c_cour * torch.min(h / vmax))


def rollout(x0, v0, u0, m, h0, alpha, n_steps, probes, dts=None, gamma=5 / 3, beta=2.0,
            alpha_u=1.0, hfact=1.2, c_cour=0.3):
    """Initial evaluation + n_steps KDK steps; loss = mean rho^2 over probes.
    Returns (loss, dts, final h).  dts given: used as is (fixed); else computed."""
    x, v, u = x0, v0, u0
    h = h0.detach().clone()
    i, j = pair_list(x, h, reach=2.5)          # h may double at corners of a lattice
    h, rho, om = density(x, m, h, i, j, hfact, iters=30)
    assert float((h / h0).max()) < 2.5
    a, du = force(x, v, u, m, h, rho, om, i, j, gamma, alpha, beta, alpha_u)
    # Courant step from the signal speeds of the force pass just done (Eq. 8),
    # i.e. with the velocities and energies that pass used
    dt_next = courant(h.detach(), x.detach(), v.detach(), u.detach(), rho.detach(), i, j,
                      gamma, float(alpha), beta, c_cour) if dts is None else None
    out_dts = []
    for k in range(n_steps):
        dt = dt_next if dts is None else float(dts[k])
        out_dts.append(dt)
        vh = v + 0.5 * dt * a
        uh = u + 0.5 * dt * du
        x = x + dt * vh
        vp = v + dt * a
        up = u + dt * du
        h_old = h.detach()
        i, j = pair_list(x.detach(), h_old, reach=1.3)
        h, rho, om = density(x, m, h, i, j, hfact)
        # the list reaches 1.3 x the old h: it holds every interacting pair
        assert float((h.detach() / h_old).max()) < 1.3
        a, du = force(x, vp, up, m, h, rho, om, i, j, gamma, alpha, beta, alpha_u)
        if dts is None:
            dt_next = courant(h.detach(), x.detach(), vp.detach(), up.detach(), rho.detach(), i, j,
                              gamma, float(alpha), beta, c_cour)
        v = vh + 0.5 * dt * a
        u = uh + 0.5 * dt * du
    loss = (rho[probes] ** 2).mean()
    return loss, out_dts, h.detach()
