"""FP64 PyTorch (CPU) reference for the differentiable rollout.

TEST INFRASTRUCTURE ONLY (used by the test suite): a plain restatement of
Eqs. 1-15 and the kick-drift-kick step (Eqs. 5-7) in torch float64, so that
torch autograd gives the reference gradient of a rollout loss.  Particles keep
their input order (no tree).  Pair sums run over an explicit list of all
pairs within a generous reach, recomputed each step without gradient; terms
beyond the kernel support are exactly zero, so the list only has to be a
superset of the interacting pairs (checked).  The smoothing length is the
root of Eq. 2, found without gradient and then polished by plain Newton steps
under autograd: the derivative of a Newton step taken at the root is the
implicit-function derivative, obtained here without writing it down (the
CUDA adjoint writes it down; this checks it).

The per-step dt sequence is an input (held fixed, no gradient through the
Courant minimum).
"""
from __future__ import annotations

import numpy as np
import torch

T = torch.float64

# Smoothing kernels (Sect. 2.3): W = C f(q) / h^3, q = r / h, zero for q >= R.
# 0 = M4 cubic spline, 1 = M6 quintic spline, 2 = Wendland C6.
M4, M6, WC6 = 0, 1, 2
C_NORM = {M4: 1.0 / np.pi, M6: 1.0 / (120.0 * np.pi), WC6: 1365.0 / (512.0 * np.pi)}
SUPPORT = {M4: 2.0, M6: 3.0, WC6: 2.0}
F0 = {M4: 1.0, M6: 66.0, WC6: 1.0}   # f(0): the self term of the density sum


def m4(q):
    """f(q), f'(q) of the M4 cubic spline (support q < 2)."""
    t = torch.clamp(2.0 - q, min=0.0)
    inner = q < 1.0
    f = torch.where(inner, 1.0 - 1.5 * q * q + 0.75 * q ** 3, 0.25 * t ** 3)
    df = torch.where(inner, -3.0 * q + 2.25 * q * q, -0.75 * t * t)
    return f, df


def m6(q):
    """f(q), f'(q) of the M6 quintic spline (support q < 3): the sum of
    (3 - q)^5, -6 (2 - q)^5 and 15 (1 - q)^5, each where its base is positive."""
    a, b, c = (torch.clamp(k - q, min=0.0) for k in (3.0, 2.0, 1.0))
    f = a ** 5 - 6.0 * b ** 5 + 15.0 * c ** 5
    df = -5.0 * (a ** 4 - 6.0 * b ** 4 + 15.0 * c ** 4)
    return f, df


def wc6(q):
    """f(q), f'(q) of the Wendland C6 kernel (support q < 2): with x = q / 2,
    (1 - x)^8 (32 x^3 + 25 x^2 + 8 x + 1); f' by the product rule."""
    x = 0.5 * q
    s = torch.clamp(1.0 - x, min=0.0)
    P = 32.0 * x ** 3 + 25.0 * x ** 2 + 8.0 * x + 1.0
    dP = 96.0 * x ** 2 + 50.0 * x + 8.0
    f = s ** 8 * P
    df = 0.5 * (-8.0 * s ** 7 * P + s ** 8 * dP)
    return f, df


def kern(q, kernel=M4):
    return (m4, m6, wc6)[kernel](q)


@torch.no_grad()
def pair_list(x, h, reach=1.3, kernel=M4):
    """All ordered pairs i != j with |x_i - x_j| < R max(h_i, h_j) * reach."""
    n = x.shape[0]
    ii, jj = [], []
    for a in range(0, n, 1024):
        d = torch.cdist(x[a:a + 1024], x)
        R = SUPPORT[kernel] * torch.maximum(h[a:a + 1024, None], h[None, :]) * reach
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


def _sums(r, m, h, i, j, n, kernel):
    """s0 = h^3 sum_j m_j W / C and s1 = -h^4 d/dh (sum_j m_j W) / C (Eqs. 1, 4),
    the particle's own term (r = 0) included."""
    f0 = F0[kernel]
    q = r / h[i]
    f, df = kern(q, kernel)
    s0 = f0 * m + torch.zeros(n, dtype=T).index_add(0, i, m[j] * f)
    s1 = 3.0 * f0 * m + torch.zeros(n, dtype=T).index_add(0, i, m[j] * (3 * f + q * df))
    return s0, s1


def density(x, m, h0, i, j, hfact=1.2, iters=12, kernel=M4, polish=3):
    """h from Eq. 2 (g(h) = sum_j m_j W(r_ij, h) - m (hfact/h)^3 = 0, Eq. 1),
    then rho = m (hfact/h)^3 and Omega (Eq. 4).

    The root is found without gradient by Newton steps safeguarded by a
    bracket (a step that leaves the bracket or [h/2, 2h], or meets g' <= 0,
    becomes bisection, or doubling / halving while one side of the bracket is
    open); then `polish` plain Newton steps run with autograd from the
    detached root.  At the root each such step carries dh/dx = -g_x / g_h, the
    implicit-function derivative, without it being written down."""
    n = x.shape[0]
    dx, r = _r(x, i, j)
    M = m * hfact ** 3
    C = C_NORM[kernel]
    with torch.no_grad():
        rd = r.detach()
        h = h0.detach().clone()
        lo = torch.zeros_like(h)
        hi = torch.full_like(h, float("inf"))
        for _ in range(iters):
            s0, s1 = _sums(rd, m, h, i, j, n, kernel)
            gt = C * s0 - M            # h^3 g: < 0 where h is too small
            gp = 3.0 * M - C * s1      # h^4 dg/dh (3 M Omega at the root)
            lo = torch.where(gt < 0, h, lo)
            hi = torch.where(gt < 0, hi, h)
            hn = h * (1.0 - gt / gp)
            ok = (gp > 0) & (hn >= lo) & (hn <= hi) & (hn >= 0.5 * h) & (hn <= 2.0 * h)
            closed = torch.isfinite(hi) & (lo > 0)
            alt = torch.where(closed, 0.5 * (lo + hi), torch.where(gt < 0, 2.0 * h, 0.5 * h))
            h = torch.where(ok, hn, alt)
    h = h.detach()
    for _ in range(polish):
        s0, s1 = _sums(r, m, h, i, j, n, kernel)
        h = h * (1.0 - (C * s0 - M) / (3.0 * M - C * s1))
    _, s1 = _sums(r, m, h, i, j, n, kernel)
    rho = M / h ** 3
    omega = 1.0 - C * s1 / (3.0 * M)
    return h, rho, omega


def force(x, v, u, m, h, rho, omega, i, j, gamma=5 / 3, alpha=1.0, beta=2.0, alpha_u=1.0,
          kernel=M4):
    """Accelerations and du/dt (Eqs. 9-15) summed over the pair list."""
    n = x.shape[0]
    dx, r = _r(x, i, j)
    rhat = dx / r[:, None]
    hi, hj = h[i], h[j]
    _, dfi = kern(r / hi, kernel)
    _, dfj = kern(r / hj, kernel)
    Fi = C_NORM[kernel] * dfi / hi ** 4
    Fj = C_NORM[kernel] * dfj / hj ** 4
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


def courant(h, x, v, u, rho, i, j, gamma=5 / 3, alpha=1.0, beta=2.0, c_cour=0.3, kernel=M4):
    """C_cour min h / vsigmax over the force sets (Eq. 8), no gradient."""
    with torch.no_grad():
        dx, r = _r(x, i, j)
        inset = r < SUPPORT[kernel] * torch.maximum(h[i], h[j])
        c = torch.sqrt(gamma * (gamma - 1.0) * u)
        vr = ((v[i] - v[j]) * dx).sum(1) / r
        vs = torch.where(inset, alpha * c[i] + beta * vr.abs(), torch.zeros_like(vr))
        vmax = torch.maximum(alpha * c, torch.zeros_like(c).index_reduce(0, i, vs, "amax"))
        return float(c_cour * torch.min(h / vmax))


def _scalar(a):
    return float(a.detach()) if torch.is_tensor(a) else float(a)


def rollout(x0, v0, u0, m, h0, alpha, n_steps, probes, dts=None, gamma=5 / 3, beta=2.0,
            alpha_u=1.0, hfact=1.2, c_cour=0.3, kernel=M4):
    """Initial evaluation + n_steps KDK steps; loss = mean rho^2 over probes.
    Returns (loss, dts, final h).  dts given: used as is (fixed); else computed."""
    x, v, u = x0, v0, u0
    h = h0.detach().clone()
    i, j = pair_list(x, h, reach=2.5, kernel=kernel)   # h may double at corners of a lattice
    h, rho, om = density(x, m, h, i, j, hfact, iters=30, kernel=kernel)
    assert float((h / h0).max()) < 2.5
    a, du = force(x, v, u, m, h, rho, om, i, j, gamma, alpha, beta, alpha_u, kernel)
    # Courant step from the signal speeds of the force pass just done (Eq. 8),
    # i.e. with the velocities and energies that pass used
    dt_next = courant(h.detach(), x.detach(), v.detach(), u.detach(), rho.detach(), i, j,
                      gamma, _scalar(alpha), beta, c_cour, kernel) if dts is None else None
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
        i, j = pair_list(x.detach(), h_old, reach=1.3, kernel=kernel)
        h, rho, om = density(x, m, h, i, j, hfact, kernel=kernel)
        # the list reaches 1.3 x the old h: it holds every interacting pair
        assert float((h.detach() / h_old).max()) < 1.3
        a, du = force(x, vp, up, m, h, rho, om, i, j, gamma, alpha, beta, alpha_u, kernel)
        if dts is None:
            dt_next = courant(h.detach(), x.detach(), vp.detach(), up.detach(), rho.detach(), i, j,
                              gamma, _scalar(alpha), beta, c_cour, kernel)
        v = vh + 0.5 * dt * a
        u = uh + 0.5 * dt * du
    loss = (rho[probes] ** 2).mean()
    return loss, out_dts, h.detach()
