"""Pins for the oracle's M4 cubic-spline kernel (Sect. 2.3, Eq. 14).

The M4 shape is fixed by: compact support 2h, f(0) = 1, C^2 continuity at
q = 1 and q = 2, and the 3D normalisation 4 pi int W r^2 dr = 1.  Those four
facts determine the piecewise cubic uniquely, so checking them pins every
coefficient; F = dW/dr and dW/dh are pinned by finite differences of W.
"""
import numpy as np
import pytest
from scipy.integrate import quad

import oracle


def W(r, h):
    return oracle.kernel_eval(np.atleast_1d(r), np.atleast_1d(h))[0]


@pytest.mark.parametrize("h", [1.0, 0.37, 2.5])
def test_normalisation(h):
    val, _ = quad(lambda r: 4 * np.pi * r * r * W(r, h)[0], 0, 2 * h, points=[h], epsabs=1e-14,
                  epsrel=1e-13, limit=200)
    assert abs(val - 1.0) < 1e-12


def test_support_and_centre():
    h = 0.7
    assert W(2 * h * (1 + 1e-12), h)[0] == 0.0
    assert W(5.0, h)[0] == 0.0
    # W(0,h) h^3 = C f(0) with f(0) = 1: the constant follows from normalisation
    w0 = W(0.0, h)[0] * h ** 3
    # f is a cubic B-spline: f(1) = f(0)/4
    assert abs(W(h, h)[0] * h ** 3 / w0 - 0.25) < 1e-14
    assert abs(w0 - 1.0 / np.pi) < 1e-15


@pytest.mark.parametrize("q0", [1.0, 2.0])
def test_c2_continuity(q0):
    h = 1.0
    e = 1e-5
    def d2(q):
        return (W(q + e, h)[0] - 2 * W(q, h)[0] + W(q - e, h)[0]) / (e * e)
    # second derivative from either side agrees at the joins (C^2 spline)
    left, right = d2(q0 - 3 * e), d2(q0 + 3 * e)
    assert abs(left - right) < 1e-3 * max(1.0, abs(left))


def test_gradient_and_h_derivative_by_fd():
    rng = np.random.default_rng(0)
    r = rng.uniform(0.01, 1.99, 200)
    h = np.ones_like(r) * rng.uniform(0.5, 2.0)
    r = r * h
    _, F, dwdh = oracle.kernel_eval(r, h)
    e = 1e-6
    Fd = (oracle.kernel_eval(r + e, h)[0] - oracle.kernel_eval(r - e, h)[0]) / (2 * e)
    Hd = (oracle.kernel_eval(r, h + e)[0] - oracle.kernel_eval(r, h - e)[0]) / (2 * e)
    assert np.max(np.abs(F - Fd)) < 1e-6 * np.max(np.abs(F))
    assert np.max(np.abs(dwdh - Hd)) < 1e-6 * np.max(np.abs(dwdh))
    assert np.all(F <= 0.0)  # monotone kernel: gradient points inward


# ------------------------------------------- M6 quintic and Wendland C6 (Sect. 2.3)
KERNELS = [oracle.M4, oracle.M6, oracle.WC6]


def Wk(r, h, k):
    return oracle.kernel_eval(np.atleast_1d(r), np.atleast_1d(h), k)[0]


@pytest.mark.parametrize("k", KERNELS)
@pytest.mark.parametrize("h", [1.0, 0.43])
def test_normalisation_all_kernels(k, h):
    R = oracle.SUPPORT[k]
    pts = [h * q for q in range(1, int(R))]
    val, _ = quad(lambda r: 4 * np.pi * r * r * Wk(r, h, k)[0], 0, R * h, points=pts or None,
                  epsabs=1e-14, epsrel=1e-13, limit=400)
    assert abs(val - 1.0) < 1e-12


@pytest.mark.parametrize("k", KERNELS)
def test_support_radius(k):
    R = oracle.SUPPORT[k]
    h = 0.8
    assert Wk(R * h * (1 + 1e-12), h, k)[0] == 0.0
    assert Wk(R * h * (1 - 1e-3), h, k)[0] > 0.0
    assert oracle.kernel_eval([R * h * (1 + 1e-9)], [h], k)[1][0] == 0.0


def test_central_values():
    # W(0) h^3 = C f(0): M6 f(0) = 3^5 - 6 2^5 + 15 = 66 with C = 1/(120 pi);
    # Wendland C6 f(0) = 1 with C = 1365/(512 pi)
    assert abs(Wk(0.0, 1.0, oracle.M6)[0] - 66.0 / (120.0 * np.pi)) < 1e-15
    assert abs(Wk(0.0, 1.0, oracle.WC6)[0] - 1365.0 / (512.0 * np.pi)) < 1e-15


def _deriv(fn, q, order, e=2e-3):
    # central finite difference of the given order
    from math import comb
    return sum((-1) ** k * comb(order, k) * fn(q + (order / 2 - k) * e) for k in range(order + 1)) / e ** order


@pytest.mark.parametrize("q0", [1.0, 2.0])
def test_m6_smoothness_at_joins(q0):
    # the quintic spline has continuous derivatives up to order 4 at its knots
    f = lambda q: Wk(q, 1.0, oracle.M6)[0] * 120 * np.pi
    for order in (1, 2, 3):
        left = _deriv(f, q0 - 0.05, order)
        right = _deriv(f, q0 + 0.05, order)
        mid = _deriv(f, q0, order)
        # across the knot the derivative changes smoothly (no jump of O(1))
        assert abs(left - 2 * mid + right) < 0.05 * max(1.0, abs(mid)), order


def test_m6_and_wendland_vanish_smoothly_at_support():
    # M6: f ~ (3 - q)^5 near q = 3; Wendland C6: f ~ (1 - q/2)^8 (4 q^3 + ...) near q = 2
    for e in (1e-2, 5e-3):
        f6 = Wk(3.0 - e, 1.0, oracle.M6)[0] * 120 * np.pi
        assert abs(f6 / e ** 5 - 1.0) < 1e-12
        fw = Wk(2.0 - e, 1.0, oracle.WC6)[0] * 512 * np.pi / 1365
        P2 = 4 * 8 + 6.25 * 4 + 4 * 2 + 1
        assert abs(fw / (e / 2) ** 8 / P2 - 1.0) < 0.02


@pytest.mark.parametrize("k", KERNELS)
def test_derivatives_by_fd_all_kernels(k):
    rng = np.random.default_rng(k + 3)
    R = oracle.SUPPORT[k]
    h = np.full(300, rng.uniform(0.5, 2.0))
    r = rng.uniform(0.01, R - 0.01, 300) * h
    _, F, dwdh = oracle.kernel_eval(r, h, k)
    e = 1e-6
    Fd = (oracle.kernel_eval(r + e, h, k)[0] - oracle.kernel_eval(r - e, h, k)[0]) / (2 * e)
    Hd = (oracle.kernel_eval(r, h + e, k)[0] - oracle.kernel_eval(r, h - e, k)[0]) / (2 * e)
    assert np.max(np.abs(F - Fd)) < 1e-6 * np.max(np.abs(F))
    assert np.max(np.abs(dwdh - Hd)) < 1e-6 * np.max(np.abs(dwdh))
    assert np.all(F <= 1e-15)      # monotone kernels: the gradient points inward


@pytest.mark.parametrize("k", [oracle.M6, oracle.WC6])
def test_lattice_continuum_limit_all_kernels(k):
    # for h >> spacing the lattice sum of a unit-normalised kernel tends to rho0 = 1
    g = np.arange(21) - 10.0
    X, Y, Z = np.meshgrid(g, g, g, indexing="ij")
    x = np.stack([X.ravel(), Y.ravel(), Z.ravel()], 1)
    r = np.linalg.norm(x, axis=1)
    for h in (1.8, 2.5):
        s = np.sum(oracle.kernel_eval(r, np.full(r.size, h), k)[0])
        assert abs(s - 1.0) < 2e-3
