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
