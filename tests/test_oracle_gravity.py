"""Pins for the oracle's direct-sum self-gravity (the a_grav term of Eq. 9):
hand-computed two- and three-body cases with and without Plummer softening,
Newton's third law, and the potential at the centre of a spherical shell
(-G M / R for any set of points on the shell)."""
import numpy as np
import pytest

import oracle


def test_two_body_by_hand():
    x = np.array([[0.0, 0.0, 0.0], [1.0, 0.0, 0.0]])
    m = np.array([2.0, 3.0])
    a, phi = oracle.gravity(x, m, G=1.0, eps=0.0)
    assert np.allclose(a, [[3.0, 0.0, 0.0], [-2.0, 0.0, 0.0]], rtol=0, atol=1e-15)
    assert np.allclose(phi, [-3.0, -2.0], rtol=0, atol=1e-15)
    # G scales everything; Plummer softening: a = G m d / (d^2 + eps^2)^(3/2)
    a, phi = oracle.gravity(x, m, G=0.5, eps=0.75)
    s = (1.0 + 0.75 ** 2) ** 1.5
    assert np.allclose(a[0], [0.5 * 3.0 / s, 0, 0], rtol=1e-14, atol=0)
    assert np.allclose(phi, [-0.5 * 3.0 / 1.25, -0.5 * 2.0 / 1.25], rtol=1e-14)


def test_three_bodies_by_hand():
    # particle 0 at the origin, 1 at (3, 0, 0), 2 at (0, 4, 0): a_0 = (m1/9, m2/16, 0)
    x = np.array([[0.0, 0.0, 0.0], [3.0, 0.0, 0.0], [0.0, 4.0, 0.0]])
    m = np.array([1.0, 2.0, 5.0])
    a, phi = oracle.gravity(x, m, eps=0.0)
    assert np.allclose(a[0], [2.0 / 9.0, 5.0 / 16.0, 0.0], rtol=1e-14)
    assert abs(phi[0] - (-2.0 / 3.0 - 5.0 / 4.0)) < 1e-14
    # on particle 1: from 0 at distance 3 along -x, from 2 at distance 5 along (-3, 4)/5
    a1 = np.array([-1.0 / 9.0, 0.0, 0.0]) + 5.0 / 25.0 * np.array([-0.6, 0.8, 0.0])
    assert np.allclose(a[1], a1, rtol=1e-14)


def test_newtons_third_law():
    rng = np.random.default_rng(3)
    x = rng.normal(size=(500, 3))
    m = rng.uniform(0.5, 2.0, 500)
    a, _ = oracle.gravity(x, m, eps=0.05)
    p = (m[:, None] * a).sum(0)
    assert np.max(np.abs(p)) < 1e-13 * np.sum(m[:, None] * np.abs(a))


def test_potential_at_the_centre_of_a_shell():
    n = 2000
    k = np.arange(n) + 0.5
    th = np.arccos(1 - 2 * k / n)
    ph = np.pi * (1 + 5 ** 0.5) * k
    R = 0.7
    shell = R * np.stack([np.sin(th) * np.cos(ph), np.sin(th) * np.sin(ph), np.cos(th)], 1)
    x = np.concatenate([[[0.0, 0.0, 0.0]], shell])
    m = np.concatenate([[1e-3], np.full(n, 1.0 / n)])
    a, phi = oracle.gravity(x, m, G=2.0, eps=0.0, targets=np.array([0]))
    assert abs(phi[0] - (-2.0 * 1.0 / R)) < 1e-12   # 2000 terms of rounding
    # and the force there nearly cancels (a Fibonacci shell is nearly uniform)
    assert np.linalg.norm(a[0]) < 1e-3 * 2.0 / R ** 2
