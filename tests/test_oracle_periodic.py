"""Pins for the oracle's periodic boundaries (nearest-image separations on
the periodic axes, the Sod and blast tube setups of Sect. 4.1-4.2):

- an explicit copy of the particles shifted by +-L on each periodic axis,
  evaluated with open boundaries, gives the same neighbour sets (bit for bit:
  coordinates on a 2^-20 grid make every FP32 difference exact), densities
  and forces as the periodic evaluation of the originals;
- on a uniform lattice filling a fully periodic box every particle has the
  same neighbourhood: equal densities, zero accelerations and du/dt;
- translating a periodic system along a periodic axis (and wrapping the
  positions) changes nothing.
"""
import numpy as np
import pytest

import oracle

L = np.array([0.0, 0.25, 0.25])       # open x, periodic y and z


def _grid_cloud(n, seed, hfact, kernel):
    rng = np.random.default_rng(seed)
    q = 2.0 ** -20
    x = np.floor(rng.uniform(0, 1, (n, 3)) * np.array([1.0, 0.25, 0.25]) / q) * q
    m = np.full(n, 1.0 / n) * rng.uniform(0.8, 1.2, n)
    v = rng.normal(0, 0.2, (n, 3))
    u = rng.uniform(0.5, 1.5, n)
    rho0 = n / 0.0625
    h = np.full(n, hfact * (1.0 / rho0) ** (1.0 / 3.0))
    assert oracle.SUPPORT[kernel] * h.max() * 1.5 < 0.125
    return x, v, m, u, h


def _images(x, v, m, u):
    """The particles and their copies shifted by -L, 0, +L in y and z."""
    xs, idx = [], []
    for sy in (-1, 0, 1):
        for sz in (-1, 0, 1):
            xs.append(x + np.array([0.0, sy * L[1], sz * L[2]]))
            idx.append(np.arange(len(x)))
    xs = np.concatenate(xs)
    idx = np.concatenate(idx)
    return xs, v[idx], m[idx], u[idx], idx


@pytest.mark.parametrize("kernel,hfact", [(oracle.M4, 1.2), (oracle.M6, 0.9), (oracle.WC6, 1.3)])
def test_periodic_equals_explicit_images(kernel, hfact):
    x, v, m, u, h0 = _grid_cloud(3000, 3 + kernel, hfact, kernel)
    n = len(m)
    d = oracle.density(x, v, m, h0, hfact=hfact, kernel=kernel, box=L)
    assert d.failures == 0
    xi, vi, mi, ui, idx = _images(x, v, m, u)
    # the originals are targets 0..n-1 of the copy (shift (0, 0) is the 5th block)
    t = np.arange(4 * n, 5 * n)
    di = oracle.density(xi, vi, mi, np.tile(h0, 9), targets=t, hfact=hfact, kernel=kernel)
    assert np.max(np.abs(di.h / d.h - 1)) < 1e-12
    assert np.max(np.abs(di.omega - d.omega)) < 1e-12
    assert np.max(np.abs(di.drhodt - d.drhodt)) < 1e-12 * np.max(np.abs(d.drhodt))
    assert np.array_equal(di.nngb, d.nngb)
    f = oracle.force(x, v, m, u, d.h, d.rho, d.omega, kernel=kernel, box=L)
    hh, rr, oo = (np.tile(a, 9) for a in (d.h, d.rho, d.omega))
    fi = oracle.force(xi, vi, mi, ui, hh, rr, oo, targets=t, kernel=kernel)
    assert np.max(np.abs(fi.acc - f.acc)) < 1e-12 * np.max(np.abs(f.acc))
    assert np.max(np.abs(fi.dudt - f.dudt)) < 1e-12 * np.max(np.abs(f.dudt))
    assert np.max(np.abs(fi.vsigmax / f.vsigmax - 1)) < 1e-12
    assert np.array_equal(fi.nforce, f.nforce)
    # neighbour sets, FP32: the same members (mapped back to the originals)
    pos4 = np.concatenate([x, m[:, None]], axis=1).astype(np.float32)
    pos4i = np.concatenate([xi, mi[:, None]], axis=1).astype(np.float32)
    h32 = d.h.astype(np.float32)
    for mode in (0, 1):
        off, ids = oracle.neighbours(pos4, h32, mode, kernel=kernel, box=L)
        oi, ii = oracle.neighbours(pos4i, np.tile(h32, 9), mode, targets=t, kernel=kernel)
        assert np.array_equal(np.diff(off), np.diff(oi))
        for k in range(n):
            a = ids[off[k]:off[k + 1]]
            b = np.sort(idx[ii[oi[k]:oi[k + 1]]])
            assert np.array_equal(a, b), (mode, k)
    # and some pairs really cross the boundary
    y = x[:, 1]
    assert np.any(d.nngb[(y < 0.02) | (y > 0.23)] > 0)


@pytest.mark.parametrize("kernel,hfact", [(oracle.M4, 1.2), (oracle.M6, 1.0)])
def test_uniform_periodic_lattice(kernel, hfact):
    side = 10
    g = (np.arange(side) + 0.5) / side
    x = np.stack(np.meshgrid(g, g, g, indexing="ij"), -1).reshape(-1, 3)
    n = len(x)
    m = np.full(n, 1.0 / n)
    v = np.zeros((n, 3))
    u = np.ones(n)
    box = (1.0, 1.0, 1.0)
    h0 = np.full(n, hfact / side)
    d = oracle.density(x, v, m, h0, hfact=hfact, kernel=kernel, box=box)
    assert d.failures == 0
    assert np.max(np.abs(d.rho / d.rho[0] - 1)) < 1e-12
    assert abs(d.rho[0] - 1.0) < 5e-3           # the summation density of the unit-density lattice
    assert np.all(d.nngb == d.nngb[0])
    f = oracle.force(x, v, m, u, d.h, d.rho, d.omega, kernel=kernel, box=box)
    scale = (2.0 / 3.0) * np.max(np.abs(oracle.kernel_eval(np.array([0.5 / side]),
                                                           np.array([d.h[0]]), kernel)[1]))
    assert np.max(np.abs(f.acc)) < 1e-12 * scale
    assert np.max(np.abs(f.dudt)) < 1e-12 * scale


def test_translation_along_periodic_axes():
    x, v, m, u, h0 = _grid_cloud(3000, 9, 1.2, oracle.M4)
    p = oracle.Params(box=tuple(L), box_lo=(0.0, 0.0, 0.0))
    d = oracle.density(x, v, m, h0, box=L)
    f = oracle.force(x, v, m, u, d.h, d.rho, d.omega, box=L)
    xs = oracle.wrap_positions(x + np.array([0.0, 0.1, 0.17]), p)
    assert np.all((xs[:, 1:] >= 0) & (xs[:, 1:] < 0.25))
    d2 = oracle.density(xs, v, m, h0, box=L)
    f2 = oracle.force(xs, v, m, u, d2.h, d2.rho, d2.omega, box=L)
    assert np.max(np.abs(d2.h / d.h - 1)) < 1e-11
    assert np.max(np.abs(f2.acc - f.acc)) < 1e-10 * np.max(np.abs(f.acc))
    assert np.max(np.abs(f2.dudt - f.dudt)) < 1e-10 * np.max(np.abs(f.dudt))
