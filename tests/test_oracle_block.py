"""Pins for the oracle's block time steps (oracle.block_step): the special
cases that reduce to the global kick-drift-kick step (kdk_step, itself
pinned against Eqs. 5-7), and two separated clouds on different levels,
each of which must evolve exactly as its own sequence of global steps."""
import numpy as np

import oracle
from paper_1909_07439_gb300 import inputs


def _state(w, shift=None):
    x = w.pos[:, :3].astype(np.float64)
    if shift is not None:
        x = x + shift
    s = oracle.SphState(x=x, v=w.vel[:, :3].astype(np.float64), u=w.vel[:, 3].astype(np.float64),
                        m=w.pos[:, 3].astype(np.float64), h=w.h.astype(np.float64))
    return oracle.evaluate(s)


def _close(a, b, tol=1e-11):
    for f in ("x", "v", "u", "h", "rho", "acc", "dudt"):
        A, B = getattr(a, f), getattr(b, f)
        assert np.max(np.abs(A - B)) <= tol * max(np.max(np.abs(B)), 1e-300), f


def test_level_zero_is_the_global_step():
    s = _state(inputs.unit_sphere(600, seed=2, sigma_v=0.3))
    dt = 0.5 * oracle.courant_dt(s)
    a = oracle.block_step(s, np.zeros(600, int), dt, 0)
    b = oracle.kdk_step(s, dt)
    _close(a, b)
    # and 2^L substeps of level 0 are L global steps in a row
    a = oracle.block_step(s, np.zeros(600, int), dt, 2)
    b = s
    for _ in range(4):
        b = oracle.kdk_step(b, dt)
    _close(a, b)


def test_one_level_for_all_is_one_long_step():
    s = _state(inputs.unit_sphere(600, seed=3, sigma_v=0.3))
    dt = 0.25 * oracle.courant_dt(s)
    a = oracle.block_step(s, np.full(600, 2), dt, 2)
    b = oracle.kdk_step(s, 4 * dt)
    _close(a, b, 1e-10)


def test_separated_clouds_on_two_levels():
    # cloud A (level 0) and cloud B (level 2) far apart: A takes four global
    # steps of dt, B one global step of 4 dt, neither sees the other
    wa = inputs.unit_sphere(500, seed=4, sigma_v=0.3)
    wb = inputs.unit_sphere(400, seed=5, sigma_v=0.3)
    sa, sb = _state(wa), _state(wb, shift=np.array([10.0, 0.0, 0.0]))
    both = oracle.SphState(**{f: np.concatenate([getattr(sa, f), getattr(sb, f)])
                              for f in ("x", "v", "u", "m", "h", "rho", "omega", "drhodt", "acc",
                                        "dudt", "vsigmax")})
    dt = 0.25 * min(oracle.courant_dt(sa), oracle.courant_dt(sb))
    lv = np.concatenate([np.zeros(500, int), np.full(400, 2)])
    r = oracle.block_step(both, lv, dt, 2)
    ra = sa
    for _ in range(4):
        ra = oracle.kdk_step(ra, dt)
    rb = oracle.kdk_step(sb, 4 * dt)
    part = lambda st, sl: oracle.SphState(**{f: getattr(st, f)[sl] for f in
                                             ("x", "v", "u", "m", "h", "rho", "omega", "drhodt",
                                              "acc", "dudt", "vsigmax")})
    _close(part(r, slice(0, 500)), ra, 1e-10)
    _close(part(r, slice(500, 900)), rb, 1e-10)


def test_levels_follow_the_courant_and_energy_rule():
    s = _state(inputs.sedov_lattice(10, seed=2))
    dt_min = oracle.courant_dt(s)
    lv = oracle.block_levels(s, dt_min, 3)
    dtc = 0.3 * np.minimum(s.h / s.vsigmax, s.u / np.abs(s.dudt))
    # level 0 also takes the particles whose energy time is below dt_min
    assert np.all((lv == 0) | (dt_min * 2.0 ** lv <= dtc * (1 + 1e-12)))
    assert np.any(dtc < dt_min)
    assert np.all((lv == 3) | (dt_min * 2.0 ** (lv + 1) > dtc))
    assert lv.min() == 0 and lv.max() > 0
