"""Pins for the exact Riemann solver (oracle/riemann.py) behind the Sod and
blast tube tests (Sect. 4.1-4.2): the tabulated star state of Sod's problem
at gamma = 1.4, the Rankine-Hugoniot conditions at every shock, the
isentropic fan with its constant Riemann invariant, continuity of p and u
at the contact, the trivial and the mirrored problem."""
import numpy as np
import pytest

from oracle import riemann as R

SOD = (R.State(1.0, 0.0, 1.0), R.State(0.125, 0.0, 0.1))
BLAST = (R.State(1.0, 0.0, 1000.0), R.State(1.0, 0.0, 0.1))
CASES = [(SOD, 1.4), (SOD, 5.0 / 3.0), (BLAST, 1.4),
         ((R.State(1.0, 0.75, 1.0), R.State(0.125, 0.0, 0.1)), 1.4),      # moving left state
         ((R.State(1.0, -2.0, 0.4), R.State(1.0, 2.0, 0.4)), 1.4),        # two rarefactions
         ((R.State(1.0, 2.0, 0.4), R.State(1.0, -2.0, 0.4)), 1.4)]        # two shocks


def test_sod_star_state_tabulated():
    # the exact star region of Sod's problem at gamma = 1.4, as tabulated in
    # the gas-dynamics literature: p* = 0.30313, u* = 0.92745,
    # rho*_L = 0.42632, rho*_R = 0.26557
    s = R.star_state(*SOD, 1.4)
    assert abs(s.p - 0.30313) < 1e-5
    assert abs(s.u - 0.92745) < 1e-5
    assert abs(s.rho_l - 0.42632) < 1e-5
    assert abs(s.rho_r - 0.26557) < 1e-5


def _flux(rho, u, p, S, gamma):
    w = u - S
    e = p / ((gamma - 1.0) * rho)
    return np.array([rho * w, rho * w * w + p, (rho * (e + 0.5 * w * w) + p) * w])


@pytest.mark.parametrize("case,gamma", CASES)
def test_rankine_hugoniot_at_shocks(case, gamma):
    left, right = case
    lh, lt, uc, rt, rh = R.wave_speeds(left, right, gamma)
    t, eps = 1.0, 1e-9
    shocks = [s for s, a, b in ((lh, lh, lt), (rh, rt, rh)) if a == b]
    for S in shocks:
        a = [float(q[0]) for q in R.sample([S - eps], t, 0.0, left, right, gamma)]
        b = [float(q[0]) for q in R.sample([S + eps], t, 0.0, left, right, gamma)]
        assert abs(a[2] - b[2]) > 1e-6 * max(a[2], b[2])        # a real jump
        fa, fb = _flux(*a, S, gamma), _flux(*b, S, gamma)
        assert np.all(np.abs(fa - fb) <= 1e-10 * np.maximum(np.abs(fa), 1.0))


@pytest.mark.parametrize("case,gamma", CASES)
def test_rarefaction_fans_are_isentropic(case, gamma):
    left, right = case
    lh, lt, uc, rt, rh = R.wave_speeds(left, right, gamma)
    for head, tail, sgn in ((lh, lt, 1.0), (rh, rt, -1.0)):
        if head == tail:
            continue
        xi = np.linspace(min(head, tail), max(head, tail), 101)[1:-1]
        rho, u, p = R.sample(xi, 1.0, 0.0, left, right, gamma)
        s = p / rho ** gamma
        c = np.sqrt(gamma * p / rho)
        J = u + sgn * 2.0 * c / (gamma - 1.0)          # the invariant carried through the fan
        assert np.max(np.abs(s / s[0] - 1)) < 1e-10
        assert np.max(np.abs(J - J[0])) < 1e-10 * max(1.0, abs(J[0]))
        # the fan is a centred wave: u - sgn c = xi inside it
        assert np.max(np.abs(u - sgn * c - xi)) < 1e-10 * max(1.0, np.max(np.abs(xi)))


@pytest.mark.parametrize("case,gamma", CASES)
def test_contact_carries_pressure_and_velocity(case, gamma):
    left, right = case
    s = R.star_state(left, right, gamma)
    a = R.sample([s.u - 1e-9], 1.0, 0.0, left, right, gamma)
    b = R.sample([s.u + 1e-9], 1.0, 0.0, left, right, gamma)
    assert abs(float(a[2][0]) - float(b[2][0])) < 1e-12 * s.p
    assert abs(float(a[1][0]) - float(b[1][0])) < 1e-12 * max(1.0, abs(s.u))
    assert abs(float(a[0][0]) - s.rho_l) < 1e-12 and abs(float(b[0][0]) - s.rho_r) < 1e-12


def test_equal_states_stay_uniform():
    st = R.State(0.7, 0.3, 2.0)
    x = np.linspace(-1, 1, 50)
    rho, u, p = R.sample(x, 0.4, 0.0, st, st, 1.4)
    assert np.allclose(rho, 0.7, rtol=1e-12) and np.allclose(u, 0.3, rtol=1e-12)
    assert np.allclose(p, 2.0, rtol=1e-12)


@pytest.mark.parametrize("case,gamma", CASES)
def test_mirrored_problem(case, gamma):
    left, right = case
    x = np.linspace(-3, 3, 301)
    a = R.sample(x, 0.1, 0.0, left, right, gamma)
    ml, mr = R.State(right.rho, -right.u, right.p), R.State(left.rho, -left.u, left.p)
    b = R.sample(-x, 0.1, 0.0, ml, mr, gamma)
    keep = np.abs(np.abs(x / 0.1) - np.abs(R.star_state(left, right, gamma).u)) > 1e-6
    assert np.allclose(a[0][keep], b[0][keep], rtol=1e-12)
    assert np.allclose(a[1][keep], -b[1][keep], rtol=1e-12, atol=1e-12)
    assert np.allclose(a[2][keep], b[2][keep], rtol=1e-12)
