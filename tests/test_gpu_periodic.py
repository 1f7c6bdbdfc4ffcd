"""Periodic boundaries on the GPU path vs the FP64 oracle, through the C ABI:
a cloud periodic in y and z (the tube tests of Sect. 4.1-4.2), with
coordinates on a 2^-20 grid.  Neighbour sets bit-exact (separate walk and
production lists), density, force and one KDK step (positions wrapped into
the box) at the M4 parity tolerances, for M4 and M6; a uniform lattice in a
fully periodic box; and the input checks (a particle outside the box, a
support wider than half the period)."""
import numpy as np
import pytest

import oracle
from paper_1909_07439_gb300 import inputs

pytestmark = pytest.mark.gpu

RHO_TOL = 1e-5
ACC_TOL = 1e-4
L = (0.0, 0.25, 0.25)
HFACT = {oracle.M4: 1.2, oracle.M6: 0.9}
KNAME = {oracle.M4: "M4", oracle.M6: "M6"}


@pytest.fixture(scope="module")
def sph():
    import torch
    from paper_1909_07439_gb300 import build, native
    build.build()
    native.load()
    ctx = native.sph_create(1 << 16, 0)
    yield native, ctx, torch
    native.sph_destroy(ctx)


def _cloud(kernel, n=6000, seed=5):
    rng = np.random.default_rng(seed)
    q = 2.0 ** -20
    x = np.floor(rng.uniform(0, 1, (n, 3)) * np.array([1.0, 0.25, 0.25]) / q) * q
    pos = np.concatenate([x, np.full((n, 1), 1.0 / n)], axis=1).astype(np.float32)
    pos[:, 3] *= rng.uniform(0.8, 1.2, n).astype(np.float32)
    vel = np.concatenate([rng.normal(0, 0.3, (n, 3)), rng.uniform(0.5, 1.5, (n, 1))], axis=1)
    h = np.full(n, HFACT[kernel] * (0.0625 / n) ** (1.0 / 3.0), np.float32)
    return inputs.Workload("periodic_cloud", pos, vel.astype(np.float32), h)


def _f64(w):
    return (w.pos[:, :3].astype(np.float64), w.vel[:, :3].astype(np.float64),
            w.pos[:, 3].astype(np.float64), w.vel[:, 3].astype(np.float64))


def _params(native, kernel, **kw):
    return native.sph_params_default(kernel=kernel, hfact=HFACT[kernel], box_lo=(0, 0, 0),
                                     box_len=L, **kw)


_cache = {}


def _oracle(kernel):
    if kernel not in _cache:
        w = _cloud(kernel)
        x, v, m, u = _f64(w)
        d = oracle.density(x, v, m, w.h, hfact=HFACT[kernel], kernel=kernel, box=L)
        assert d.failures == 0
        f = oracle.force(x, v, m, u, d.h, d.rho, d.omega, kernel=kernel, box=L)
        _cache[kernel] = (w, d, f)
    return _cache[kernel]


def _evaluate(native, ctx, w, h, p):
    from paper_1909_07439_gb300 import DeviceState
    s = DeviceState.from_arrays(w.pos, w.vel, h)
    native.sph_build_tree(ctx, s.c, p)
    native.sph_density(ctx, s.c, p)
    native.sph_force(ctx, s.c, p)
    native.sph_sync(ctx)
    return s


@pytest.mark.parametrize("kernel", [oracle.M4, oracle.M6])
def test_periodic_density_force_parity(sph, parity, kernel):
    native, ctx, torch = sph
    w, d, f = _oracle(kernel)
    native.sph_get_stats(ctx)
    s = _evaluate(native, ctx, w, w.h, _params(native, kernel))
    lab = f"{KNAME[kernel]} periodic cloud 6000"
    assert parity(f"density {lab}: max |rho/rho_o - 1|",
                  np.max(np.abs(s.in_original_order("rho") / d.rho - 1)), RHO_TOL)
    assert parity(f"density {lab}: max |h/h_o - 1|",
                  np.max(np.abs(s.in_original_order("h") / d.h - 1)), RHO_TOL / 3)
    om = s.in_original_order("omega")
    assert parity(f"density {lab}: max |dOmega| / max |Omega|",
                  np.max(np.abs(om - d.omega)) / np.max(np.abs(d.omega)), 1e-5)
    dr = s.in_original_order("drhodt")
    assert parity(f"density {lab}: max |d drho/dt| / max |drho/dt|",
                  np.max(np.abs(dr - d.drhodt)) / np.max(np.abs(d.drhodt)), ACC_TOL)
    acc = s.in_original_order("acc")
    assert parity(f"force {lab}: max |da| / max |a|",
                  np.max(np.abs(acc[:, :3] - f.acc)) / np.max(np.abs(f.acc)), ACC_TOL)
    assert parity(f"force {lab}: max |d du/dt| / max |du/dt|",
                  np.max(np.abs(acc[:, 3] - f.dudt)) / np.max(np.abs(f.dudt)), ACC_TOL)
    x, v, m, u = _f64(w)
    lo = oracle.force(x, v, m, u, d.h, d.rho, d.omega, vsig_scale=1 - 1e-4, kernel=kernel, box=L)
    hi = oracle.force(x, v, m, u, d.h, d.rho, d.omega, vsig_scale=1 + 1e-4, kernel=kernel, box=L)
    vs = s.in_original_order("vsigmax")
    assert np.all(vs >= lo.vsigmax * (1 - 1e-5)) and np.all(vs <= hi.vsigmax * (1 + 1e-5))


@pytest.mark.parametrize("mode", [0, 1, 2, 3])
@pytest.mark.parametrize("kernel", [oracle.M4, oracle.M6])
def test_periodic_neighbour_sets_bit_exact(sph, parity, kernel, mode):
    native, ctx, torch = sph
    w, d, _ = _oracle(kernel)
    rng = np.random.default_rng(mode + 61)
    h = (d.h * (rng.uniform(0.8, 1.1, w.n) if mode < 2 else rng.uniform(0.95, 1.0, w.n)))
    h = h.astype(np.float32)
    from paper_1909_07439_gb300 import DeviceState
    s = DeviceState.from_arrays(w.pos, w.vel, h)
    p = _params(native, kernel)
    native.sph_build_tree(ctx, s.c, p)
    off = torch.zeros(w.n + 1, dtype=torch.int64, device="cuda")
    total = native.sph_neighbours(ctx, s.c, p, mode, off)
    idx = torch.zeros(total, dtype=torch.int32, device="cuda")
    native.sph_neighbours(ctx, s.c, p, mode, off, idx, total)
    off, idx = off.cpu().numpy(), idx.cpu().numpy()
    perm = s.numpy("perm").astype(np.int64)
    oo, oi = oracle.neighbours(w.pos, h, mode & 1, kernel=kernel, box=L)
    assert total == oo[-1]
    crossing = bad = 0
    for slot in range(w.n):
        i = perm[slot]
        got = perm[idx[off[slot]:off[slot + 1]]]
        assert len(np.unique(got)) == len(got), (slot, i)
        ref = oi[oo[i]:oo[i + 1]]
        bad += not np.array_equal(np.sort(got), ref)
        dy = np.abs(w.pos[ref, 1] - w.pos[i, 1])
        crossing += int(np.sum(dy > 0.125))
    src = "walk" if mode < 2 else "list build"
    assert parity(f"neighbour sets ({src}) {KNAME[kernel]} periodic cloud 6000 mode {mode & 1}: "
                  "targets with a different set", bad, 0)
    assert crossing > 0       # some members are reached only across the boundary


def _wrapped_diff(a, b):
    d = a - b
    for ax in (1, 2):
        d[:, ax] -= L[ax] * np.round(d[:, ax] / L[ax])
    return d


@pytest.mark.parametrize("kernel", [oracle.M4, oracle.M6])
def test_periodic_step_parity(sph, parity, kernel):
    native, ctx, torch = sph
    w, d, f = _oracle(kernel)
    p = _params(native, kernel)
    s = _evaluate(native, ctx, w, w.h, p)
    x, v, m, u = _f64(w)
    op = oracle.Params(hfact=HFACT[kernel], kernel=kernel, box=L, box_lo=(0, 0, 0))
    st = oracle.SphState(x=x, v=v, u=u, m=m, h=d.h, rho=d.rho, omega=d.omega, drhodt=d.drhodt,
                         acc=f.acc, dudt=f.dudt, vsigmax=f.vsigmax)
    dt = float(np.float32(2.0 * oracle.courant_dt(st, op)))   # 2x Courant: more wrapping
    n1 = oracle.kdk_step(st, dt, op)
    d_dt = torch.full((1,), dt, dtype=torch.float32, device="cuda")
    native.sph_step(ctx, s.c, p, d_dt)
    native.sph_sync(ctx)
    pos = s.in_original_order("pos")
    assert np.all((pos[:, 1:3] >= 0) & (pos[:, 1:3] < 0.25))
    moved = np.sum(np.abs(pos[:, 1:3] - w.pos[:, 1:3]) > 0.125)
    assert moved > 0                                          # some particles wrapped
    lab = f"{KNAME[kernel]} periodic cloud 6000"
    assert parity(f"KDK step, {lab}: max |dx| (nearest image)",
                  np.max(np.abs(_wrapped_diff(pos[:, :3].astype(np.float64), n1.x))), 1e-6)
    vel = s.in_original_order("vel")
    assert parity(f"KDK step, {lab}: max |dv| / max |v|",
                  np.max(np.abs(vel[:, :3] - n1.v)) / np.max(np.abs(n1.v)), 1e-5)
    assert parity(f"KDK step, {lab}: max |u/u_o - 1|", np.max(np.abs(vel[:, 3] / n1.u - 1)), 1e-5)
    assert parity(f"KDK step, {lab}: max |rho/rho_o - 1|",
                  np.max(np.abs(s.in_original_order("rho") / n1.rho - 1)), RHO_TOL)
    acc = s.in_original_order("acc")
    assert parity(f"KDK step, {lab}: max |da| / max |a|",
                  np.max(np.abs(acc[:, :3] - n1.acc)) / np.max(np.abs(n1.acc)), ACC_TOL)
    assert parity(f"KDK step, {lab}: max |d du/dt| / max |du/dt|",
                  np.max(np.abs(acc[:, 3] - n1.dudt)) / np.max(np.abs(n1.dudt)), ACC_TOL)
    # drho/dt of the step, written by its force pass (nearest-image separations)
    dr = s.in_original_order("drhodt")
    assert parity(f"KDK step, {lab}: max |d drho/dt| / max |drho/dt|",
                  np.max(np.abs(dr - n1.drhodt)) / np.max(np.abs(n1.drhodt)), ACC_TOL)


def test_uniform_periodic_lattice(sph):
    native, ctx, torch = sph
    side = 16
    g = ((np.arange(side) + 0.5) / side).astype(np.float32)
    x = np.stack(np.meshgrid(g, g, g, indexing="ij"), -1).reshape(-1, 3)
    n = len(x)
    pos = np.concatenate([x, np.full((n, 1), 1.0 / n, np.float32)], axis=1)
    vel = np.concatenate([np.zeros((n, 3)), np.ones((n, 1))], axis=1).astype(np.float32)
    w = inputs.Workload("lattice", pos, vel, np.full(n, 1.2 / side, np.float32))
    p = native.sph_params_default(box_lo=(0, 0, 0), box_len=(1, 1, 1))
    s = _evaluate(native, ctx, w, w.h, p)
    rho = s.in_original_order("rho")
    assert np.max(np.abs(rho / rho[0] - 1)) < 2e-6
    d = oracle.density(*_f64(w)[:3], w.h, box=(1, 1, 1))
    assert np.max(np.abs(rho / d.rho - 1)) <= RHO_TOL
    acc = s.in_original_order("acc")
    fscale = np.max(np.abs(oracle.kernel_eval(np.array([0.5 / side]), np.array([d.h[0]]))[1]))
    assert np.max(np.abs(acc[:, :3])) < 1e-5 * fscale        # zero up to FP32 rounding


def test_particle_outside_the_box_is_rejected(sph):
    native, ctx, torch = sph
    w = _cloud(oracle.M4, n=2000, seed=8)
    w.pos[17, 1] = 0.25                                   # = lo + L: outside [lo, lo + L)
    from paper_1909_07439_gb300 import DeviceState
    s = DeviceState.from_arrays(w.pos, w.vel, w.h)
    with pytest.raises(native.SphError) as e:
        native.sph_build_tree(ctx, s.c, _params(native, oracle.M4))
        native.sph_sync(ctx)
    assert e.value.status == 1
    native.sph_sync(ctx)


def test_support_wider_than_half_the_period_is_rejected(sph):
    # a force pass whose 2 h reaches past L / 2 = 0.125 reports it
    native, ctx, torch = sph
    w = _cloud(oracle.M4, n=2000, seed=9)
    w.h[:] = 0.07
    from paper_1909_07439_gb300 import DeviceState
    s = DeviceState.from_arrays(w.pos, w.vel, w.h)
    p = _params(native, oracle.M4)
    native.sph_build_tree(ctx, s.c, p)
    native.sph_sync(ctx)
    s.rho.fill_(1.0)
    s.omega.fill_(1.0)
    with pytest.raises(native.SphError) as e:
        native.sph_force(ctx, s.c, p)
        native.sph_sync(ctx)
    assert e.value.status == 1
    native.sph_sync(ctx)
