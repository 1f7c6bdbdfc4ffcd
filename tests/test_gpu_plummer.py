"""Strongly inhomogeneous workload: Plummer sphere (density contrast ~1e5,
smoothing lengths spanning ~50x).  Keys, sort order and tree bit-exact over
all particles; density on radius-stratified samples solved by the oracle
against all particles; force on samples via the oracle on a ball around each
target that holds every particle reaching it or its neighbours; invariants."""
import numpy as np
import pytest

import oracle
from paper_1909_07439_gb300 import inputs

pytestmark = pytest.mark.gpu


def _run(n):
    from paper_1909_07439_gb300 import DeviceState, build, native
    build.build()
    w = inputs.plummer(n)
    ctx = native.sph_create(w.n, 0)
    s = DeviceState.from_arrays(w.pos, w.vel, w.h)
    p = native.sph_params_default()
    native.sph_build_tree(ctx, s.c, p)
    native.sph_density(ctx, s.c, p)
    native.sph_force(ctx, s.c, p)
    native.sph_sync(ctx)
    return w, s, p, ctx, native


def _stratified(w, k, seed):
    r = np.linalg.norm(w.pos[:, :3].astype(np.float64), axis=1)
    order = np.argsort(r)
    rng = np.random.default_rng(seed)
    cuts = np.array_split(order, k)
    return np.array(sorted(int(rng.choice(c)) for c in cuts))


@pytest.fixture(scope="module")
def mid():
    w, s, p, ctx, native = _run(1 << 18)
    yield w, s, p, ctx, native
    native.sph_destroy(ctx)


def test_plummer_density_and_force_sampled(mid, parity):
    w, s, p, ctx, native = mid
    x = w.pos[:, :3].astype(np.float64)
    v = w.vel[:, :3].astype(np.float64)
    m = w.pos[:, 3].astype(np.float64)
    u = w.vel[:, 3].astype(np.float64)
    t = _stratified(w, 32, 1)
    d = oracle.density(x, v, m, w.h, targets=t)
    assert d.failures == 0
    rho = s.in_original_order("rho")[t]
    assert parity("density Plummer 2^18 (32 stratified): max |rho/rho_o - 1|",
                  np.max(np.abs(rho / d.rho - 1)), 1e-5)
    hg = s.in_original_order("h")
    acc = s.in_original_order("acc")
    ra, ga, rd, gd = [], [], [], []
    for i in _stratified(w, 12, 2):
        Ru = 10.0 * float(hg[i])
        for _ in range(4):
            ball = np.where(np.linalg.norm(x - x[i], axis=1) < Ru)[0]
            k = int(np.searchsorted(ball, i))
            dd = oracle.density(x[ball], v[ball], m[ball], w.h[ball])
            rr = np.linalg.norm(x[ball] - x[i], axis=1)
            near = rr < 2.0 * np.maximum(dd.h[k], dd.h) * 1.01
            if np.all(rr[near] + 2.2 * dd.h[near] < Ru):
                break
            Ru *= 1.6
        assert np.all(rr[near] + 2.2 * dd.h[near] < Ru)
        f = oracle.force(x[ball], v[ball], m[ball], u[ball], dd.h, dd.rho, dd.omega, targets=[k])
        ra.append(f.acc[0]); ga.append(acc[i, :3]); rd.append(f.dudt[0]); gd.append(acc[i, 3])
        # each sampled target's own scale: accelerations vary by decades across the sphere
        assert parity("force Plummer 2^18 (12 stratified): max over targets of |da_i| / max |a_i|",
                      np.max(np.abs(acc[i, :3] - f.acc[0])) / np.max(np.abs(f.acc[0])), 1e-4)
        assert parity("force Plummer 2^18 (12 stratified): max over targets of "
                      "|d du_i| / (|du_i| + 0.01 max |du|)",
                      abs(acc[i, 3] - f.dudt[0]) / (abs(f.dudt[0]) + 1e-2 * np.max(np.abs(rd))), 1e-4)


def test_plummer_invariants(mid):
    w, s, p, ctx, native = mid
    acc = s.numpy("acc").astype(np.float64)
    pos = s.numpy("pos").astype(np.float64)
    vel = s.numpy("vel").astype(np.float64)
    m = pos[:, 3]
    ma = m[:, None] * acc[:, :3]
    assert np.max(np.abs(ma.sum(0))) <= 2e-6 * np.sum(np.abs(ma))
    assert np.max(np.abs(np.cross(pos[:, :3], ma).sum(0))) <= 2e-6 * np.sum(np.abs(np.cross(pos[:, :3], ma)))
    h = s.numpy("h")
    assert h.max() / h.min() > 20       # the workload really spans a wide range of h


def test_plummer_full_size_exact_and_sampled(parity):
    w, s, p, ctx, native = _run(1 << 24)
    try:
        keys = oracle.morton_keys(w.pos)
        order = oracle.sort_order(keys)
        sk = keys[order]
        assert parity("keys/sort Plummer 2^24: mismatching keys and perm entries",
                      np.sum(s.numpy("perm").astype(np.int64) != order)
                      + np.sum(s.numpy("keys").view(np.uint64) != sk), 0)
        nodes, groups = native.sph_get_tree(ctx)
        ch = oracle.chop(sk, p.n_leaf)
        for f, ref in (("level", ch.level), ("first", ch.first), ("count", ch.count)):
            assert np.array_equal(nodes[f], ref), f
        t = _stratified(w, 24, 3)
        x = w.pos[:, :3].astype(np.float64)
        d = oracle.density(x, w.vel[:, :3].astype(np.float64), w.pos[:, 3].astype(np.float64),
                           w.h, targets=t)
        assert d.failures == 0
        assert parity("density Plummer 2^24 (24 stratified): max |rho/rho_o - 1|",
                      np.max(np.abs(s.in_original_order("rho")[t] / d.rho - 1)), 1e-5)
    finally:
        native.sph_destroy(ctx)
