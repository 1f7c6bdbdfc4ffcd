"""Full-size checks on the 128^3 Sedov workload the benchmark times, in the
bench's launch configuration (default parameters, one context).

- keys, sort order, tree and groups: bit-exact over all 2,097,152 particles;
- density: sampled targets, each solved by the oracle against all particles;
- force: sampled targets; the oracle runs on the ball of radius 9 h0 around
  each target, which contains every particle that reaches the target or its
  neighbours (kernels have compact support 2h), checked per target;
- invariants (momentum, energy rate) over all particles;
- a 100-step run: Sedov-Taylor shock radius and energy conservation.
"""
import numpy as np
import pytest

import oracle
from paper_1909_07439_gb300 import inputs

pytestmark = pytest.mark.gpu
SIDE = 128


@pytest.fixture(scope="module")
def sedov():
    import torch
    from paper_1909_07439_gb300 import DeviceState, build, native
    build.build()
    w = inputs.sedov_lattice(SIDE)
    ctx = native.sph_create(w.n, 0)
    s = DeviceState.from_arrays(w.pos, w.vel, w.h)
    p = native.sph_params_default()
    native.sph_build_tree(ctx, s.c, p)
    native.sph_density(ctx, s.c, p)
    native.sph_force(ctx, s.c, p)
    native.sph_sync(ctx)
    yield w, s, p, ctx, native, torch
    native.sph_destroy(ctx)


def _f64(w):
    return (w.pos[:, :3].astype(np.float64), w.vel[:, :3].astype(np.float64),
            w.pos[:, 3].astype(np.float64), w.vel[:, 3].astype(np.float64))


def _samples(w, k=48, seed=99):
    x = w.pos[:, :3].astype(np.float64)
    r = np.linalg.norm(x - 0.5, axis=1)
    rng = np.random.default_rng(seed)
    blast = np.argsort(r)[:8]                                 # hot centre
    edge = np.where(np.min(np.minimum(x, 1 - x), axis=1) < 0.01)[0]
    return np.unique(np.concatenate([blast, rng.choice(edge, 8, replace=False),
                                     rng.choice(w.n, k - 16, replace=False)]))


def test_fullsize_keys_sort_tree_exact(sedov, parity):
    w, s, p, ctx, native, torch = sedov
    keys = oracle.morton_keys(w.pos)
    order = oracle.sort_order(keys)
    sk = keys[order]
    assert parity("keys/sort Sedov 128^3: mismatching keys and perm entries",
                  np.sum(s.numpy("perm").astype(np.int64) != order)
                  + np.sum(s.numpy("keys").view(np.uint64) != sk), 0)
    nodes, groups = native.sph_get_tree(ctx)
    ch = oracle.chop(sk, p.n_leaf)
    for f, ref in (("level", ch.level), ("first", ch.first), ("count", ch.count),
                   ("nchild", ch.nchild)):
        assert np.array_equal(nodes[f], ref), f
    cg = oracle.chop(sk, p.n_group)
    term = cg.nchild == 0
    o = np.argsort(cg.first[term])
    assert np.array_equal(groups["first"], cg.first[term][o])
    assert np.array_equal(groups["count"], cg.count[term][o])


def test_fullsize_density_sampled(sedov, parity):
    w, s, p, ctx, native, torch = sedov
    x, v, m, u = _f64(w)
    t = _samples(w)
    d = oracle.density(x, v, m, w.h, targets=t)
    assert d.failures == 0
    rho = s.in_original_order("rho")[t]
    h = s.in_original_order("h")[t]
    assert parity("density Sedov 128^3 initial (48 sampled): max |rho/rho_o - 1|",
                  np.max(np.abs(rho / d.rho - 1)), 1e-5)
    assert parity("density Sedov 128^3 initial (48 sampled): max |h/h_o - 1|",
                  np.max(np.abs(h / d.h - 1)), 1e-5 / 3)


def test_fullsize_force_sampled(sedov, parity):
    w, s, p, ctx, native, torch = sedov
    x, v, m, u = _f64(w)
    t = _samples(w, k=24, seed=5)
    acc = s.in_original_order("acc")
    ref_a, got_a, ref_du, got_du = [], [], [], []
    h0 = float(w.h[0])
    Ru = 9.0 * h0
    for i in t:
        ball = np.where(np.linalg.norm(x - x[i], axis=1) < Ru)[0]
        k = int(np.searchsorted(ball, i))
        d = oracle.density(x[ball], v[ball], m[ball], w.h[ball])
        f = oracle.force(x[ball], v[ball], m[ball], u[ball], d.h, d.rho, d.omega, targets=[k])
        # everything that reaches the target, or its neighbours, sits well inside the ball
        rr = np.linalg.norm(x[ball] - x[i], axis=1)
        near = rr < 2.0 * np.maximum(d.h[k], d.h) * 1.01
        assert np.all(rr[near] + 2.2 * d.h[near] < Ru)
        ref_a.append(f.acc[0]); got_a.append(acc[i, :3])
        ref_du.append(f.dudt[0]); got_du.append(acc[i, 3])
    ref_a, got_a = np.array(ref_a), np.array(got_a)
    ref_du, got_du = np.array(ref_du), np.array(got_du)
    assert parity("force Sedov 128^3 initial (24 sampled): max |da| / max |a|",
                  np.max(np.abs(got_a - ref_a)) / np.max(np.abs(ref_a)), 1e-4)
    assert parity("force Sedov 128^3 initial (24 sampled): max |d du/dt| / max |du/dt|",
                  np.max(np.abs(got_du - ref_du)) / np.max(np.abs(ref_du)), 1e-4)


def test_fullsize_invariants(sedov):
    w, s, p, ctx, native, torch = sedov
    acc = s.numpy("acc").astype(np.float64)
    pos = s.numpy("pos").astype(np.float64)
    vel = s.numpy("vel").astype(np.float64)
    m = pos[:, 3]
    ma = m[:, None] * acc[:, :3]
    assert np.max(np.abs(ma.sum(0))) <= 2e-6 * np.sum(np.abs(ma))
    tq = np.cross(pos[:, :3] - 0.5, ma)
    assert np.max(np.abs(tq.sum(0))) <= 2e-6 * np.sum(np.abs(tq))
    de = m * (np.sum(vel[:, :3] * acc[:, :3], 1) + acc[:, 3])
    # at t = 0 v = 0: the energy rate is the net conduction, zero pairwise
    assert abs(de.sum()) <= 2e-6 * np.sum(np.abs(m * acc[:, 3]))


def test_sedov_100_steps(sedov, parity):
    w, s0, p, ctx, native, torch = sedov
    from paper_1909_07439_gb300 import DeviceState
    s = DeviceState.from_arrays(w.pos, w.vel, w.h)
    native.sph_build_tree(ctx, s.c, p)
    native.sph_density(ctx, s.c, p)
    native.sph_force(ctx, s.c, p)
    e = torch.zeros(8, dtype=torch.float64, device="cuda")
    native.sph_conserved(ctx, s.c, e)
    E0 = float(e[0] + e[1])
    d_dt = torch.zeros(1, dtype=torch.float32, device="cuda")
    d_t = torch.zeros(1, dtype=torch.float64, device="cuda")
    native.sph_timestep(ctx, s.c, p, d_dt)
    for _ in range(100):
        native.sph_step(ctx, s.c, p, d_dt, d_t)
    native.sph_sync(ctx)
    native.sph_conserved(ctx, s.c, e)
    E1 = float(e[0] + e[1])
    t = float(d_t.item())
    meta = w.meta
    R = oracle.sedov_radius(meta["E"], meta["rho0"], t, 5.0 / 3.0)
    rs, prof, edges = oracle.shock_radius_from_profile(s.numpy("pos")[:, :3], s.numpy("rho"),
                                                       meta["centre"], nbins=80, rmax=2.0 * R)
    print(f"t={t:.4e} R_sedov={R:.4f} R_peak={rs:.4f} dE/E={abs(E1 - E0) / E0:.2e}")
    # measured on GB300: R_peak / R_sedov = 0.987 (the profile's bins are
    # R / 40 wide), dE/E = 1.56e-3 after 100 steps at C_cour = 0.3 (the paper
    # finds the Sedov energy error erratic at this Courant number)
    assert parity("Sedov 128^3, 100 steps: |R_shock / R_similarity - 1|", abs(rs / R - 1), 0.05)
    assert parity("Sedov 128^3, 100 steps: |dE/E|", abs(E1 - E0) / E0, 3e-3)
    # the shell is compressed: peak density well above the ambient rho0 = 1
    assert prof.max() > 1.5


# ------------------------------------------------ the list path in mid-blast
@pytest.fixture(scope="module")
def sedov_mid(sedov):
    """The benchmark's state: initial evaluation, then 6 sph_steps (the bench's
    warm-up), then one more step with fresh counters: the list path timed by
    the benchmark, with no walking fallback."""
    w, s0, p, ctx, native, torch = sedov
    from paper_1909_07439_gb300 import DeviceState
    s = DeviceState.from_arrays(w.pos, w.vel, w.h)
    native.sph_build_tree(ctx, s.c, p)
    native.sph_density(ctx, s.c, p)
    native.sph_force(ctx, s.c, p)
    d_dt = torch.zeros(1, dtype=torch.float32, device="cuda")
    native.sph_timestep(ctx, s.c, p, d_dt)
    for _ in range(6):
        native.sph_step(ctx, s.c, p, d_dt)
    native.sph_sync(ctx)
    native.sph_get_stats(ctx)
    native.sph_step(ctx, s.c, p, d_dt)
    native.sph_sync(ctx)
    stats = native.sph_get_stats(ctx)
    return w, s, p, ctx, native, torch, stats


def _mid_samples(x, rho, n, k=56, seed=7):
    r = np.linalg.norm(x - 0.5, axis=1)
    rng = np.random.default_rng(seed)
    hot = np.argsort(r)[:8]                                   # rarefied hot centre
    shell = np.where(rho > 0.8 * rho.max())[0]                # compressed shell
    edge = np.where(np.min(np.minimum(x, 1 - x), axis=1) < 0.01)[0]
    pick = [hot, rng.choice(shell, min(12, len(shell)), replace=False),
            rng.choice(edge, 8, replace=False), rng.choice(n, k - 28, replace=False)]
    return np.unique(np.concatenate(pick))


def test_midblast_step_uses_lists_only(sedov_mid):
    w, s, p, ctx, native, torch, st = sedov_mid
    assert st["density_rewalks"] == 0 and st["force_rewalks"] == 0
    assert st["list_overflows"] == 0 and st["streamed_groups"] == 0
    assert st["density_pairs"] > 0 and st["force_pairs"] > 0


def test_midblast_density_and_force_parity(sedov_mid, parity):
    # the step's own h and rho (Eqs. 1-4 at the step's positions), then
    # sph_force on the step's lists (current v, u): element by element
    # against the oracle on sampled targets
    w, s, p, ctx, native, torch, _ = sedov_mid
    pos, vel = s.numpy("pos"), s.numpy("vel")
    x, v = pos[:, :3].astype(np.float64), vel[:, :3].astype(np.float64)
    m, u = pos[:, 3].astype(np.float64), vel[:, 3].astype(np.float64)
    hg, rg = s.numpy("h"), s.numpy("rho")
    t = _mid_samples(x, rg, s.n)
    assert len(t) >= 48
    d = oracle.density(x, v, m, hg, targets=t)
    assert d.failures == 0
    assert parity("density Sedov 128^3 mid-blast step (sampled): max |rho/rho_o - 1|",
                  np.max(np.abs(rg[t] / d.rho - 1)), 1e-5)
    assert parity("density Sedov 128^3 mid-blast step (sampled): max |h/h_o - 1|",
                  np.max(np.abs(hg[t] / d.h - 1)), 1e-5 / 3)
    native.sph_get_stats(ctx)
    native.sph_force(ctx, s.c, p)
    native.sph_sync(ctx)
    assert native.sph_get_stats(ctx)["force_rewalks"] == 0
    acc = s.numpy("acc")
    ra, ga, rd, gd = [], [], [], []
    for i in t:
        r = np.linalg.norm(x - x[i], axis=1)
        near = np.where(r < 2.1 * np.maximum(hg[i], hg))[0]       # the force set, with margin
        ball = np.where(r < r[near].max() + 2.3 * hg[near].max())[0]
        dd = oracle.density(x[ball], v[ball], m[ball], hg[ball],
                            targets=np.searchsorted(ball, near))
        assert dd.failures == 0
        hb, rb, ob = (hg[ball].astype(np.float64), rg[ball].astype(np.float64),
                      s.numpy("omega")[ball].astype(np.float64))
        kk = np.searchsorted(ball, near)
        hb[kk], rb[kk], ob[kk] = dd.h, dd.rho, dd.omega
        # every particle that reaches i under the oracle's h is in `near`
        rr = r[ball]
        k = int(np.searchsorted(ball, i))
        assert np.all(np.isin(np.where(rr < 2.0 * np.maximum(hb[k], hb))[0], kk))
        f = oracle.force(x[ball], v[ball], m[ball], u[ball], hb, rb, ob, targets=[k])
        ra.append(f.acc[0]); ga.append(acc[i, :3]); rd.append(f.dudt[0]); gd.append(acc[i, 3])
    ra, ga, rd, gd = map(np.array, (ra, ga, rd, gd))
    err_a = np.max(np.abs(ga - ra)) / np.max(np.abs(ra))
    err_d = np.max(np.abs(gd - rd)) / np.max(np.abs(rd))
    print(f"mid-blast: {len(t)} targets, max|da|/max|a| = {err_a:.2e}, "
          f"max|ddu|/max|du| = {err_d:.2e}")
    assert parity("force Sedov 128^3 mid-blast lists (sampled): max |da| / max |a|", err_a, 1e-4)
    assert parity("force Sedov 128^3 mid-blast lists (sampled): max |d du/dt| / max |du/dt|", err_d, 1e-4)


def test_midblast_lists_bit_exact_sampled(sedov_mid, parity):
    # the production lists at the mid-blast state, filtered by the exact
    # test, against the oracle's brute-force sets for sampled targets
    w, s, p, ctx, native, torch, _ = sedov_mid
    pos, hg = s.numpy("pos"), s.numpy("h")
    t = _mid_samples(pos[:, :3].astype(np.float64), s.numpy("rho"), s.n, seed=11)
    for mode in (0, 1):
        bad = 0
        off = torch.zeros(s.n + 1, dtype=torch.int64, device="cuda")
        total = native.sph_neighbours(ctx, s.c, p, 2 + mode, off)
        idx = torch.zeros(total, dtype=torch.int32, device="cuda")
        native.sph_neighbours(ctx, s.c, p, 2 + mode, off, idx, total)
        off, idx = off.cpu().numpy(), idx.cpu().numpy()
        oo, oi = oracle.neighbours(pos, hg, mode, targets=t)
        for q, i in enumerate(t):
            got = np.sort(idx[off[i]:off[i + 1]])
            bad += not np.array_equal(got, oi[oo[q]:oo[q + 1]])
        assert parity(f"neighbour lists Sedov 128^3 mid-blast (sampled) mode {mode}: "
                      "targets with a different set", bad, 0)
