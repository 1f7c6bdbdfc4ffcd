"""Block (individual power-of-two) time steps on the GPU path vs the oracle's
block step (oracle.block_step, pinned in test_oracle_block.py), through the
C ABI: a Sedov blast whose hot centre sits on level 0 and whose cold
surroundings sit on the top level, and a periodic cloud; the level rule of
sph_block_levels; and the work saved against global steps."""
import numpy as np
import pytest

import oracle
from paper_1909_07439_gb300 import inputs

pytestmark = pytest.mark.gpu

RHO_TOL = 1e-5
ACC_TOL = 1e-4


@pytest.fixture(scope="module")
def sph():
    import torch
    from paper_1909_07439_gb300 import build, native
    build.build()
    native.load()
    ctx = native.sph_create(1 << 16, 0)
    yield native, ctx, torch
    native.sph_destroy(ctx)


def _f64(w):
    return (w.pos[:, :3].astype(np.float64), w.vel[:, :3].astype(np.float64),
            w.pos[:, 3].astype(np.float64), w.vel[:, 3].astype(np.float64))


def _run(sph, w, max_level, op, **pk):
    native, ctx, torch = sph
    from paper_1909_07439_gb300 import DeviceState
    x, v, m, u = _f64(w)
    st = oracle.evaluate(oracle.SphState(x=x, v=v, u=u, m=m, h=w.h.astype(np.float64)), op)
    dt_min = float(np.float32(oracle.courant_dt(st, op)))
    levels = oracle.block_levels(st, dt_min, max_level, op)
    ref = oracle.block_step(st, levels, dt_min, max_level, op)

    s = DeviceState.from_arrays(w.pos, w.vel, w.h)
    p = native.sph_params_default(**pk)
    native.sph_build_tree(ctx, s.c, p)
    native.sph_density(ctx, s.c, p)
    native.sph_force(ctx, s.c, p)
    d_level = torch.as_tensor(levels.astype(np.int32), device="cuda")
    d_dt = torch.full((1,), dt_min, dtype=torch.float32, device="cuda")
    d_t = torch.zeros(1, dtype=torch.float64, device="cuda")
    native.sph_sync(ctx)
    native.sph_get_stats(ctx)
    native.sph_step_block(ctx, s.c, p, max_level, d_level, d_dt, d_t)
    native.sph_sync(ctx)
    stats = native.sph_get_stats(ctx)
    assert abs(d_t.item() / (dt_min * 2 ** max_level) - 1) < 1e-12
    return s, ref, levels, stats, dt_min * 2 ** max_level


def _wrapped(d, box):
    if box is None:
        return d
    for a in range(3):
        if box[a] > 0:
            d[:, a] -= box[a] * np.round(d[:, a] / box[a])
    return d


def _compare(s, ref, span, parity, lab, op, box=None):
    # u: 1e-5 relative, plus what the du/dt tolerance (ACC_TOL of max |du/dt|)
    # can add through the kicks of the block (span = its length)
    pos = s.in_original_order("pos")
    vel = s.in_original_order("vel")
    assert parity(f"block step, {lab}: max |dx|",
                  np.max(np.abs(_wrapped(pos[:, :3].astype(np.float64) - ref.x, box))), 1e-6)
    assert parity(f"block step, {lab}: max |dv| / max |v|",
                  np.max(np.abs(vel[:, :3] - ref.v)) / np.max(np.abs(ref.v)), 1e-5)
    du_tol = ACC_TOL * np.max(np.abs(ref.dudt)) * span
    assert parity(f"block step, {lab}: max |du| / (1e-5 |u| + 1e-4 max |du/dt| span)",
                  np.max(np.abs(vel[:, 3] - ref.u) / (1e-5 * np.abs(ref.u) + du_tol)), 1.0)
    assert parity(f"block step, {lab}: max |rho/rho_o - 1|",
                  np.max(np.abs(s.in_original_order("rho") / ref.rho - 1)), RHO_TOL)
    # every particle's density is solved in the block's last substep: the same
    # solve by the oracle at the device's final (FP32) positions separates the
    # density pass's own error from the rounding of the FP32 drifts above
    d = oracle.density(pos[:, :3].astype(np.float64), vel[:, :3].astype(np.float64),
                       pos[:, 3].astype(np.float64), s.in_original_order("h"), hfact=op.hfact,
                       kernel=op.kernel, box=op.box)
    assert d.failures == 0
    assert parity(f"block step, {lab}: max |rho/rho_o - 1| at the device's final positions",
                  np.max(np.abs(s.in_original_order("rho") / d.rho - 1)), RHO_TOL)
    assert parity(f"block step, {lab}: max |h/h_o - 1|",
                  np.max(np.abs(s.in_original_order("h") / ref.h - 1)), RHO_TOL)
    acc = s.in_original_order("acc")
    assert parity(f"block step, {lab}: max |da| / max |a|",
                  np.max(np.abs(acc[:, :3] - ref.acc)) / np.max(np.abs(ref.acc)), ACC_TOL)
    assert parity(f"block step, {lab}: max |d du/dt| / max |du/dt|",
                  np.max(np.abs(acc[:, 3] - ref.dudt)) / np.max(np.abs(ref.dudt)), ACC_TOL)
    # drho/dt of each particle's last substep, written by the force pass
    dr = s.in_original_order("drhodt")
    assert parity(f"block step, {lab}: max |d drho/dt| / max |drho/dt|",
                  np.max(np.abs(dr - ref.drhodt)) / np.max(np.abs(ref.drhodt)), ACC_TOL)


def test_block_step_sedov(sph, parity):
    w = inputs.sedov_lattice(14, seed=3)
    s, ref, levels, stats, span = _run(sph, w, 3, oracle.Params())
    counts = np.bincount(levels, minlength=4)
    print("levels", counts, "force pairs", stats["force_pairs"])
    assert counts[0] > 0 and counts[3] > 0.5 * w.n          # hot centre low, cold rest high
    _compare(s, ref, span, parity, f"Sedov 14^3 ({w.n}), 4 levels", oracle.Params())


def test_block_step_periodic_m6(sph, parity):
    rng = np.random.default_rng(8)
    n = 4000
    q = 2.0 ** -20
    x = np.floor(rng.uniform(0, 1, (n, 3)) * np.array([1.0, 0.25, 0.25]) / q) * q
    pos = np.concatenate([x, np.full((n, 1), 1.0 / n)], axis=1).astype(np.float32)
    u = np.where(x[:, 0] < 0.3, 8.0, 0.5)                    # a hot slab: two time scales
    vel = np.concatenate([rng.normal(0, 0.2, (n, 3)), u[:, None]], axis=1).astype(np.float32)
    h = np.full(n, 0.9 * (0.0625 / n) ** (1.0 / 3.0), np.float32)
    w = inputs.Workload("cloud", pos, vel, h)
    box = (0.0, 0.25, 0.25)
    op = oracle.Params(hfact=0.9, kernel=oracle.M6, box=box, box_lo=(0, 0, 0))
    s, ref, levels, _, span = _run(sph, w, 2, op, kernel=1, hfact=0.9, box_lo=(0, 0, 0), box_len=box)
    assert len(np.unique(levels)) > 1
    _compare(s, ref, span, parity, f"M6 periodic cloud {n}, 3 levels", op, box)


def test_block_levels_rule(sph):
    native, ctx, torch = sph
    from paper_1909_07439_gb300 import DeviceState
    w = inputs.sedov_lattice(14, seed=3)
    s = DeviceState.from_arrays(w.pos, w.vel, w.h)
    p = native.sph_params_default()
    native.sph_build_tree(ctx, s.c, p)
    native.sph_density(ctx, s.c, p)
    native.sph_force(ctx, s.c, p)
    d_dt = torch.zeros(1, dtype=torch.float32, device="cuda")
    d_ref = torch.zeros(1, dtype=torch.float32, device="cuda")
    d_level = torch.full((w.n,), -1, dtype=torch.int32, device="cuda")
    native.sph_block_levels(ctx, s.c, p, 3, d_dt, d_level)
    native.sph_timestep(ctx, s.c, p, d_ref)
    native.sph_sync(ctx)
    assert d_dt.item() == d_ref.item()
    lv = d_level.cpu().numpy()
    h = s.in_original_order("h")
    vs = s.in_original_order("vsigmax")
    vel = s.in_original_order("vel")
    acc = s.in_original_order("acc")
    with np.errstate(divide="ignore"):
        tu = np.where(acc[:, 3] != 0, vel[:, 3] / np.abs(acc[:, 3]), np.float32(np.inf))
    dtc = np.float32(p.c_cour) * np.minimum(h / vs, tu.astype(np.float32))   # FP32, as the library
    dtm = np.float32(d_dt.item())
    step = dtm * (2.0 ** lv).astype(np.float32)
    assert np.all((lv >= 0) & (lv <= 3))
    assert np.all((lv == 0) | (step <= dtc))
    assert np.all((lv == 3) | (dtm * (2.0 ** (lv + 1)).astype(np.float32) > dtc))


def test_block_step_saves_work(sph):
    # the same span of time: one block of 8 substeps against 8 global steps
    native, ctx, torch = sph
    from paper_1909_07439_gb300 import DeviceState
    w = inputs.sedov_lattice(24, seed=4)
    p = native.sph_params_default()
    pairs = []
    for mode in ("global", "block"):
        s = DeviceState.from_arrays(w.pos, w.vel, w.h)
        native.sph_build_tree(ctx, s.c, p)
        native.sph_density(ctx, s.c, p)
        native.sph_force(ctx, s.c, p)
        d_dt = torch.zeros(1, dtype=torch.float32, device="cuda")
        d_level = torch.zeros(w.n, dtype=torch.int32, device="cuda")
        native.sph_block_levels(ctx, s.c, p, 3, d_dt, d_level)
        native.sph_sync(ctx)
        dt0 = d_dt.item()
        native.sph_get_stats(ctx)
        if mode == "global":
            for _ in range(8):
                d_dt.fill_(dt0)           # sph_step writes the next Courant dt: keep dt_min
                native.sph_step(ctx, s.c, p, d_dt)
        else:
            native.sph_step_block(ctx, s.c, p, 3, d_level, d_dt)
        native.sph_sync(ctx)
        pairs.append(native.sph_get_stats(ctx)["force_pairs"])
    print("force pairs: 8 global steps", pairs[0], "one block", pairs[1])
    assert pairs[1] < 0.5 * pairs[0]


def test_block_level_out_of_range_is_reported(sph):
    # a level outside [0, max_level] is device data: the substep kernel
    # reports it through the error word (read by sph_sync) and steps the
    # particle as level 0
    native, ctx, torch = sph
    from paper_1909_07439_gb300 import DeviceState
    w = inputs.unit_sphere(3000, seed=11, sigma_v=0.1)
    s = DeviceState.from_arrays(w.pos, w.vel, w.h)
    p = native.sph_params_default()
    native.sph_build_tree(ctx, s.c, p)
    native.sph_density(ctx, s.c, p)
    native.sph_force(ctx, s.c, p)
    native.sph_sync(ctx)
    d_dt = torch.zeros(1, dtype=torch.float32, device="cuda")
    d_level = torch.zeros(w.n, dtype=torch.int32, device="cuda")
    native.sph_block_levels(ctx, s.c, p, 2, d_dt, d_level)
    d_level[17] = 3                         # above max_level = 2
    native.sph_step_block(ctx, s.c, p, 2, d_level, d_dt)
    with pytest.raises(native.SphError) as e:
        native.sph_sync(ctx)
    assert e.value.status == 1  # SPH_ERR_INVALID_ARG
    # the context stays usable
    native.sph_build_tree(ctx, s.c, p)
    native.sph_density(ctx, s.c, p)
    native.sph_sync(ctx)
