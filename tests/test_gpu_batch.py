"""Batched form: many independent instances in one state, one tree build, one
persistent density/force launch and a graph-replayed step.  Every instance's
results must equal those of the single-instance path run on that instance
alone (same kernels, same per-instance arithmetic), bit for bit; one instance
is also checked against the FP64 oracle directly."""
import numpy as np
import pytest

import oracle
from paper_1909_07439_gb300 import inputs

pytestmark = pytest.mark.gpu

FIELDS = ("pos", "vel", "acc", "h", "rho", "omega", "drhodt", "vsigmax")


def _batch(n_inst=7, seed=21):
    w, off = inputs.sedov_batch(n_inst, seed=seed, nmin=300, nmax=6000)
    rng = np.random.default_rng(seed)
    w.vel[:, :3] = rng.normal(0, 0.05, (w.n, 3)).astype(np.float32)  # make every term active
    return w, off


@pytest.fixture(scope="module")
def lib():
    import torch
    from paper_1909_07439_gb300 import build, native
    build.build()
    native.load()
    return native, torch


def _plain_run(native, torch, ctx, w, a, b, nsteps, p):
    from paper_1909_07439_gb300 import DeviceState
    s = DeviceState.from_arrays(w.pos[a:b], w.vel[a:b], w.h[a:b])
    native.sph_build_tree(ctx, s.c, p)
    native.sph_density(ctx, s.c, p)
    native.sph_force(ctx, s.c, p)
    dt = torch.zeros(1, dtype=torch.float32, device="cuda")
    t = torch.zeros(1, dtype=torch.float64, device="cuda")
    native.sph_timestep(ctx, s.c, p, dt)
    dts = [dt.item()]
    for _ in range(nsteps):
        native.sph_step(ctx, s.c, p, dt, t)
    native.sph_sync(ctx)
    return s, dt.item(), t.item(), dts[0]


@pytest.mark.parametrize("grav", [False, True])
@pytest.mark.parametrize("nsteps", [0, 3])
def test_batch_equals_single_instance_runs(lib, nsteps, grav):
    # with self-gravity on too: the evaluation and the steps add each
    # instance's own Barnes-Hut term to acc
    native, torch = lib
    from paper_1909_07439_gb300 import DeviceState
    w, off = _batch()
    p = (native.sph_params_default(grav_G=1.0, grav_eps=0.01, grav_theta=0.5) if grav
         else native.sph_params_default())
    ctx = native.sph_create(w.n, 0)
    try:
        s = DeviceState.from_arrays(w.pos, w.vel, w.h)
        d_off = torch.as_tensor(off, device="cuda")
        k = len(off) - 1
        dt = torch.zeros(k, dtype=torch.float32, device="cuda")
        t = torch.zeros(k, dtype=torch.float64, device="cuda")
        native.sph_batch_evaluate(ctx, s.c, d_off, k, p, dt)
        dt0 = dt.cpu().numpy().copy()
        native.sph_batch_step(ctx, s.c, d_off, k, nsteps, p, dt, t)
        native.sph_sync(ctx)
        perm = s.numpy("perm").astype(np.int64)
        got = {f: s.numpy(f) for f in FIELDS}
        for i in range(k):
            a, b = int(off[i]), int(off[i + 1])
            assert np.all((perm[a:b] >= a) & (perm[a:b] < b))   # instances keep their slots
            ps, dti, ti, dt0i = _plain_run(native, torch, ctx, w, a, b, nsteps, p)
            assert dt0[i] == dt0i
            assert np.array_equal(perm[a:b] - a, ps.numpy("perm").astype(np.int64))
            for f in FIELDS:
                assert np.array_equal(got[f][a:b], ps.numpy(f)), (i, f)
            assert dt.cpu().numpy()[i] == dti
            assert t.cpu().numpy()[i] == ti
    finally:
        native.sph_destroy(ctx)


def test_batch_instance_against_oracle(lib, parity):
    native, torch = lib
    from paper_1909_07439_gb300 import DeviceState
    w, off = _batch(n_inst=4, seed=5)
    p = native.sph_params_default()
    ctx = native.sph_create(w.n, 0)
    try:
        s = DeviceState.from_arrays(w.pos, w.vel, w.h)
        d_off = torch.as_tensor(off, device="cuda")
        dt = torch.zeros(4, dtype=torch.float32, device="cuda")
        native.sph_batch_evaluate(ctx, s.c, d_off, 4, p, dt)
        native.sph_sync(ctx)
        a, b = int(off[2]), int(off[3])
        x = w.pos[a:b, :3].astype(np.float64)
        v = w.vel[a:b, :3].astype(np.float64)
        m = w.pos[a:b, 3].astype(np.float64)
        u = w.vel[a:b, 3].astype(np.float64)
        d = oracle.density(x, v, m, w.h[a:b])
        f = oracle.force(x, v, m, u, d.h, d.rho, d.omega)
        perm = s.numpy("perm").astype(np.int64)
        sel = np.where((perm >= a) & (perm < b))[0]
        order = np.argsort(perm[sel])
        rho = s.numpy("rho")[sel][order]
        acc = s.numpy("acc")[sel][order]
        lab = f"batch of 4 instances, instance 2 ({b - a} particles)"
        assert parity(f"density {lab}: max |rho/rho_o - 1|", np.max(np.abs(rho / d.rho - 1)), 1e-5)
        assert parity(f"force {lab}: max |da| / max |a|",
                      np.max(np.abs(acc[:, :3] - f.acc)) / np.max(np.abs(f.acc)), 1e-4)
        assert parity(f"force {lab}: max |d du/dt| / max |du/dt|",
                      np.max(np.abs(acc[:, 3] - f.dudt)) / np.max(np.abs(f.dudt)), 1e-4)
    finally:
        native.sph_destroy(ctx)


def test_batch_rejects_bad_offsets(lib):
    native, torch = lib
    from paper_1909_07439_gb300 import DeviceState
    w, off = _batch(n_inst=3)
    ctx = native.sph_create(w.n, 0)
    try:
        s = DeviceState.from_arrays(w.pos, w.vel, w.h)
        d_off = torch.as_tensor(off, device="cuda")
        dt = torch.zeros(3, dtype=torch.float32, device="cuda")
        with pytest.raises(native.SphError):
            native.sph_batch_evaluate(ctx, s.c, d_off, 0, native.sph_params_default(), dt)
    finally:
        native.sph_destroy(ctx)


@pytest.mark.parametrize("case", ["past_n", "not_increasing", "not_from_zero"])
def test_batch_reports_inconsistent_offsets(lib, case):
    # offsets are device data: the library checks them on the device and
    # reports SPH_ERR_INVALID_ARG through the error word; the pass itself
    # stays inside the state's slots, and the context stays usable
    native, torch = lib
    from paper_1909_07439_gb300 import DeviceState
    w, off = _batch(n_inst=4)
    bad = off.copy()
    if case == "past_n":
        bad[-1] = w.n + 1000
    elif case == "not_increasing":
        bad[2] = bad[1]
    else:
        bad[0] = 5
    ctx = native.sph_create(w.n, 0)
    try:
        s = DeviceState.from_arrays(w.pos, w.vel, w.h)
        p = native.sph_params_default()
        dt = torch.zeros(4, dtype=torch.float32, device="cuda")
        native.sph_batch_evaluate(ctx, s.c, torch.as_tensor(bad, device="cuda"), 4, p, dt)
        with pytest.raises(native.SphError) as e:
            native.sph_sync(ctx)
        assert e.value.status == 1  # SPH_ERR_INVALID_ARG
        s = DeviceState.from_arrays(w.pos, w.vel, w.h)
        native.sph_batch_evaluate(ctx, s.c, torch.as_tensor(off, device="cuda"), 4, p, dt)
        native.sph_sync(ctx)
        assert np.all(np.isfinite(s.numpy("acc")))
    finally:
        native.sph_destroy(ctx)
