"""GPU path vs the FP64 oracle, element by element, through the C ABI.

Bars: keys, sort order, tree, groups and neighbour sets bit-exact; rho within
1e-5 relative; accelerations and du/dt within 1e-4 of max|.|.  All inputs
come from the seeded generators; every expected value from the oracle.
"""
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
    ctx = native.sph_create(1 << 18, 0)
    yield native, ctx, torch
    native.sph_destroy(ctx)


def upload(native, w):
    from paper_1909_07439_gb300 import DeviceState
    return DeviceState.from_arrays(w.pos, w.vel, w.h)


def f64(w):
    return (w.pos[:, :3].astype(np.float64), w.vel[:, :3].astype(np.float64),
            w.pos[:, 3].astype(np.float64), w.vel[:, 3].astype(np.float64))


def small_cases():
    a = inputs.unit_sphere(8192, seed=1)                      # C1: N = 8192 unit sphere
    b = inputs.unit_sphere(3001, seed=7, sigma_v=0.3)         # ragged, several tiles
    rng = np.random.default_rng(7)
    b.pos[:, 3] *= rng.uniform(0.5, 1.5, b.n).astype(np.float32)   # unequal masses
    b.vel[:, 3] *= rng.uniform(0.5, 2.0, b.n).astype(np.float32)   # pressure gradients
    return {"c1_8192": a, "ragged_3001": b}


CASES = small_cases()


def evaluate_gpu(native, ctx, w, **pk):
    s = upload(native, w)
    p = native.sph_params_default(**pk)
    native.sph_build_tree(ctx, s.c, p)
    native.sph_density(ctx, s.c, p)
    native.sph_force(ctx, s.c, p)
    native.sph_sync(ctx)
    return s, p


_oracle_cache = {}


def oracle_eval(name, w):
    if name not in _oracle_cache:
        x, v, m, u = f64(w)
        d = oracle.density(x, v, m, w.h)
        assert d.failures == 0
        f = oracle.force(x, v, m, u, d.h, d.rho, d.omega)
        _oracle_cache[name] = (d, f)
    return _oracle_cache[name]


# ------------------------------------------------------------ keys / sort / tree
@pytest.mark.parametrize("n", [1, 2, 37, 1000, 8192])
def test_keys_sort_perm_bit_exact(sph, parity, n):
    native, ctx, torch = sph
    w = inputs.unit_sphere(n, seed=n)
    s = upload(native, w)
    p = native.sph_params_default()
    native.sph_build_tree(ctx, s.c, p)
    native.sph_sync(ctx)
    keys_o = oracle.morton_keys(w.pos)
    order = oracle.sort_order(keys_o)
    assert parity(f"keys/sort n={n}: mismatching keys and perm entries",
                  np.sum(s.numpy("perm").astype(np.int64) != order)
                  + np.sum(s.numpy("keys").view(np.uint64) != keys_o[order]), 0)
    assert np.array_equal(s.numpy("pos"), w.pos[order])     # permuted, bit for bit
    assert np.array_equal(s.numpy("h"), w.h[order])


def _tight_clusters(n, size, seed):
    # clusters of `size` distinct particles within ~1e-6 of the box: their keys
    # share the top 32 bits (cells of 2^-10 of the box per axis) and differ
    # below, so the sort has to order them by the low 32 bits
    w = inputs.unit_sphere(n, seed=seed)
    rng = np.random.default_rng(seed)
    bases = rng.choice(n, size=n // (2 * size), replace=False)
    k = 0
    for b in bases:
        for q in range(size):
            if k >= n:
                break
            if k != b:
                w.pos[k, :3] = w.pos[b, :3] + rng.uniform(-1e-6, 1e-6, 3).astype(np.float32)
            k += 1
    return w


@pytest.mark.parametrize("size", [3, 20, 40])
def test_sort_of_keys_that_share_their_top_bits(sph, size):
    # runs of up to 32 equal top bits are ordered by the fix-up pass, longer
    # runs by the passes over all 64 bits
    native, ctx, torch = sph
    w = _tight_clusters(6000, size, seed=size)
    s = upload(native, w)
    native.sph_build_tree(ctx, s.c, native.sph_params_default())
    native.sph_sync(ctx)
    keys_o = oracle.morton_keys(w.pos)
    order = oracle.sort_order(keys_o)
    top = keys_o[order] >> np.uint64(32)
    assert np.sum(top[1:] == top[:-1]) > 0          # the case has runs
    assert np.array_equal(s.numpy("perm").astype(np.int64), order)
    assert np.array_equal(s.numpy("keys").view(np.uint64), keys_o[order])


def _clustered(n=20000):
    w = inputs.plummer(n, seed=11)
    # a block of exact duplicates exercises identical keys (depth-21 leaves)
    w.pos[100:160] = w.pos[100]
    return w


@pytest.mark.parametrize("case", ["c1", "plummer_dups", "tiny"])
def test_tree_and_groups_exact(sph, case):
    native, ctx, torch = sph
    w = {"c1": CASES["c1_8192"], "plummer_dups": _clustered(), "tiny": inputs.unit_sphere(5)}[case]
    s = upload(native, w)
    p = native.sph_params_default()
    native.sph_build_tree(ctx, s.c, p)
    native.sph_sync(ctx)
    nodes, groups = native.sph_get_tree(ctx)
    sk = oracle.morton_keys(w.pos)
    sk = sk[oracle.sort_order(sk)]
    ch = oracle.chop(sk, p.n_leaf)
    assert np.array_equal(nodes["level"], ch.level)
    assert np.array_equal(nodes["first"], ch.first)
    assert np.array_equal(nodes["count"], ch.count)
    assert np.array_equal(nodes["nchild"], ch.nchild)
    assert np.array_equal(np.where(ch.nchild > 0, nodes["child"], -1),
                          np.where(ch.nchild > 0, ch.child_first, -1))
    cg = oracle.chop(sk, p.n_group)
    term = cg.nchild == 0
    assert np.array_equal(groups["first"], np.sort(cg.first[term]))
    assert np.array_equal(groups["count"], cg.count[term][np.argsort(cg.first[term])])


@pytest.mark.parametrize("mode", [0, 1])
@pytest.mark.parametrize("case", ["c1_8192", "ragged_3001"])
def test_neighbour_sets_bit_exact(sph, parity, mode, case):
    native, ctx, torch = sph
    w = CASES[case]
    rng = np.random.default_rng(mode + 17)
    h = (w.h * rng.uniform(0.7, 1.4, w.n)).astype(np.float32)   # same h array on both sides
    s = upload(native, inputs.Workload("x", w.pos, w.vel, h))
    p = native.sph_params_default()
    native.sph_build_tree(ctx, s.c, p)
    off = torch.zeros(w.n + 1, dtype=torch.int64, device="cuda")
    total = native.sph_neighbours(ctx, s.c, p, mode, off)
    idx = torch.zeros(total, dtype=torch.int32, device="cuda")
    native.sph_neighbours(ctx, s.c, p, mode, off, idx, total)
    off, idx = off.cpu().numpy(), idx.cpu().numpy()
    perm = s.numpy("perm").astype(np.int64)
    oo, oi = oracle.neighbours(w.pos, h, mode)
    assert total == oo[-1]
    bad = 0
    for slot in range(w.n):
        i = perm[slot]
        got = np.sort(perm[idx[off[slot]:off[slot + 1]]])
        bad += not np.array_equal(got, oi[oo[i]:oo[i + 1]])
    assert parity(f"neighbour sets (walk) {case} mode {mode}: targets with a different set", bad, 0)


@pytest.mark.parametrize("mode", [0, 1, 2, 3])
@pytest.mark.parametrize("case", ["c1_8192", "ragged_3001"])
def test_production_lists_bit_exact(sph, parity, mode, case):
    # the neighbour lists the density and force passes read (list-building walk
    # of the density pass, shared walks, leaf caps), each filtered by the exact
    # canonical test: the density set (mode 0) or force set (mode 1) bit for bit
    # at the converged h (the production state) and at h shrunk by up to 5 %
    # per particle (the lists hold at most 192 entries: a larger h could
    # overflow them, and then the walking kernels take over)
    native, ctx, torch = sph
    w = CASES[case]
    d, _ = oracle_eval(case, w)
    rng = np.random.default_rng(mode + 31)
    h = (d.h * (1.0 if mode < 2 else rng.uniform(0.95, 1.0, w.n))).astype(np.float32)
    mode &= 1
    s = upload(native, inputs.Workload("x", w.pos, w.vel, h))
    p = native.sph_params_default()
    native.sph_build_tree(ctx, s.c, p)
    native.sph_get_stats(ctx)
    off = torch.zeros(w.n + 1, dtype=torch.int64, device="cuda")
    total = native.sph_neighbours(ctx, s.c, p, 2 + mode, off)
    assert native.sph_get_stats(ctx)["list_overflows"] == 0
    idx = torch.zeros(total, dtype=torch.int32, device="cuda")
    native.sph_neighbours(ctx, s.c, p, 2 + mode, off, idx, total)
    off, idx = off.cpu().numpy(), idx.cpu().numpy()
    perm = s.numpy("perm").astype(np.int64)
    oo, oi = oracle.neighbours(w.pos, h, mode)
    assert total == oo[-1]
    bad = 0
    for slot in range(w.n):
        i = perm[slot]
        got = perm[idx[off[slot]:off[slot + 1]]]
        assert len(np.unique(got)) == len(got), (slot, i)        # no entry twice
        bad += not np.array_equal(np.sort(got), oi[oo[i]:oo[i + 1]])
    assert parity(f"neighbour lists (list build) {case} mode {mode}: targets with a different set",
                  bad, 0)


def test_list_path_after_steps(sph, parity):
    # a few steps, then sph_density and sph_force from the converged h: both
    # passes read the neighbour lists (no walking fallback) and give the
    # oracle's values for the stepped state
    native, ctx, torch = sph
    w = CASES["ragged_3001"]
    s, p = evaluate_gpu(native, ctx, w)
    d_dt = torch.zeros(1, dtype=torch.float32, device="cuda")
    native.sph_timestep(ctx, s.c, p, d_dt)
    for _ in range(3):
        native.sph_step(ctx, s.c, p, d_dt)
    native.sph_sync(ctx)
    native.sph_get_stats(ctx)
    native.sph_density(ctx, s.c, p)
    native.sph_force(ctx, s.c, p)
    native.sph_sync(ctx)
    st = native.sph_get_stats(ctx)
    assert st["density_rewalks"] == 0 and st["force_rewalks"] == 0 and st["list_overflows"] == 0
    assert st["force_pairs"] > 0
    pos = s.in_original_order("pos")
    vel = s.in_original_order("vel")
    x, v = pos[:, :3].astype(np.float64), vel[:, :3].astype(np.float64)
    m, u = pos[:, 3].astype(np.float64), vel[:, 3].astype(np.float64)
    d = oracle.density(x, v, m, s.in_original_order("h"))
    assert d.failures == 0
    assert parity("list path after 3 steps, ragged 3001: max |rho/rho_o - 1|",
                  np.max(np.abs(s.in_original_order("rho") / d.rho - 1)), RHO_TOL)
    f = oracle.force(x, v, m, u, d.h, d.rho, d.omega)
    acc = s.in_original_order("acc")
    assert parity("list path after 3 steps, ragged 3001: max |da| / max |a|",
                  np.max(np.abs(acc[:, :3] - f.acc)) / np.max(np.abs(f.acc)), ACC_TOL)
    assert parity("list path after 3 steps, ragged 3001: max |d du/dt| / max |du/dt|",
                  np.max(np.abs(acc[:, 3] - f.dudt)) / np.max(np.abs(f.dudt)), ACC_TOL)


# ------------------------------------------------------------------ density
@pytest.mark.parametrize("case", ["c1_8192", "ragged_3001"])
def test_density_parity(sph, parity, case):
    native, ctx, torch = sph
    w = CASES[case]
    s, p = evaluate_gpu(native, ctx, w)
    d, _ = oracle_eval(case, w)
    rho = s.in_original_order("rho")
    h = s.in_original_order("h")
    om = s.in_original_order("omega")
    dr = s.in_original_order("drhodt")
    assert parity(f"density {case}: max |rho/rho_o - 1|", np.max(np.abs(rho / d.rho - 1)), RHO_TOL)
    assert parity(f"density {case}: max |h/h_o - 1|", np.max(np.abs(h / d.h - 1)), RHO_TOL / 3)
    assert parity(f"density {case}: max |dOmega| / max |Omega|",
                  np.max(np.abs(om - d.omega)) / np.max(np.abs(d.omega)), 1e-5)
    assert parity(f"density {case}: max |d drho/dt| / max |drho/dt|",
                  np.max(np.abs(dr - d.drhodt)) / np.max(np.abs(d.drhodt)), ACC_TOL)


def test_density_fixed_iterations(sph, parity):
    native, ctx, torch = sph
    w = CASES["ragged_3001"]
    s, p = evaluate_gpu(native, ctx, w, density_iters=3)
    x, v, m, u = f64(w)
    d3 = oracle.density(x, v, m, w.h, fixed_iters=3)
    h = s.in_original_order("h")
    # three Newton updates from the same h0; both sides take the same branch
    rel = np.abs(h / d3.h - 1)
    worst = np.argsort(rel)[-5:]
    print("fixed-3 worst rel err", rel[worst], "h0", w.h[worst], "h3", d3.h[worst])
    assert parity("density, 3 fixed Newton iterations, ragged 3001: max |h/h_o - 1|", np.max(rel), 1e-5)


# -------------------------------------------------------------------- force
@pytest.mark.parametrize("case", ["c1_8192", "ragged_3001"])
def test_force_parity(sph, parity, case):
    native, ctx, torch = sph
    w = CASES[case]
    s, p = evaluate_gpu(native, ctx, w)
    d, f = oracle_eval(case, w)
    acc = s.in_original_order("acc")
    amax = np.max(np.abs(f.acc))
    assert parity(f"force {case}: max |da| / max |a|", np.max(np.abs(acc[:, :3] - f.acc)) / amax, ACC_TOL)
    assert parity(f"force {case}: max |d du/dt| / max |du/dt|",
                  np.max(np.abs(acc[:, 3] - f.dudt)) / np.max(np.abs(f.dudt)), ACC_TOL)
    # vsigmax is a max over a set: bracket it by the sets at radius (1 -/+ 1e-4)
    x, v, m, u = f64(w)
    lo = oracle.force(x, v, m, u, d.h, d.rho, d.omega, vsig_scale=1 - 1e-4).vsigmax
    hi = oracle.force(x, v, m, u, d.h, d.rho, d.omega, vsig_scale=1 + 1e-4).vsigmax
    vs = s.in_original_order("vsigmax")
    assert np.all(vs >= lo * (1 - 1e-5)) and np.all(vs <= hi * (1 + 1e-5))


@pytest.mark.parametrize("shape", [(4, 2, 4), (16, 8, 2), (16, 1, 4), (8, 4, 4)])
def test_launch_shapes_keep_parity(sph, parity, shape):
    # the autotuner's launch shapes of the list pair kernels (targets per batch,
    # warps per block, entries per iteration) change only the FP32 summation
    # order, on the walking first evaluation and on the list path after it
    native, ctx, torch = sph
    t, wp, u = shape
    w = CASES["ragged_3001"]
    s, p = evaluate_gpu(native, ctx, w, pair_targets=t, pair_warps=wp, pair_unroll=u, n_group=16)
    d, f = oracle_eval("ragged_3001", w)
    # then both passes again from the converged h: every batch on the list kernels
    native.sph_get_stats(ctx)
    native.sph_density(ctx, s.c, p)
    native.sph_force(ctx, s.c, p)
    native.sph_sync(ctx)
    st = native.sph_get_stats(ctx)
    assert st["density_rewalks"] == 0 and st["force_rewalks"] == 0 and st["list_overflows"] == 0
    assert parity("launch shapes (list path), ragged 3001: max |rho/rho_o - 1|",
                  np.max(np.abs(s.in_original_order("rho") / d.rho - 1)), RHO_TOL)
    acc = s.in_original_order("acc")
    assert parity("launch shapes (list path), ragged 3001: max |da| / max |a|",
                  np.max(np.abs(acc[:, :3] - f.acc)) / np.max(np.abs(f.acc)), ACC_TOL)
    assert parity("launch shapes (list path), ragged 3001: max |d du/dt| / max |du/dt|",
                  np.max(np.abs(acc[:, 3] - f.dudt)) / np.max(np.abs(f.dudt)), ACC_TOL)


def test_bad_launch_shape_rejected(sph):
    native, ctx, torch = sph
    s = upload(native, inputs.unit_sphere(64))
    for bad in ({"pair_targets": 5}, {"pair_warps": 3}, {"pair_unroll": 8}):
        with pytest.raises(native.SphError) as e:
            native.sph_build_tree(ctx, s.c, native.sph_params_default(**bad))
        assert e.value.status == 1


def test_force_invariants(sph):
    native, ctx, torch = sph
    w = CASES["ragged_3001"]
    s, p = evaluate_gpu(native, ctx, w)
    acc = s.in_original_order("acc").astype(np.float64)
    x, v, m, u = f64(w)
    ma = m[:, None] * acc[:, :3]
    assert np.max(np.abs(ma.sum(0))) <= 2e-6 * np.sum(np.abs(ma))
    de = m * (np.sum(v * acc[:, :3], 1) + acc[:, 3])
    assert abs(de.sum()) <= 2e-6 * np.sum(np.abs(m * np.sum(v * acc[:, :3], 1)) + np.abs(m * acc[:, 3]))


# ---------------------------------------------------------- step / reductions
def test_timestep_and_step_parity(sph, parity):
    native, ctx, torch = sph
    w = CASES["ragged_3001"]
    s, p = evaluate_gpu(native, ctx, w)
    d, f = oracle_eval("ragged_3001", w)
    x, v, m, u = f64(w)
    st = oracle.SphState(x=x, v=v, u=u, m=m, h=d.h, rho=d.rho, omega=d.omega, drhodt=d.drhodt,
                         acc=f.acc, dudt=f.dudt, vsigmax=f.vsigmax)
    dt_o = oracle.courant_dt(st)
    d_dt = torch.zeros(1, dtype=torch.float32, device="cuda")
    native.sph_timestep(ctx, s.c, p, d_dt)
    assert parity("Courant dt, ragged 3001: |dt/dt_o - 1|", abs(d_dt.item() / dt_o - 1), 1e-4)
    d_dt.fill_(dt_o)
    d_t = torch.zeros(1, dtype=torch.float64, device="cuda")
    native.sph_step(ctx, s.c, p, d_dt, d_t)
    native.sph_sync(ctx)
    assert abs(d_t.item() - np.float32(dt_o)) <= 1e-12
    n1 = oracle.kdk_step(st, float(np.float32(dt_o)))
    pos = s.in_original_order("pos")
    vel = s.in_original_order("vel")
    rho = s.in_original_order("rho")
    acc = s.in_original_order("acc")
    assert parity("KDK step, ragged 3001: max |dx|", np.max(np.abs(pos[:, :3] - n1.x)), 1e-6)
    vscale = np.max(np.abs(n1.v))
    assert parity("KDK step, ragged 3001: max |dv| / max |v|", np.max(np.abs(vel[:, :3] - n1.v)) / vscale, 1e-5)
    assert parity("KDK step, ragged 3001: max |u/u_o - 1|", np.max(np.abs(vel[:, 3] / n1.u - 1)), 1e-5)
    assert parity("KDK step, ragged 3001: max |rho/rho_o - 1|", np.max(np.abs(rho / n1.rho - 1)), RHO_TOL)
    assert parity("KDK step, ragged 3001: max |da| / max |a|",
                  np.max(np.abs(acc[:, :3] - n1.acc)) / np.max(np.abs(n1.acc)), ACC_TOL)
    assert parity("KDK step, ragged 3001: max |d du/dt| / max |du/dt|",
                  np.max(np.abs(acc[:, 3] - n1.dudt)) / np.max(np.abs(n1.dudt)), ACC_TOL)
    # drho/dt of the step (written by its force pass) at the predicted velocities
    dr = s.in_original_order("drhodt")
    assert parity("KDK step, ragged 3001: max |d drho/dt| / max |drho/dt|",
                  np.max(np.abs(dr - n1.drhodt)) / np.max(np.abs(n1.drhodt)), ACC_TOL)
    # the step wrote the next Courant dt
    n1.vsigmax = n1.vsigmax
    assert abs(d_dt.item() / oracle.courant_dt(n1) - 1) <= 1e-3


def test_conserved_fp64(sph, parity):
    native, ctx, torch = sph
    w = CASES["c1_8192"]
    s = upload(native, w)
    out = torch.zeros(8, dtype=torch.float64, device="cuda")
    native.sph_conserved(ctx, s.c, out)
    ref = oracle.conserved(*f64(w))
    got = out.cpu().numpy()
    scale = np.array([ref[0], ref[1]] + [np.sum(np.abs(w.vel[:, :3]) * w.pos[:, 3:4])] * 3 +
                     [np.sum(np.abs(ref[5:]))] * 3)
    assert parity("conserved sums (FP64), C1 8192: max |d| / scale",
                  np.max(np.abs(got - ref) / np.maximum(scale, 1e-30)), 1e-12)


@pytest.mark.parametrize("pinned,steps", [(True, 1), (True, 3), (False, 2)])
def test_step_host_matches_device_step(sph, pinned, steps):
    # pinned buffers: the last step copies each output back while it runs
    # (its own graph); pageable buffers: plain copies after the steps
    import ctypes
    native, ctx, torch = sph
    w = CASES["ragged_3001"]
    s, p = evaluate_gpu(native, ctx, w)
    d_dt = torch.zeros(1, dtype=torch.float32, device="cuda")
    native.sph_timestep(ctx, s.c, p, d_dt)
    dt0 = d_dt.item()
    fields = s.FIELDS4 + s.FIELDS1 + ("perm", "keys")
    host = {k: getattr(s, k).cpu() for k in fields}
    if pinned:
        host = {k: t.pin_memory() for k, t in host.items()}
    hs = native.sph_state()
    hs.n = s.n
    for k, t in host.items():
        setattr(hs, k, t.data_ptr())
    for _ in range(steps):
        native.sph_step(ctx, s.c, p, d_dt)
    native.sph_sync(ctx)
    hdt = ctypes.c_float(dt0)
    native.sph_step_host(ctx, hs, p, steps, hdt)
    for k in fields:
        assert torch.equal(host[k][: s.n], getattr(s, k)[: s.n].cpu()), k
    assert hdt.value == d_dt.item()


def test_step_graph_slots_are_reused(sph):
    # more argument sets than the context keeps graphs for: the least recently
    # used graph is dropped and recorded again when its arguments come back
    native, ctx, torch = sph
    fields = ("pos", "vel", "acc", "h", "rho", "omega", "drhodt", "vsigmax", "perm", "keys")
    states = []
    for k in range(6):
        w = inputs.unit_sphere(700 + 50 * k, seed=40 + k)
        s, p = evaluate_gpu(native, ctx, w)
        d_dt = torch.zeros(1, dtype=torch.float32, device="cuda")
        native.sph_timestep(ctx, s.c, p, d_dt)
        native.sph_sync(ctx)
        states.append((w, s, p, d_dt, d_dt.clone()))
    for _ in range(2):
        for w, s, p, d_dt, _ in states:
            native.sph_step(ctx, s.c, p, d_dt)
    native.sph_sync(ctx)
    for w, s, p, d_dt, dt0 in states:
        s2, p2 = evaluate_gpu(native, ctx, w)
        dt2 = dt0.clone()
        for _ in range(2):
            native.sph_step(ctx, s2.c, p2, dt2)
        native.sph_sync(ctx)
        for k in fields:
            assert torch.equal(getattr(s, k), getattr(s2, k)), k
        assert d_dt.item() == dt2.item()


def test_step_graph_matches_eager(sph):
    """sph_step replays a recorded CUDA graph; inside a caller's own capture it
    enqueues the kernels directly.  Both give the same state bit for bit, and
    the stage timers of the graph (event nodes) see every stage."""
    native, ctx, torch = sph
    w = CASES["ragged_3001"]
    s, p = evaluate_gpu(native, ctx, w)
    d_dt = torch.zeros(1, dtype=torch.float32, device="cuda")
    d_t = torch.zeros(1, dtype=torch.float64, device="cuda")
    native.sph_timestep(ctx, s.c, p, d_dt)
    native.sph_sync(ctx)
    fields = s.FIELDS4 + s.FIELDS1 + ("perm", "keys")
    snap = {k: getattr(s, k).clone() for k in fields}
    dt0 = d_dt.clone()

    def restore():
        for k in fields:
            getattr(s, k).copy_(snap[k])
        d_dt.copy_(dt0)
        d_t.zero_()

    def result():
        native.sph_sync(ctx)
        return {k: getattr(s, k).clone() for k in fields}, d_dt.item(), d_t.item()

    steps = 3
    native.sph_get_timing(ctx)
    for _ in range(steps):                       # graph, no timing
        native.sph_step(ctx, s.c, p, d_dt, d_t)
    a = result()
    _, launches0 = native.sph_get_timing(ctx)
    restore()
    native.sph_set_timing(ctx, True)
    for _ in range(steps):                       # graph with event nodes
        native.sph_step(ctx, s.c, p, d_dt, d_t)
    b = result()
    ms, launches1 = native.sph_get_timing(ctx)
    native.sph_set_timing(ctx, False)
    restore()
    g = torch.cuda.CUDAGraph()                   # the caller's capture: direct launches
    cs = torch.cuda.Stream()
    cs.wait_stream(torch.cuda.current_stream())
    with torch.cuda.graph(g, stream=cs):
        native.sph_step(ctx, s.c, p, d_dt, d_t)
    torch.cuda.current_stream().wait_stream(cs)
    torch.cuda.synchronize()
    native.sph_get_timing(ctx)
    for _ in range(steps):
        g.replay()
    c = result()
    for other in (b, c):
        assert other[1] == a[1] and other[2] == a[2]
        for k in fields:
            assert torch.equal(other[0][k], a[0][k]), k
    assert launches1 == launches0 and sum(launches0.values()) > 0
    for stage in ("tree", "lists", "density", "force", "leapfrog", "reduce"):
        assert ms[stage] > 0, stage


def test_step_graphs_of_two_states_do_not_mix(sph):
    """Steps of two states interleaved on one context (one recorded graph
    each) give the states that each gets alone on its own context."""
    native, ctx, torch = sph
    fields = ("pos", "vel", "acc", "h", "rho", "omega", "drhodt", "vsigmax", "perm", "keys")

    def prepare(context, w):
        s, p = evaluate_gpu(native, context, w)
        d_dt = torch.zeros(1, dtype=torch.float32, device="cuda")
        native.sph_timestep(context, s.c, p, d_dt)
        return s, p, d_dt

    a = prepare(ctx, CASES["ragged_3001"])
    b = prepare(ctx, CASES["c1_8192"])
    for _ in range(2):
        for s, p, d_dt in (a, b):
            native.sph_step(ctx, s.c, p, d_dt)
    native.sph_sync(ctx)
    for (s, _, d_dt), name in ((a, "ragged_3001"), (b, "c1_8192")):
        own = native.sph_create(1 << 14, 0)
        try:
            s2, p2, dt2 = prepare(own, CASES[name])
            for _ in range(2):
                native.sph_step(own, s2.c, p2, dt2)
            native.sph_sync(own)
            for k in fields:
                assert torch.equal(getattr(s, k), getattr(s2, k)), (name, k)
            assert d_dt.item() == dt2.item()
        finally:
            native.sph_destroy(own)


# ------------------------------------------------------------------ edge cases
def test_empty_is_noop(sph):
    native, ctx, torch = sph
    from paper_1909_07439_gb300 import DeviceState
    s = DeviceState(0)
    p = native.sph_params_default()
    for fn in (native.sph_build_tree, native.sph_density, native.sph_force):
        fn(ctx, s.c, p)
    native.sph_sync(ctx)


def test_too_few_particles_has_no_root(sph):
    # with fewer than ~6 particles sum_j m W(r, h) never reaches m (hfact/h)^3:
    # the fixed point does not exist and the solve must say so
    native, ctx, torch = sph
    w = inputs.unit_sphere(3, seed=2)
    s = upload(native, w)
    p = native.sph_params_default(max_h_iter=20)
    native.sph_build_tree(ctx, s.c, p)
    native.sph_density(ctx, s.c, p)
    with pytest.raises(native.SphError) as e:
        native.sph_sync(ctx)
    assert e.value.status == 4


def test_nonfinite_input_is_rejected(sph):
    native, ctx, torch = sph
    w = inputs.unit_sphere(500, seed=3)
    w.pos[17, 1] = np.nan
    s = upload(native, w)
    p = native.sph_params_default()
    native.sph_build_tree(ctx, s.c, p)
    with pytest.raises(native.SphError) as e:
        native.sph_sync(ctx)
    assert e.value.status == 6


@pytest.mark.parametrize("what,status", [("u<0", 7), ("m=0", 6), ("h=0", 6), ("v=inf", 6),
                                         ("v=-inf", 6), ("u=nan", 6)])
def test_bad_input_is_reported(sph, what, status):
    # host-injected bad inputs: each condition is found on the device and
    # returned, with its own status, by the next sph_sync
    native, ctx, torch = sph
    w = inputs.unit_sphere(700, seed=12)
    k = 123
    if what == "u<0":
        w.vel[k, 3] = -0.01
    elif what == "m=0":
        w.pos[k, 3] = 0.0
    elif what == "h=0":
        w.h[k] = 0.0
    elif what == "v=inf":
        w.vel[k, 1] = np.inf
    elif what == "v=-inf":
        w.vel[k, 0] = -np.inf
    elif what == "u=nan":
        w.vel[k, 3] = np.nan
    s = upload(native, w)
    p = native.sph_params_default()
    with pytest.raises(native.SphError) as e:
        native.sph_build_tree(ctx, s.c, p)
        native.sph_sync(ctx)
        native.sph_density(ctx, s.c, p)
        native.sph_sync(ctx)
        native.sph_force(ctx, s.c, p)
        native.sph_sync(ctx)
    assert e.value.status == status, str(e.value)
    native.sph_sync(ctx)          # the error word was cleared


def test_lookback_wait_times_out(sph):
    # a sort pass whose look-back predecessor never publishes gives up after its
    # poll limit and reports SPH_ERR_TIMEOUT; the context stays usable
    native, ctx, torch = sph
    native.sph_sync(ctx)
    native.sph_test_lookback_timeout(ctx, 64)
    with pytest.raises(native.SphError) as e:
        native.sph_sync(ctx)
    assert e.value.status == 8
    native.sph_sync(ctx)
    w = CASES["ragged_3001"]
    s, p = evaluate_gpu(native, ctx, w)
    keys_o = oracle.morton_keys(w.pos)
    assert np.array_equal(s.numpy("perm").astype(np.int64), oracle.sort_order(keys_o))


def test_list_overflow_is_reported(sph):
    # h doubled: about 8x the neighbours, past the 128-entry lists; the list
    # sets cannot be returned (status 5) and the context stays usable
    native, ctx, torch = sph
    w = CASES["c1_8192"]
    d, _ = oracle_eval("c1_8192", w)
    h = (2.0 * d.h).astype(np.float32)
    s = upload(native, inputs.Workload("x", w.pos, w.vel, h))
    p = native.sph_params_default()
    native.sph_build_tree(ctx, s.c, p)
    off = torch.zeros(w.n + 1, dtype=torch.int64, device="cuda")
    with pytest.raises(native.SphError) as e:
        native.sph_neighbours(ctx, s.c, p, 2, off)
    assert e.value.status == 5
    native.sph_sync(ctx)
    assert native.sph_get_stats(ctx)["list_overflows"] > 0


def test_invalid_arguments(sph):
    native, ctx, torch = sph
    s = upload(native, inputs.unit_sphere(64))
    with pytest.raises(native.SphError):
        native.sph_build_tree(ctx, s.c, native.sph_params_default(n_group=0))
    big = s.c
    big.n = 1 << 20
    with pytest.raises(native.SphError):
        native.sph_build_tree(ctx, big, native.sph_params_default())


def test_coincident_particles(sph):
    native, ctx, torch = sph
    w = inputs.unit_sphere(2000, seed=9)
    w.pos[500:504, :3] = w.pos[500, :3]   # 4 particles at one point (r = 0 pairs)
    s, p = evaluate_gpu(native, ctx, w)
    x, v, m, u = f64(w)
    d = oracle.density(x, v, m, w.h)
    assert d.failures == 0
    f = oracle.force(x, v, m, u, d.h, d.rho, d.omega)
    assert np.max(np.abs(s.in_original_order("rho") / d.rho - 1)) <= RHO_TOL
    acc = s.in_original_order("acc")
    assert np.max(np.abs(acc[:, :3] - f.acc)) <= ACC_TOL * np.max(np.abs(f.acc))


def test_point_mass_cluster_has_no_root(sph):
    # k coincident particles give sum_j m W(0, h) = k m C / h^3 > m hfact^3 / h^3
    # once k C > hfact^3 (k >= 6 for the M4 kernel): g(h) > 0 for every h, so
    # the h-rho fixed point does not exist; the oracle and the GPU both report it
    native, ctx, torch = sph
    w = inputs.unit_sphere(2000, seed=9)
    w.pos[500:520, :3] = w.pos[500, :3]
    x, v, m, u = f64(w)
    assert oracle.density(x, v, m, w.h, targets=[500], max_iter=60).failures == 1
    s = upload(native, w)
    p = native.sph_params_default()
    native.sph_build_tree(ctx, s.c, p)
    native.sph_density(ctx, s.c, p)
    with pytest.raises(native.SphError) as e:
        native.sph_sync(ctx)
    assert e.value.status == 4
