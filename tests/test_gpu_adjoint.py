"""Adjoint kernels and the differentiable rollout vs FP64 torch autograd.

The reference (oracle/adjoint_ref.py) is pinned to the C oracle's forward and
to finite differences (tests/test_oracle_adjoint.py).  Bar: gradients within
1e-3 relative (in norm over particles) of the reference."""
import numpy as np
import pytest

import oracle
from paper_1909_07439_gb300 import inputs

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
from oracle import adjoint_ref as R  # noqa: E402

T = torch.float64
HFACT = {R.M4: 1.2, R.M6: 0.9, R.WC6: 1.3}
KERNELS = [R.M4, R.M6, R.WC6]
KNAME = {R.M4: "M4", R.M6: "M6", R.WC6: "Wendland C6"}
_rec = {}


@pytest.fixture(autouse=True)
def _bind_parity(parity, request):
    # the error recorder and the test's kernel, for _check
    cs = getattr(request.node, "callspec", None)
    _rec["parity"] = parity
    _rec["kernel"] = KNAME[cs.params.get("kernel", R.M4)] if cs else "M4"


@pytest.fixture(scope="module")
def lib():
    from paper_1909_07439_gb300 import build, native
    build.build()
    native.load()
    ctx = native.sph_create(1 << 16, 0)
    yield native, ctx
    native.sph_destroy(ctx)


def _cloud(n=1500, seed=3, kernel=R.M4):
    w = inputs.unit_sphere(n, seed=seed, sigma_v=0.3, hfact=HFACT[kernel])
    rng = np.random.default_rng(seed)
    w.vel[:, 3] *= rng.uniform(0.5, 2.0, n).astype(np.float32)
    return w


def _rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def _elem(a, b):
    """Largest element error relative to the largest reference element."""
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


def _check(name, got, ref, tol=1e-3, elem_tol=1e-3):
    e_norm, e_elem = _rel(got, ref), _elem(got, ref)
    print(f"{name}: rel L2 {e_norm:.2e}, max elem {e_elem:.2e}")
    par, k = _rec["parity"], _rec["kernel"]
    assert par(f"adjoint {name} ({k}): |d|_2 / |ref|_2", e_norm, tol), name
    assert par(f"adjoint {name} ({k}): max |d| / max |ref|", e_elem, elem_tol), name


@pytest.mark.parametrize("kernel", KERNELS)
def test_force_bwd_matches_autograd(lib, kernel):
    native, ctx = lib
    from paper_1909_07439_gb300 import DeviceState
    w = _cloud(kernel=kernel)
    x, v, m, u = (w.pos[:, :3].astype(np.float64), w.vel[:, :3].astype(np.float64),
                  w.pos[:, 3].astype(np.float64), w.vel[:, 3].astype(np.float64))
    d = oracle.density(x, v, m, w.h, hfact=HFACT[kernel], kernel=kernel)
    # both sides use the oracle's h, rho, Omega (rounded to float32) as inputs
    h32, r32, o32 = (d.h.astype(np.float32), d.rho.astype(np.float32), d.omega.astype(np.float32))
    s = DeviceState.from_arrays(w.pos, w.vel, h32)
    p = native.sph_params_default(kernel=kernel, hfact=HFACT[kernel])
    native.sph_build_tree(ctx, s.c, p)
    perm = s.numpy("perm").astype(np.int64)
    s.rho[: s.n] = torch.as_tensor(r32[perm], device="cuda")
    s.omega[: s.n] = torch.as_tensor(o32[perm], device="cuda")
    native.sph_force(ctx, s.c, p)
    wgt = np.random.default_rng(1).normal(size=(w.n, 4)).astype(np.float32)
    gacc = torch.as_tensor(wgt[perm], device="cuda")
    z4 = lambda: torch.zeros((w.n, 4), dtype=torch.float32, device="cuda")
    z1 = lambda: torch.zeros(w.n, dtype=torch.float32, device="cuda")
    gpos, gvel, gh, grho, gom = z4(), z4(), z1(), z1(), z1()
    gal = torch.zeros(1, dtype=torch.float64, device="cuda")
    native.sph_force_bwd(ctx, s.c, p, gacc, gpos, gvel, gh, grho, gom, gal)
    native.sph_sync(ctx)

    def orig(t):
        a = t.cpu().numpy()
        out = np.empty_like(a)
        out[perm] = a
        return out

    tx = torch.tensor(w.pos[:, :3], dtype=T, requires_grad=True)
    tv = torch.tensor(w.vel[:, :3], dtype=T, requires_grad=True)
    tu = torch.tensor(w.vel[:, 3], dtype=T, requires_grad=True)
    th = torch.tensor(h32, dtype=T, requires_grad=True)
    tr = torch.tensor(r32, dtype=T, requires_grad=True)
    to = torch.tensor(o32, dtype=T, requires_grad=True)
    ta = torch.tensor(1.0, dtype=T, requires_grad=True)
    tm = torch.tensor(w.pos[:, 3], dtype=T)
    i, j = R.pair_list(tx.detach(), th.detach(), 1.0001, kernel=kernel)
    acc, du = R.force(tx, tv, tu, tm, th, tr, to, i, j, alpha=ta, kernel=kernel)
    L = (torch.tensor(wgt[:, :3], dtype=T) * acc).sum() + (torch.tensor(wgt[:, 3], dtype=T) * du).sum()
    L.backward()
    _check("dL/dx", orig(gpos)[:, :3], tx.grad.numpy())
    _check("dL/dv", orig(gvel)[:, :3], tv.grad.numpy())
    _check("dL/du", orig(gvel)[:, 3], tu.grad.numpy())
    _check("dL/dh", orig(gh), th.grad.numpy())
    _check("dL/drho", orig(grho), tr.grad.numpy())
    _check("dL/dOmega", orig(gom), to.grad.numpy())
    assert _rec["parity"](f"adjoint force dL/dalpha ({_rec['kernel']}): relative",
                          abs(gal.item() - float(ta.grad)) / abs(float(ta.grad)), 1e-3)


@pytest.mark.parametrize("kernel", KERNELS)
def test_density_bwd_matches_autograd(lib, kernel):
    native, ctx = lib
    from paper_1909_07439_gb300 import DeviceState
    w = _cloud(1200, seed=8, kernel=kernel)
    s = DeviceState.from_arrays(w.pos, w.vel, w.h)
    p = native.sph_params_default(kernel=kernel, hfact=HFACT[kernel])
    native.sph_build_tree(ctx, s.c, p)
    native.sph_density(ctx, s.c, p)
    perm = s.numpy("perm").astype(np.int64)
    rng = np.random.default_rng(4)
    cg = rng.normal(size=(3, w.n)).astype(np.float32)
    gh = torch.as_tensor(cg[0][perm], device="cuda")
    gr = torch.as_tensor(cg[1][perm], device="cuda")
    go = torch.as_tensor(cg[2][perm], device="cuda")
    gpos = torch.zeros((w.n, 4), dtype=torch.float32, device="cuda")
    native.sph_density_bwd(ctx, s.c, p, gh, gr, go, gpos)
    native.sph_sync(ctx)
    got = np.empty((w.n, 4), np.float32)
    got[perm] = gpos.cpu().numpy()
    tx = torch.tensor(w.pos[:, :3], dtype=T, requires_grad=True)
    tm = torch.tensor(w.pos[:, 3], dtype=T)
    h0 = torch.tensor(w.h, dtype=T)
    i, j = R.pair_list(tx.detach(), h0, 2.6, kernel=kernel)
    h, rho, om = R.density(tx, tm, h0, i, j, hfact=HFACT[kernel], iters=40, kernel=kernel)
    L = (torch.tensor(cg[0], dtype=T) * h + torch.tensor(cg[1], dtype=T) * rho +
         torch.tensor(cg[2], dtype=T) * om).sum()
    L.backward()
    _check("density dL/dx", got[:, :3], tx.grad.numpy())


def _sedov16(kernel=R.M4):
    w = inputs.sedov_lattice(16, seed=6, hfact=HFACT[kernel])
    return w, inputs.probe_indices(w.n, 256, seed=7)


@pytest.mark.parametrize("kernel", [R.M4, R.M6])
def test_rollout_gradient_matches_fp64_reference(lib, kernel):
    native, ctx = lib
    from paper_1909_07439_gb300 import DeviceState
    w, probes = _sedov16(kernel)
    s = DeviceState.from_arrays(w.pos, w.vel, w.h)
    p = native.sph_params_default(kernel=kernel, hfact=HFACT[kernel])
    d_probes = torch.as_tensor(probes, device="cuda")
    gvel = torch.zeros((w.n, 4), dtype=torch.float32, device="cuda")
    loss, galpha = native.sph_rollout(ctx, s.c, p, 20, 5, d_probes, len(probes), gvel)
    g = gvel.cpu().numpy()
    x = torch.tensor(w.pos[:, :3], dtype=T)
    v = torch.tensor(w.vel[:, :3], dtype=T, requires_grad=True)
    u = torch.tensor(w.vel[:, 3], dtype=T, requires_grad=True)
    m = torch.tensor(w.pos[:, 3], dtype=T)
    al = torch.tensor(1.0, dtype=T, requires_grad=True)
    Lr, dts, _ = R.rollout(x, v, u, m, torch.tensor(w.h, dtype=T), al, 20, torch.tensor(probes),
                           hfact=HFACT[kernel], kernel=kernel)
    Lr.backward()
    par, k = _rec["parity"], _rec["kernel"]
    assert par(f"adjoint rollout loss ({k}): |L/L_ref - 1|", abs(loss / float(Lr) - 1), 1e-4)
    _check("rollout dL/dv0", g[:, :3], v.grad.numpy())
    _check("rollout dL/du0", g[:, 3], u.grad.numpy())
    assert par(f"adjoint rollout dL/dalpha ({k}): relative", abs(galpha / float(al.grad) - 1), 1e-3)


def test_autograd_function_and_no_grad_path(lib):
    native, ctx = lib
    from paper_1909_07439_gb300 import DeviceState
    from paper_1909_07439_gb300.adjoint import rollout_loss
    w, probes = _sedov16()
    s = DeviceState.from_arrays(w.pos, w.vel, w.h)
    p = native.sph_params_default()
    d_probes = torch.as_tensor(probes, device="cuda")
    velu = s.vel[: s.n].clone().requires_grad_(True)
    al = torch.tensor(1.0, dtype=torch.float64, requires_grad=True)
    L = rollout_loss(ctx, s.pos[: s.n], velu, s.h[: s.n], al, p, 6, 3, d_probes)
    L.backward()
    g = torch.zeros((w.n, 4), dtype=torch.float32, device="cuda")
    loss2, ga2 = native.sph_rollout(ctx, s.c, p, 6, 3, d_probes, len(probes), g)
    assert float(L) == loss2
    assert torch.equal(velu.grad, g)
    # dL/dalpha is an FP64 sum accumulated with atomics: equal up to summation order
    assert abs(float(al.grad) - ga2) <= 1e-12 * abs(ga2)
    loss3, _ = native.sph_rollout(ctx, s.c, p, 6, 3, d_probes, len(probes))   # loss only
    assert loss3 == loss2


def test_rollout_buffers_reused_across_lengths(lib):
    # a longer rollout after a shorter one on the same context (same checkpoint
    # interval) must give what a fresh context gives: the work buffers are
    # replaced when they are too small for the new number of steps
    native, ctx = lib
    from paper_1909_07439_gb300 import DeviceState
    w, probes = _sedov16()
    s = DeviceState.from_arrays(w.pos, w.vel, w.h)
    p = native.sph_params_default()
    d_probes = torch.as_tensor(probes, device="cuda")
    g_short = torch.zeros((w.n, 4), dtype=torch.float32, device="cuda")
    native.sph_rollout(ctx, s.c, p, 6, 5, d_probes, len(probes), g_short)
    g = torch.zeros((w.n, 4), dtype=torch.float32, device="cuda")
    loss, ga = native.sph_rollout(ctx, s.c, p, 10, 5, d_probes, len(probes), g)
    fresh = native.sph_create(1 << 16, 0)
    try:
        g2 = torch.zeros((w.n, 4), dtype=torch.float32, device="cuda")
        loss2, ga2 = native.sph_rollout(fresh, s.c, p, 10, 5, d_probes, len(probes), g2)
    finally:
        native.sph_destroy(fresh)
    assert loss == loss2
    assert torch.equal(g, g2)
    assert abs(ga - ga2) <= 1e-12 * abs(ga2)


def test_single_evaluation_user_loss_matches_fp64_autograd(lib):
    # a loss of the caller's own making over every differentiable output of one
    # evaluation (h, rho, Omega, a, du/dt); gradients w.r.t. positions,
    # velocities, internal energies and alpha_AV against FP64 torch autograd
    native, ctx = lib
    from paper_1909_07439_gb300.adjoint import evaluate
    w = _cloud(1500, seed=11)
    x, v, m, u = (w.pos[:, :3].astype(np.float64), w.vel[:, :3].astype(np.float64),
                  w.pos[:, 3].astype(np.float64), w.vel[:, 3].astype(np.float64))
    d = oracle.density(x, v, m, w.h)
    h0 = d.h.astype(np.float32) * np.float32(1.01)        # a starting guess near the root
    rng = np.random.default_rng(12)
    c = {k: rng.normal(size=sh) for k, sh in (("rho", w.n), ("h", w.n), ("om", w.n),
                                             ("a", (w.n, 3)), ("du", w.n))}

    def loss(h, rho, om, a, du, lib_):
        t = lambda k: lib_.tensor(c[k], dtype=h.dtype, device=h.device)
        return ((t("rho") * rho * rho).sum() + (t("h") * h).sum() * 10.0 + (t("om") * om).sum() +
                (t("a") * a).sum() * 1e-3 + (t("du") * du).sum() * 1e-3)

    pos = torch.tensor(w.pos, device="cuda", requires_grad=True)
    velu = torch.tensor(w.vel, device="cuda", requires_grad=True)
    al = torch.tensor(1.0, dtype=torch.float64, requires_grad=True)
    p = native.sph_params_default()
    hg, rg, og, acc = evaluate(ctx, pos, velu, torch.tensor(h0, device="cuda"), al, p)
    L = loss(hg.double(), rg.double(), og.double(), acc[:, :3].double(), acc[:, 3].double(), torch)
    L.backward()
    tx = torch.tensor(x, dtype=T, requires_grad=True)
    tv = torch.tensor(v, dtype=T, requires_grad=True)
    tu = torch.tensor(u, dtype=T, requires_grad=True)
    ta = torch.tensor(1.0, dtype=T, requires_grad=True)
    tm = torch.tensor(m, dtype=T)
    i, j = R.pair_list(tx.detach(), torch.tensor(d.h, dtype=T), 1.05)
    hh, rr, oo = R.density(tx, tm, torch.tensor(h0, dtype=T), i, j, iters=40)
    ar, dr = R.force(tx, tv, tu, tm, hh, rr, oo, i, j, alpha=ta)
    Lr = loss(hh, rr, oo, ar, dr, torch)
    Lr.backward()
    assert abs(float(L) / float(Lr) - 1) < 1e-4
    _check("evaluate dL/dx", pos.grad[:, :3].cpu().numpy(), tx.grad.numpy())
    _check("evaluate dL/dv", velu.grad[:, :3].cpu().numpy(), tv.grad.numpy())
    _check("evaluate dL/du", velu.grad[:, 3].cpu().numpy(), tu.grad.numpy())
    assert abs(float(al.grad) / float(ta.grad) - 1) < 1e-3
    assert torch.all(pos.grad[:, 3] == 0)
