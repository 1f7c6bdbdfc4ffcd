"""Pins for the FP64 torch rollout reference used to check the CUDA adjoint:
its forward equals the C oracle (Eqs. 1-15), and its autograd gradient of
the rollout loss equals central finite differences of the same FP64 forward
(dt sequence held fixed)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
from oracle import adjoint_ref as R
from paper_1909_07439_gb300 import inputs

T = torch.float64
HFACT = {R.M4: 1.2, R.M6: 0.9, R.WC6: 1.3}
KERNELS = [R.M4, R.M6, R.WC6]


def test_kernel_constants_match_the_oracle():
    # the two restatements of Sect. 2.3 agree: W, F = dW/dr over the support
    for k in KERNELS:
        assert R.SUPPORT[k] == oracle.SUPPORT[k]
        r = np.linspace(0.0, 1.05 * R.SUPPORT[k], 400)
        h = np.ones_like(r)
        W, F, _ = oracle.kernel_eval(r, h, k)
        f, df = R.kern(torch.tensor(r, dtype=T), k)
        assert np.allclose(R.C_NORM[k] * f.numpy(), W, rtol=1e-13, atol=1e-15)
        assert np.allclose(R.C_NORM[k] * df.numpy(), F, rtol=1e-13, atol=1e-15)
        assert float(f[0]) == R.F0[k]


def _case(side=8, seed=2, sigma=0.3, kernel=R.M4):
    w = inputs.sedov_lattice(side, seed=seed, hfact=HFACT[kernel])
    v = w.vel[:, :3].astype(np.float64) + np.random.default_rng(seed).normal(0, sigma, (w.n, 3))
    x = torch.tensor(w.pos[:, :3], dtype=T)
    m = torch.tensor(w.pos[:, 3], dtype=T)
    u = torch.tensor(w.vel[:, 3], dtype=T)
    h0 = torch.tensor(w.h, dtype=T)
    return w, x, torch.tensor(v), u, m, h0


@pytest.mark.parametrize("kernel", KERNELS)
def test_forward_equals_c_oracle(kernel):
    w, x, v, u, m, h0 = _case(kernel=kernel)
    hf = HFACT[kernel]
    i, j = R.pair_list(x, h0, 2.5, kernel=kernel)
    h, rho, om = R.density(x, m, h0, i, j, hfact=hf, iters=30, kernel=kernel)
    d = oracle.density(x.numpy(), v.numpy(), m.numpy(), h0.numpy(), hfact=hf, kernel=kernel)
    assert np.max(np.abs(h.numpy() / d.h - 1)) < 1e-12
    assert np.max(np.abs(om.numpy() - d.omega)) < 1e-12
    a, du = R.force(x, v, u, m, h, rho, om, i, j, kernel=kernel)
    f = oracle.force(x.numpy(), v.numpy(), m.numpy(), u.numpy(), d.h, d.rho, d.omega, kernel=kernel)
    assert np.max(np.abs(a.numpy() - f.acc)) < 1e-12 * np.max(np.abs(f.acc))
    assert np.max(np.abs(du.numpy() - f.dudt)) < 1e-12 * np.max(np.abs(f.dudt))


@pytest.mark.parametrize("kernel", KERNELS)
def test_autograd_equals_finite_differences(kernel):
    w, x, v, u, m, h0 = _case(kernel=kernel)
    kw = dict(hfact=HFACT[kernel], kernel=kernel)
    probes = torch.tensor(inputs.probe_indices(w.n, 64))
    vv = v.clone().requires_grad_(True)
    uu = u.clone().requires_grad_(True)
    al = torch.tensor(1.0, dtype=T, requires_grad=True)
    L, dts, _ = R.rollout(x, vv, uu, m, h0, al, 4, probes, **kw)
    L.backward()
    gv, gu, ga = vv.grad.numpy(), uu.grad.numpy(), float(al.grad)

    def loss(v_, u_, a_):
        with torch.no_grad():
            return float(R.rollout(x, v_, u_, m, h0, torch.tensor(a_, dtype=T), 4, probes, dts=dts,
                                   **kw)[0])

    rng = np.random.default_rng(0)
    checks = []
    for k in [int(np.argmax(np.abs(gv).max(1)))] + list(rng.choice(w.n, 3, replace=False)):
        c = int(np.argmax(np.abs(gv[k])))
        e = 1e-5
        vp, vm = v.clone(), v.clone()
        vp[k, c] += e
        vm[k, c] -= e
        checks.append((gv[k, c], (loss(vp, u, 1.0) - loss(vm, u, 1.0)) / (2 * e)))
    k = int(np.argmax(np.abs(gu * u.numpy())))
    e = 1e-5 * float(u[k])
    up, um = u.clone(), u.clone()
    up[k] += e
    um[k] -= e
    checks.append((gu[k], (loss(v, up, 1.0) - loss(v, um, 1.0)) / (2 * e)))
    checks.append((ga, (loss(v, u, 1.0 + 1e-5) - loss(v, u, 1.0 - 1e-5)) / 2e-5))
    scale = max(abs(fd) for _, fd in checks)
    for g, fd in checks:
        assert abs(g - fd) <= 1e-5 * scale + 1e-6 * abs(fd), (g, fd)


def test_rollout_equals_c_oracle_steps():
    # the torch rollout (with its Courant steps) reproduces the C oracle's KDK steps
    w = inputs.sedov_lattice(8, seed=6)
    x, v, u, m = (torch.tensor(w.pos[:, :3], dtype=T), torch.tensor(w.vel[:, :3], dtype=T),
                  torch.tensor(w.vel[:, 3], dtype=T), torch.tensor(w.pos[:, 3], dtype=T))
    with torch.no_grad():
        L, dts, _ = R.rollout(x, v, u, m, torch.tensor(w.h, dtype=T), torch.tensor(1.0, dtype=T),
                              3, torch.arange(w.n))
    s = oracle.evaluate(oracle.SphState(x=x.numpy().copy(), v=v.numpy().copy(), u=u.numpy().copy(),
                                        m=m.numpy(), h=w.h.astype(np.float64)))
    for k in range(3):
        dt = oracle.courant_dt(s)
        assert abs(dts[k] / dt - 1) < 1e-12
        s = oracle.kdk_step(s, dt)
    assert abs(float(L) / float(np.mean(s.rho ** 2)) - 1) < 1e-12
