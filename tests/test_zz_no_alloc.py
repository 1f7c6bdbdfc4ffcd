"""sph_conserved_noalloc: the context-free conserved-quantities entry point.

It exists for callers that cannot call cudaMalloc (a host framework that owns
all device memory, or code that must not risk the synchronisation an
allocation can cause), so it keeps its scratch in a fixed array inside the
library.  Here it must agree with sph_conserved (which uses context scratch)
to FP64 rounding, on two calls in a row with different particle counts, so
that a call never sees partial sums left by the previous one.
"""
import numpy as np
import pytest

from paper_1909_07439_gb300 import inputs

pytestmark = pytest.mark.gpu


def test_conserved_noalloc_matches_context_entry_point():
    import torch
    from paper_1909_07439_gb300 import DeviceState, build, native
    build.build()
    native.load()
    a = inputs.unit_sphere(8192, seed=1)
    b = inputs.sedov_lattice(24, seed=3)               # 13,824 particles: a different block count
    b.vel[:, :3] = np.random.default_rng(2).normal(0, 0.2, (b.n, 3)).astype(np.float32)
    ctx = native.sph_create(max(a.n, b.n), 0)
    try:
        for w in (a, b):                               # two calls in a row
            s = DeviceState.from_arrays(w.pos, w.vel, w.h)
            ref = torch.zeros(8, dtype=torch.float64, device="cuda")
            got = torch.full((8,), float("nan"), dtype=torch.float64, device="cuda")
            native.sph_conserved(ctx, s.c, ref)
            native.sph_conserved_noalloc(s.n, s.pos, s.vel, got)
            torch.cuda.synchronize()
            ref, got = ref.cpu().numpy(), got.cpu().numpy()
            m = w.pos[:, 3].astype(np.float64)
            v = w.vel[:, :3].astype(np.float64)
            x = w.pos[:, :3].astype(np.float64)
            scale = np.array([ref[0], ref[1]] + [np.sum(m[:, None] * np.abs(v))] * 3 +
                             [np.sum(m * np.linalg.norm(x, axis=1) * np.linalg.norm(v, axis=1))] * 3)
            assert np.all(np.abs(got - ref) <= 1e-12 * np.maximum(scale, 1e-300)), (got, ref)
    finally:
        native.sph_destroy(ctx)


def test_conserved_noalloc_rejects_oversize():
    import torch
    from paper_1909_07439_gb300 import build, native
    build.build()
    out = torch.zeros(8, dtype=torch.float64, device="cuda")
    dummy = torch.zeros((4, 4), dtype=torch.float32, device="cuda")
    with pytest.raises(native.SphError) as e:
        native.sph_conserved_noalloc(native.CONSERVED_NOALLOC_MAX_N + 1, dummy, dummy, out)
    assert e.value.status == 1


def test_conserved_noalloc_rejects_misaligned_output():
    # d_out8 receives doubles: an address that is not 8-byte aligned is rejected
    # on the host, before anything is launched
    import torch
    from paper_1909_07439_gb300 import build, native
    build.build()
    buf = torch.zeros(20, dtype=torch.float32, device="cuda")
    dummy = torch.zeros((4, 4), dtype=torch.float32, device="cuda")
    with pytest.raises(native.SphError) as e:
        native.sph_conserved_noalloc(4, dummy, dummy, buf[1:])     # base + 4 bytes
    assert e.value.status == 1
