"""torch.autograd.Function over the differentiable rollout of libsph.

``rollout_loss(ctx, pos, velu, h, alpha, ...)`` returns the scalar loss
(mean squared density of probe particles after n_steps leapfrog steps) as a
torch tensor whose backward gives dL/d(velocities, internal energies) and
dL/dalpha_AV from the library's adjoint kernels (sph_rollout).  Marshalling
only: the forward and backward sweeps run in libsph.
"""
from __future__ import annotations

import torch

from . import native


class _Rollout(torch.autograd.Function):
    @staticmethod
    def forward(fctx, velu, alpha, pos, h, handle, params, n_steps, ckpt, probes):
        p = native.sph_params_default(**{k: getattr(params, k) for k, _ in params._fields_})
        p.alpha_av = float(alpha)
        st = native.sph_state()
        st.n = pos.shape[0]
        st.pos, st.vel, st.h = pos.data_ptr(), velu.data_ptr(), h.data_ptr()
        need = velu.requires_grad or alpha.requires_grad
        g = torch.zeros_like(velu, memory_format=torch.contiguous_format) if need else None
        loss, ga = native.sph_rollout(handle, st, p, n_steps, ckpt, probes, probes.numel(), g)
        if need:
            fctx.save_for_backward(g)
            fctx.ga = ga
        return torch.tensor(loss, dtype=torch.float64, device=velu.device)

    @staticmethod
    def backward(fctx, gl):
        (g,) = fctx.saved_tensors
        s = gl.to(torch.float32)
        return (g * s, gl * fctx.ga, None, None, None, None, None, None, None)


def rollout_loss(handle, pos, velu, h, alpha, params, n_steps, ckpt, probes):
    """pos [n,4] (x,y,z,m), velu [n,4] (vx,vy,vz,u), h [n]: CUDA float32 tensors;
    alpha: 0-dim float64 tensor (alpha_AV); probes: CUDA int64 tensor.
    The library reads raw pointers, so every array must be a contiguous
    float32 CUDA tensor (velu is not copied: a copy would cut it off from
    autograd); anything else is rejected."""
    for name, t in (("pos", pos), ("velu", velu), ("h", h)):
        if t.dtype != torch.float32 or not t.is_cuda:
            raise TypeError(f"{name} must be a float32 CUDA tensor")
    if not velu.is_contiguous():
        raise ValueError("velu must be contiguous (pass velu.contiguous() as the leaf)")
    if pos.shape != velu.shape or pos.shape[-1] != 4 or h.shape != pos.shape[:1]:
        raise ValueError("pos and velu must be [n, 4] and h [n]")
    if probes.dtype != torch.int64 or not probes.is_cuda or not probes.is_contiguous():
        raise TypeError("probes must be a contiguous int64 CUDA tensor")
    return _Rollout.apply(velu, alpha, pos.contiguous(), h.contiguous(), handle, params,
                          n_steps, ckpt, probes)
