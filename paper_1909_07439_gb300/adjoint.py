"""torch.autograd.Functions over libsph's differentiable forms.

``evaluate(ctx, pos, velu, h0, alpha, params)``: one evaluation (tree build,
density solve, force pass) returning h, rho, Omega and acc = (a, du/dt) in
the caller's particle order; its backward takes arbitrary cotangents of those
outputs and returns dL/dx, dL/d(v, u) and dL/dalpha_AV from the library's
adjoint kernels (sph_force_bwd, then sph_density_bwd through the h-rho
fixed point by the implicit-function theorem).  The backward recomputes the
evaluation (same inputs, deterministic kernels: the same tree and neighbour
sets), so the context may be used for other work in between.

``rollout_loss(ctx, pos, velu, h, alpha, ...)`` returns the scalar loss
(mean squared density of probe particles after n_steps leapfrog steps) as a
torch tensor whose backward gives dL/d(velocities, internal energies) and
dL/dalpha_AV from the library's adjoint rollout (sph_rollout).

Marshalling only: the forward and backward sweeps run in libsph.
"""
from __future__ import annotations

import torch

from . import native
from .state import DeviceState


def _params(params, alpha):
    p = native.sph_params_default(**{k: getattr(params, k) for k, _ in params._fields_})
    p.alpha_av = float(alpha)
    return p


def _check_cuda_f32(**arrays):
    for name, t in arrays.items():
        if t.dtype != torch.float32 or not t.is_cuda:
            raise TypeError(f"{name} must be a float32 CUDA tensor")


def _run_forward(handle, pos, velu, h0, p):
    """Tree build, density and force of a fresh state; returns the state."""
    s = DeviceState(pos.shape[0], device=pos.device)
    s.pos[: s.n].copy_(pos.detach())
    s.vel[: s.n].copy_(velu.detach())
    s.h[: s.n].copy_(h0.detach())
    native.sph_build_tree(handle, s.c, p)
    native.sph_density(handle, s.c, p)
    native.sph_force(handle, s.c, p)
    return s


class _Evaluate(torch.autograd.Function):
    @staticmethod
    def forward(fctx, pos, velu, h0, alpha, handle, params):
        p = _params(params, alpha)
        s = _run_forward(handle, pos, velu, h0, p)
        native.sph_sync(handle)
        perm = s.perm[: s.n].long()
        n = s.n
        out = []
        for f in ("h", "rho", "omega", "acc"):
            a = getattr(s, f)[:n]
            o = torch.empty_like(a)
            o[perm] = a                     # curve order -> caller order
            out.append(o)
        fctx.save_for_backward(pos, velu, h0, alpha)
        fctx.handle, fctx.params = handle, params
        return tuple(out)

    @staticmethod
    def backward(fctx, gh, grho, gom, gacc):
        pos, velu, h0, alpha = fctx.saved_tensors
        handle = fctx.handle
        p = _params(fctx.params, alpha)
        s = _run_forward(handle, pos, velu, h0, p)   # the same tree and neighbour sets
        n, dev = s.n, pos.device
        perm = s.perm[:n].long()

        def to_curve(g, shape):
            return (torch.zeros(shape, dtype=torch.float32, device=dev) if g is None
                    else g.to(torch.float32)[perm].contiguous())

        gacc_c = to_curve(gacc, (n, 4))
        z4 = lambda: torch.zeros((n, 4), dtype=torch.float32, device=dev)
        z1 = lambda: torch.zeros(n, dtype=torch.float32, device=dev)
        gpos_c, gvel_c, gh_f, grho_f, gom_f = z4(), z4(), z1(), z1(), z1()
        galpha = torch.zeros(1, dtype=torch.float64, device=dev)
        native.sph_force_bwd(handle, s.c, p, gacc_c, gpos_c, gvel_c, gh_f, grho_f, gom_f, galpha)
        gh_t = (gh_f + to_curve(gh, (n,))).contiguous()
        grho_t = (grho_f + to_curve(grho, (n,))).contiguous()
        gom_t = (gom_f + to_curve(gom, (n,))).contiguous()
        native.sph_density_bwd(handle, s.c, p, gh_t, grho_t, gom_t, gpos_c)
        native.sph_sync(handle)
        gpos = torch.empty_like(gpos_c)
        gvel = torch.empty_like(gvel_c)
        gpos[perm] = gpos_c
        gvel[perm] = gvel_c
        gpos[:, 3] = 0.0                    # masses are constants of the problem
        return gpos, gvel, None, galpha.reshape(()).to(device=alpha.device, dtype=alpha.dtype), None, None


def evaluate(handle, pos, velu, h0, alpha, params):
    """One differentiable SPH evaluation (Eqs. 1-4 and 9-15).

    pos [n,4] (x, y, z, m), velu [n,4] (vx, vy, vz, u), h0 [n] (starting
    guess of the h-rho solve, not differentiated): float32 CUDA tensors;
    alpha: 0-dim tensor (alpha_AV); params: sph_params (alpha_av replaced by
    alpha); handle: a context with max_n >= n.  Returns (h, rho, Omega,
    acc) in the caller's order, acc [n,4] = (a xyz, du/dt); gradients flow to
    the positions, velocities, internal energies and alpha (masses get zero)."""
    _check_cuda_f32(pos=pos, velu=velu, h0=h0)
    if pos.shape != velu.shape or pos.shape[-1] != 4 or h0.shape != pos.shape[:1]:
        raise ValueError("pos and velu must be [n, 4] and h0 [n]")
    return _Evaluate.apply(pos, velu, h0, alpha, handle, params)


class _Rollout(torch.autograd.Function):
    @staticmethod
    def forward(fctx, velu, alpha, pos, h, handle, params, n_steps, ckpt, probes):
        p = _params(params, alpha)
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
