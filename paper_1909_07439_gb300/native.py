"""Thin ctypes binding of libsph (include/sph.h).

Argument marshalling only: every step of the SPH path runs in the CUDA
library.  Functions keep the C names.  A missing library is an error
(``NativeLibraryMissing``), never a fallback.
"""
from __future__ import annotations

import ctypes
import os
from ctypes import POINTER, c_double, c_float, c_int, c_int32, c_int64, c_uint64, c_void_p

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "lib", "libsph.so")

SPH_OK = 0
STATUS = {0: "SPH_OK", 1: "SPH_ERR_INVALID_ARG", 2: "SPH_ERR_CUDA", 3: "SPH_ERR_NOMEM",
          4: "SPH_ERR_NOT_CONVERGED", 5: "SPH_ERR_TILE_OVERFLOW", 6: "SPH_ERR_NONFINITE",
          7: "SPH_ERR_NEGATIVE_U", 8: "SPH_ERR_TIMEOUT"}
STAGES = ("tree", "density", "force", "reduce", "leapfrog", "prep", "lists", "gravity")


class NativeLibraryMissing(RuntimeError):
    pass


class SphError(RuntimeError):
    def __init__(self, status, text):
        super().__init__(f"{STATUS.get(status, status)}: {text}")
        self.status = status


class sph_params(ctypes.Structure):
    _fields_ = [("gamma", c_float), ("hfact", c_float), ("alpha_av", c_float),
                ("beta_av", c_float), ("alpha_u", c_float), ("c_cour", c_float),
                ("h_tol", c_float), ("kernel", c_int32), ("n_leaf", c_int32),
                ("n_group", c_int32), ("tile", c_int32), ("max_h_iter", c_int32),
                ("density_iters", c_int32), ("pair_targets", c_int32), ("pair_warps", c_int32),
                ("pair_unroll", c_int32), ("box_lo", c_float * 3), ("box_len", c_float * 3),
                ("grav_G", c_float), ("grav_eps", c_float), ("grav_theta", c_float)]


class sph_state(ctypes.Structure):
    _fields_ = [("n", c_int64), ("pos", c_void_p), ("vel", c_void_p), ("acc", c_void_p),
                ("h", c_void_p), ("rho", c_void_p), ("omega", c_void_p), ("drhodt", c_void_p),
                ("vsigmax", c_void_p), ("perm", c_void_p), ("keys", c_void_p)]


class sph_stats(ctypes.Structure):
    _fields_ = [(k, c_uint64) for k in (
        "density_pairs", "density_candidates", "force_pairs", "force_candidates",
        "newton_iters", "density_rewalks", "streamed_groups", "n_nodes", "n_groups",
        "list_entries", "list_overflows", "force_rewalks", "gravity_cells", "gravity_particles")]

    def as_dict(self):
        return {k: int(getattr(self, k)) for k, _ in self._fields_}


_lib = None
EXPORTS = ("sph_params_default", "sph_create", "sph_destroy", "sph_build_tree", "sph_density",
           "sph_force", "sph_gravity", "sph_timestep", "sph_step", "sph_block_levels", "sph_step_block", "sph_step_host", "sph_batch_evaluate",
           "sph_batch_step", "sph_force_bwd", "sph_density_bwd", "sph_rollout", "sph_conserved",
           "sph_conserved_noalloc",
           "sph_neighbours", "sph_get_tree", "sph_get_stats", "sph_set_timing", "sph_get_timing", "sph_sync",
           "sph_last_error", "sph_test_lookback_timeout", "sph_fp32_probe")


def load():
    """Load libsph.so from the package (build it with ``build.build()``)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise NativeLibraryMissing(
            f"{LIB_PATH} is missing: build it with paper_1909_07439_gb300.build.build()")
    lib = ctypes.CDLL(LIB_PATH)
    P = c_void_p
    lib.sph_params_default.argtypes = [POINTER(sph_params)]
    lib.sph_params_default.restype = None
    lib.sph_create.argtypes = [POINTER(c_void_p), c_int64, c_int]
    lib.sph_destroy.argtypes = [P]
    lib.sph_destroy.restype = None
    for name in ("sph_build_tree", "sph_density", "sph_force"):
        getattr(lib, name).argtypes = [P, POINTER(sph_state), POINTER(sph_params), P]
    lib.sph_timestep.argtypes = [P, POINTER(sph_state), POINTER(sph_params), P, P]
    lib.sph_gravity.argtypes = [P, POINTER(sph_state), POINTER(sph_params), P, P]
    lib.sph_block_levels.argtypes = [P, POINTER(sph_state), POINTER(sph_params), c_int, P, P, P]
    lib.sph_step_block.argtypes = [P, POINTER(sph_state), POINTER(sph_params), c_int, P, P, P, P]
    lib.sph_step.argtypes = [P, POINTER(sph_state), POINTER(sph_params), P, P, P]
    lib.sph_step_host.argtypes = [P, POINTER(sph_state), POINTER(sph_params), c_int,
                                  POINTER(c_float), P]
    lib.sph_batch_evaluate.argtypes = [P, POINTER(sph_state), P, c_int, POINTER(sph_params), P, P]
    lib.sph_batch_step.argtypes = [P, POINTER(sph_state), P, c_int, c_int, POINTER(sph_params), P,
                                   P, P]
    lib.sph_force_bwd.argtypes = [P, POINTER(sph_state), POINTER(sph_params), P, P, P, P, P, P, P,
                                  P]
    lib.sph_density_bwd.argtypes = [P, POINTER(sph_state), POINTER(sph_params), P, P, P, P, P]
    lib.sph_rollout.argtypes = [P, POINTER(sph_state), POINTER(sph_params), c_int, c_int, P, c_int,
                                POINTER(c_double), P, POINTER(c_double), P]
    lib.sph_conserved.argtypes = [P, POINTER(sph_state), P, P]
    lib.sph_conserved_noalloc.argtypes = [c_int64, P, P, P, P]
    lib.sph_neighbours.argtypes = [P, POINTER(sph_state), POINTER(sph_params), c_int, P, P,
                                   c_int64, POINTER(c_int64), P]
    lib.sph_get_tree.argtypes = [P, P, P, P, P, P, c_int64, P, P, c_int64, POINTER(c_int64),
                                 POINTER(c_int64)]
    lib.sph_get_stats.argtypes = [P, POINTER(sph_stats)]
    lib.sph_test_lookback_timeout.argtypes = [P, c_int, P]
    lib.sph_fp32_probe.argtypes = [P, c_int, c_int, c_int, P]
    lib.sph_set_timing.argtypes = [P, c_int]
    lib.sph_get_timing.argtypes = [P, POINTER(c_double), POINTER(c_int64)]
    lib.sph_sync.argtypes = [P, P]
    lib.sph_last_error.argtypes = [P]
    lib.sph_last_error.restype = ctypes.c_char_p
    for name in EXPORTS:
        if name not in ("sph_params_default", "sph_destroy", "sph_last_error"):
            getattr(lib, name).restype = c_int
    _lib = lib
    return lib


def _check(ctx, status):
    if status != SPH_OK:
        text = load().sph_last_error(ctx)
        raise SphError(status, text.decode() if text else "")
    return status


def _stream(stream):
    if stream is None:
        try:
            import torch
            return c_void_p(torch.cuda.current_stream().cuda_stream)
        except Exception:
            return c_void_p(0)
    if isinstance(stream, int):
        return c_void_p(stream)
    return c_void_p(stream.cuda_stream)


def _ptr(t):
    return None if t is None else c_void_p(t.data_ptr())


# ---------------------------------------------------------------- C names
def sph_params_default(**overrides) -> sph_params:
    p = sph_params()
    load().sph_params_default(ctypes.byref(p))
    for k, v in overrides.items():
        if not hasattr(p, k):
            raise KeyError(k)
        if k in ("box_lo", "box_len"):
            v = (c_float * 3)(*[float(x) for x in v])
        setattr(p, k, v)
    return p


def sph_create(max_n: int, device: int = 0):
    h = c_void_p()
    st = load().sph_create(ctypes.byref(h), int(max_n), int(device))
    if st != SPH_OK:
        raise SphError(st, "sph_create failed")
    return h


def sph_destroy(ctx):
    load().sph_destroy(ctx)


def sph_build_tree(ctx, state, params, stream=None):
    return _check(ctx, load().sph_build_tree(ctx, ctypes.byref(state), ctypes.byref(params),
                                             _stream(stream)))


def sph_density(ctx, state, params, stream=None):
    return _check(ctx, load().sph_density(ctx, ctypes.byref(state), ctypes.byref(params),
                                          _stream(stream)))


def sph_force(ctx, state, params, stream=None):
    return _check(ctx, load().sph_force(ctx, ctypes.byref(state), ctypes.byref(params),
                                        _stream(stream)))


def sph_block_levels(ctx, state, params, max_level, d_dt_min, d_level, stream=None):
    """Courant dt_min (device float[1]) and per-particle levels (device int32[n], caller order)."""
    return _check(ctx, load().sph_block_levels(ctx, ctypes.byref(state), ctypes.byref(params),
                                               int(max_level), _ptr(d_dt_min), _ptr(d_level),
                                               _stream(stream)))


def sph_step_block(ctx, state, params, max_level, d_level, d_dt_min, d_time=None, stream=None):
    """One block of 2^max_level substeps of dt_min with individual levels."""
    return _check(ctx, load().sph_step_block(ctx, ctypes.byref(state), ctypes.byref(params),
                                             int(max_level), _ptr(d_level), _ptr(d_dt_min),
                                             _ptr(d_time), _stream(stream)))


def sph_gravity(ctx, state, params, d_out4, stream=None):
    """Self-gravity alone: d_out4 (n x 4 float32 on the device) = (a, phi), G included."""
    return _check(ctx, load().sph_gravity(ctx, ctypes.byref(state), ctypes.byref(params),
                                          _ptr(d_out4), _stream(stream)))


def sph_timestep(ctx, state, params, d_dt, stream=None):
    return _check(ctx, load().sph_timestep(ctx, ctypes.byref(state), ctypes.byref(params),
                                           _ptr(d_dt), _stream(stream)))


def sph_step(ctx, state, params, d_dt, d_time=None, stream=None):
    return _check(ctx, load().sph_step(ctx, ctypes.byref(state), ctypes.byref(params),
                                       _ptr(d_dt), _ptr(d_time), _stream(stream)))


def sph_step_host(ctx, host_state, params, n_steps, h_dt: c_float, stream=None):
    return _check(ctx, load().sph_step_host(ctx, ctypes.byref(host_state), ctypes.byref(params),
                                            int(n_steps), ctypes.byref(h_dt), _stream(stream)))


def sph_batch_evaluate(ctx, state, d_offsets, n_inst, params, d_dt, stream=None):
    return _check(ctx, load().sph_batch_evaluate(ctx, ctypes.byref(state), _ptr(d_offsets),
                                                 int(n_inst), ctypes.byref(params), _ptr(d_dt),
                                                 _stream(stream)))


def sph_batch_step(ctx, state, d_offsets, n_inst, n_steps, params, d_dt, d_time=None, stream=None):
    return _check(ctx, load().sph_batch_step(ctx, ctypes.byref(state), _ptr(d_offsets), int(n_inst),
                                             int(n_steps), ctypes.byref(params), _ptr(d_dt),
                                             _ptr(d_time), _stream(stream)))


def sph_force_bwd(ctx, state, params, gacc, gpos, gvel, gh, grho, gomega, galpha, stream=None):
    return _check(ctx, load().sph_force_bwd(ctx, ctypes.byref(state), ctypes.byref(params),
                                            _ptr(gacc), _ptr(gpos), _ptr(gvel), _ptr(gh),
                                            _ptr(grho), _ptr(gomega), _ptr(galpha),
                                            _stream(stream)))


def sph_density_bwd(ctx, state, params, gh, grho, gomega, gpos, stream=None):
    return _check(ctx, load().sph_density_bwd(ctx, ctypes.byref(state), ctypes.byref(params),
                                              _ptr(gh), _ptr(grho), _ptr(gomega), _ptr(gpos),
                                              _stream(stream)))


def sph_rollout(ctx, init_state, params, n_steps, ckpt, d_probes, n_probes, d_gvel=None,
                stream=None):
    """Returns (loss, dL/dalpha or None); fills d_gvel with dL/d(v0, u0) if given."""
    loss = c_double(0.0)
    ga = c_double(0.0)
    _check(ctx, load().sph_rollout(ctx, ctypes.byref(init_state), ctypes.byref(params),
                                   int(n_steps), int(ckpt), _ptr(d_probes), int(n_probes),
                                   ctypes.byref(loss), _ptr(d_gvel),
                                   ctypes.byref(ga) if d_gvel is not None else None,
                                   _stream(stream)))
    return loss.value, (ga.value if d_gvel is not None else None)


def sph_conserved(ctx, state, d_out8, stream=None):
    return _check(ctx, load().sph_conserved(ctx, ctypes.byref(state), _ptr(d_out8),
                                            _stream(stream)))


CONSERVED_NOALLOC_MAX_N = 16777216


def sph_conserved_noalloc(n, d_pos, d_vel, d_out8, stream=None):
    """Context-free conserved sums for callers that cannot allocate device
    memory (see include/sph.h); scratch is a fixed array inside the library."""
    st = load().sph_conserved_noalloc(int(n), _ptr(d_pos), _ptr(d_vel), _ptr(d_out8),
                                      _stream(stream))
    if st == 1:
        raise SphError(st, f"sph_conserved_noalloc rejected its arguments (n = {n}, limit "
                           f"{CONSERVED_NOALLOC_MAX_N}; pos/vel 16-byte and out 8-byte aligned)")
    if st != SPH_OK:
        raise SphError(st, "sph_conserved_noalloc: a CUDA launch or the scratch address lookup failed")
    return st


def sph_neighbours(ctx, state, params, mode, d_off, d_idx=None, cap=0, stream=None):
    total = c_int64(0)
    _check(ctx, load().sph_neighbours(ctx, ctypes.byref(state), ctypes.byref(params), int(mode),
                                      _ptr(d_off), _ptr(d_idx), int(cap), ctypes.byref(total),
                                      _stream(stream)))
    return int(total.value)


def sph_get_tree(ctx, node_cap=1 << 26, group_cap=1 << 26):
    """Nodes (level, first, count, nchild, child) and groups (first, count) as numpy."""
    import numpy as np
    nn, ng = c_int64(0), c_int64(0)
    lib = load()
    _check(ctx, lib.sph_get_tree(ctx, None, None, None, None, None, 0, None, None, 0,
                                 ctypes.byref(nn), ctypes.byref(ng)))
    arrs = [np.zeros(max(nn.value, 1), np.int32) for _ in range(5)]
    garrs = [np.zeros(max(ng.value, 1), np.int32) for _ in range(2)]
    pp = [a.ctypes.data_as(c_void_p) for a in arrs + garrs]
    _check(ctx, lib.sph_get_tree(ctx, *pp[:5], nn.value, *pp[5:], ng.value, ctypes.byref(nn),
                                 ctypes.byref(ng)))
    n, g = nn.value, ng.value
    return ({"level": arrs[0][:n], "first": arrs[1][:n], "count": arrs[2][:n],
             "nchild": arrs[3][:n], "child": arrs[4][:n]},
            {"first": garrs[0][:g], "count": garrs[1][:g]})


def sph_test_lookback_timeout(ctx, spin_cap, stream=None):
    return _check(ctx, load().sph_test_lookback_timeout(ctx, int(spin_cap), _stream(stream)))


def sph_fp32_probe(d_sink, blocks, iters, packed=False, stream=None):
    st = load().sph_fp32_probe(_ptr(d_sink), int(blocks), int(iters), 1 if packed else 0,
                               _stream(stream))
    if st != SPH_OK:
        raise SphError(st, "sph_fp32_probe failed")
    return st


def sph_get_stats(ctx) -> dict:
    s = sph_stats()
    _check(ctx, load().sph_get_stats(ctx, ctypes.byref(s)))
    return s.as_dict()


def sph_set_timing(ctx, enable: bool):
    return _check(ctx, load().sph_set_timing(ctx, 1 if enable else 0))


def sph_get_timing(ctx):
    ms = (c_double * len(STAGES))()
    n = (c_int64 * len(STAGES))()
    _check(ctx, load().sph_get_timing(ctx, ms, n))
    return {k: float(ms[i]) for i, k in enumerate(STAGES)}, {k: int(n[i]) for i, k in enumerate(STAGES)}


def sph_sync(ctx, stream=None):
    return _check(ctx, load().sph_sync(ctx, _stream(stream)))


def sph_last_error(ctx) -> str:
    t = load().sph_last_error(ctx)
    return t.decode() if t else ""
