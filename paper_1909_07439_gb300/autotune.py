"""Autotuners for the group size (N_group) and the leaf size (N_leaf): time a
few steps of the actual state (graph-replayed for a batch) per candidate,
restoring the state between trials.  Results are cached in a JSON file keyed
by device, particle count and instance count (or workload tag)."""
from __future__ import annotations

import json
import os

from . import native

CANDIDATES = [(g, l) for g in (4, 8, 16) for l in (8, 16)]


def cache_path() -> str:
    base = os.environ.get("XDG_CACHE_HOME", os.path.join(os.path.expanduser("~"), ".cache"))
    return os.path.join(base, "paper_1909_07439_gb300", "autotune.json")


def _key(torch, n, n_inst):
    return f"{torch.cuda.get_device_name()}|n={n}|inst={n_inst}"


def _load_cache():
    try:
        with open(cache_path()) as f:
            return json.load(f)
    except Exception:
        return {}


def _save_cache(c):
    path = cache_path()
    try:
        os.makedirs(os.path.dirname(path), exist_ok=True)
        with open(path + ".tmp", "w") as f:
            json.dump(c, f, indent=1)
        os.replace(path + ".tmp", path)
    except OSError:
        pass


def tune_batch(ctx, state, d_offsets, n_inst, base=None, steps=2, use_cache=True,
               candidates=CANDIDATES):
    """Return (sph_params, report) with the fastest (n_group, n_leaf) for this batch.
    ``state`` (a DeviceState) is left exactly as it was on entry."""
    import torch
    base = base or native.sph_params_default()
    key = _key(torch, state.n, n_inst)
    cache = _load_cache() if use_cache else {}
    if key in cache and "n_leaf" in cache[key]:
        g, l = cache[key]["n_group"], cache[key]["n_leaf"]
        return native.sph_params_default(**{**_as_dict(base), "n_group": g, "n_leaf": l}), cache[key]
    saved = {f: getattr(state, f).clone() for f in state.FIELDS4 + state.FIELDS1 + ("perm", "keys")}
    dt = torch.zeros(n_inst, dtype=torch.float32, device=state.device)
    trials = []
    for g, l in candidates:
        for f, v in saved.items():
            getattr(state, f).copy_(v)
        p = native.sph_params_default(**{**_as_dict(base), "n_group": g, "n_leaf": l})
        native.sph_batch_evaluate(ctx, state.c, d_offsets, n_inst, p, dt)
        native.sph_batch_step(ctx, state.c, d_offsets, n_inst, 1, p, dt)  # capture + warm
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        native.sph_batch_step(ctx, state.c, d_offsets, n_inst, steps, p, dt)
        e1.record()
        native.sph_sync(ctx)
        trials.append({"n_group": g, "n_leaf": l, "ms_per_step": e0.elapsed_time(e1) / steps})
    for f, v in saved.items():
        getattr(state, f).copy_(v)
    best = min(trials, key=lambda r: r["ms_per_step"])
    report = {"n_group": best["n_group"], "n_leaf": best["n_leaf"], "trials": trials}
    if use_cache:
        cache[key] = report
        _save_cache(cache)
    return native.sph_params_default(**{**_as_dict(base), "n_group": best["n_group"],
                                        "n_leaf": best["n_leaf"]}), report


STEP_CANDIDATES = [(g, l) for g in (8, 16, 32) for l in (16, 32)]


def tune_step(ctx, state, d_dt, tag, base=None, steps=3, use_cache=True,
              candidates=STEP_CANDIDATES, evaluate_only=False):
    """Return (sph_params, report) with the fastest (n_group, n_leaf) for
    sph_step on this state (or, with evaluate_only, for one tree build +
    density + force evaluation).  ``state`` and ``d_dt`` are left as they were."""
    import torch
    base = base or native.sph_params_default()
    key = _key(torch, state.n, tag)
    cache = _load_cache() if use_cache else {}
    if key in cache and "n_leaf" in cache[key]:
        g, l = cache[key]["n_group"], cache[key]["n_leaf"]
        return native.sph_params_default(**{**_as_dict(base), "n_group": g, "n_leaf": l}), cache[key]
    saved = {f: getattr(state, f).clone() for f in state.FIELDS4 + state.FIELDS1 + ("perm", "keys")}
    dt0 = d_dt.clone()
    trials = []
    for g, l in candidates:
        p = native.sph_params_default(**{**_as_dict(base), "n_group": g, "n_leaf": l})
        def run(k):
            for _ in range(k):
                if evaluate_only:
                    native.sph_build_tree(ctx, state.c, p)
                    native.sph_density(ctx, state.c, p)
                    native.sph_force(ctx, state.c, p)
                else:
                    native.sph_step(ctx, state.c, p, d_dt)
        for f, v in saved.items():
            getattr(state, f).copy_(v)
        d_dt.copy_(dt0)
        run(1)  # warm
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        run(steps)
        e1.record()
        native.sph_sync(ctx)
        trials.append({"n_group": g, "n_leaf": l, "ms_per_step": e0.elapsed_time(e1) / steps})
    for f, v in saved.items():
        getattr(state, f).copy_(v)
    d_dt.copy_(dt0)
    native.sph_sync(ctx)
    best = min(trials, key=lambda r: r["ms_per_step"])
    report = {"n_group": best["n_group"], "n_leaf": best["n_leaf"], "trials": trials}
    if use_cache:
        cache[key] = report
        _save_cache(cache)
    return native.sph_params_default(**{**_as_dict(base), "n_group": best["n_group"],
                                        "n_leaf": best["n_leaf"]}), report


def _as_dict(p):
    return {k: getattr(p, k) for k, _ in p._fields_}
