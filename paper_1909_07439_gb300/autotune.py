"""Autotuners for the tree sizes and the launch shape of the pair kernels.

Stage 1 picks the group size (N_group) and the leaf size (N_leaf); stage 2,
at those sizes, picks the launch shape of the neighbour-list density and
force kernels: targets per warp batch (32 / targets lanes per target), warps
per block and list entries per lane and iteration.  Each candidate is timed
on a few steps of the actual state (graph-replayed for a batch), restoring
the state between trials.  Results are cached in a JSON file keyed by
device, particle count and instance count (or workload tag)."""
from __future__ import annotations

import json
import os

from . import native

CANDIDATES = [(g, l) for g in (8, 16, 32) for l in (8, 16, 32)]
# launch shapes of the pair kernels: (targets per batch, warps per block, entries per iteration)
SHAPES = [(t, w, u) for t in (4, 8, 16) for w in (2, 4, 8) for u in (2, 4)]
TUNED = ("n_group", "n_leaf", "pair_targets", "pair_warps", "pair_unroll")


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


def _with(base, **kw):
    return native.sph_params_default(**{**_as_dict(base), **kw})


def _search(trial, base, candidates, shapes):
    """Stage 1 over (n_group, n_leaf), stage 2 over the launch shapes at the
    stage-1 winner; trial(params) returns ms per step."""
    trials = []
    for g, l in candidates:
        p = _with(base, n_group=g, n_leaf=l)
        trials.append({"n_group": g, "n_leaf": l, "pair_targets": p.pair_targets,
                       "pair_warps": p.pair_warps, "pair_unroll": p.pair_unroll,
                       "ms_per_step": trial(p)})
    best = min(trials, key=lambda r: r["ms_per_step"])
    for t, w, u in shapes:
        if (t, w, u) == (best["pair_targets"], best["pair_warps"], best["pair_unroll"]):
            continue
        p = _with(base, n_group=best["n_group"], n_leaf=best["n_leaf"], pair_targets=t,
                  pair_warps=w, pair_unroll=u)
        trials.append({"n_group": best["n_group"], "n_leaf": best["n_leaf"], "pair_targets": t,
                       "pair_warps": w, "pair_unroll": u, "ms_per_step": trial(p)})
    best = min(trials, key=lambda r: r["ms_per_step"])
    report = {k: best[k] for k in TUNED}
    report["trials"] = trials
    return _with(base, **{k: best[k] for k in TUNED}), report


def _cached(cache, key, base):
    r = cache.get(key)
    if r and all(k in r for k in TUNED):
        return _with(base, **{k: r[k] for k in TUNED}), r
    return None


def tune_batch(ctx, state, d_offsets, n_inst, base=None, steps=2, use_cache=True,
               candidates=CANDIDATES, shapes=SHAPES):
    """Return (sph_params, report) with the fastest tree sizes and launch shape
    for this batch.  ``state`` (a DeviceState) is left exactly as it was on entry."""
    import torch
    base = base or native.sph_params_default()
    key = _key(torch, state.n, n_inst)
    cache = _load_cache() if use_cache else {}
    hit = _cached(cache, key, base)
    if hit:
        return hit
    saved = {f: getattr(state, f).clone() for f in state.FIELDS4 + state.FIELDS1 + ("perm", "keys")}
    dt = torch.zeros(n_inst, dtype=torch.float32, device=state.device)

    def trial(p):
        for f, v in saved.items():
            getattr(state, f).copy_(v)
        native.sph_batch_evaluate(ctx, state.c, d_offsets, n_inst, p, dt)
        native.sph_batch_step(ctx, state.c, d_offsets, n_inst, 1, p, dt)  # capture + warm
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        native.sph_batch_step(ctx, state.c, d_offsets, n_inst, steps, p, dt)
        e1.record()
        native.sph_sync(ctx)
        return e0.elapsed_time(e1) / steps

    p, report = _search(trial, base, candidates, shapes)
    for f, v in saved.items():
        getattr(state, f).copy_(v)
    if use_cache:
        cache[key] = report
        _save_cache(cache)
    return p, report


STEP_CANDIDATES = [(g, l) for g in (8, 16, 32) for l in (16, 32)]


def tune_step(ctx, state, d_dt, tag, base=None, steps=3, use_cache=True,
              candidates=STEP_CANDIDATES, shapes=SHAPES, evaluate_only=False):
    """Return (sph_params, report) with the fastest tree sizes and launch shape
    for sph_step on this state (or, with evaluate_only, for one tree build +
    density + force evaluation).  ``state`` and ``d_dt`` are left as they were."""
    import torch
    base = base or native.sph_params_default()
    key = _key(torch, state.n, tag)
    cache = _load_cache() if use_cache else {}
    hit = _cached(cache, key, base)
    if hit:
        return hit
    saved = {f: getattr(state, f).clone() for f in state.FIELDS4 + state.FIELDS1 + ("perm", "keys")}
    dt0 = d_dt.clone()

    def trial(p):
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
        run(1)  # warm (records the step graph)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        run(steps)
        e1.record()
        native.sph_sync(ctx)
        return e0.elapsed_time(e1) / steps

    p, report = _search(trial, base, candidates, shapes)
    for f, v in saved.items():
        getattr(state, f).copy_(v)
    d_dt.copy_(dt0)
    native.sph_sync(ctx)
    if use_cache:
        cache[key] = report
        _save_cache(cache)
    return p, report


def _as_dict(p):
    return {k: getattr(p, k) for k, _ in p._fields_}
