"""Autotuner for the launch knobs of pic_step (pic_set_tuning).

The knobs change how the work is laid out on the GPU, never the result (the
particle grid and the walk form leave every SP bit-identical; the batch
solver's block budget changes only the reduction order; the Chebyshev degree
changes the preconditioner, not the stopping rule).  The tuner times whole
steps on the caller's own state: it snapshots the state once (potential, SPs,
step index), and before each candidate restores it, runs warm-up steps,
restores it again and times ``steps`` steps, so every candidate does exactly
the same physical work.  Search: coordinate descent from the current knobs,
one knob at a time over its candidate values, repeated while it improves.

Results are cached in a JSON file keyed by device name and workload signature
(precision, replicas, tetrahedra, SPs in flight rounded to a power of two),
so a second run of the same workload reuses them.
"""
from __future__ import annotations

import json
import os
import time

import numpy as np

SPACE = {
    "particle_blocks_per_sm": (4, 8, 16, 24, 32),
    "walk_form": (1, 2, 3),
    "pcg_blocks_per_sm": (0, 1, 2, 4),
    "pcg_cheb_degree": (0, 4, 6, 8),
    "pcg_balance": (0, 1),
}


def default_cache_path() -> str:
    base = os.environ.get("XDG_CACHE_HOME", os.path.join(os.path.expanduser("~"), ".cache"))
    return os.path.join(base, "paper_1906_08125_gb300", "tuning.json")


def signature(ctx) -> str:
    """Workload signature of a loaded context (what the best knobs depend on)."""
    import torch
    info = ctx.info()
    n_sp = max(1, ctx.num_particles())
    dev = torch.cuda.get_device_name(torch.cuda.current_device())
    return (f"{dev}|prec{ctx.params['precision']}|rep{info['n_rep']}|tets{info['n_tets']}"
            f"|sp2^{int(round(np.log2(n_sp)))}")


class _Snapshot:
    def __init__(self, ctx):
        self.ctx = ctx
        self.phi = ctx.potential()
        self.parts = ctx.particles()
        self.k = ctx.step_index

    def restore(self):
        self.ctx.set_potential(self.phi)
        self.ctx.set_particles(*self.parts)
        self.ctx.step_index = self.k


def _time_steps(ctx, snap, steps, warmup) -> float:
    snap.restore()
    if warmup:
        ctx.step(warmup, stats=False)
    snap.restore()
    ctx.sync()
    t0 = time.perf_counter()
    ctx.step(steps, stats=False)
    ctx.sync()
    return (time.perf_counter() - t0) * 1e3 / steps


def tune(ctx, steps=4, warmup=2, space=None, cache_path=None, use_cache=True, log=None):
    """Pick the fastest knobs for the context's current workload, apply them
    and return ``(knobs, ms_per_step, trials)``.  The context's state is
    restored to the snapshot afterwards."""
    space = dict(space or SPACE)
    info = ctx.info()
    if info["n_rep"] <= 1:
        space.pop("pcg_balance", None)             # one system: nothing to balance
        if info["pcg_resident"]:
            space.pop("pcg_blocks_per_sm", None)   # the resident solver ignores it
    if ctx.params["pcg_cheb_degree"] < 2 and "pcg_cheb_degree" in space:
        # a plain Jacobi form stays Jacobi: the degree is part of what it is
        space.pop("pcg_cheb_degree")
    cache_path = cache_path or default_cache_path()
    key = signature(ctx)
    if use_cache and os.path.exists(cache_path):
        try:
            hit = json.load(open(cache_path)).get(key)
        except (OSError, ValueError):
            hit = None
        if hit:
            ctx.set_tuning(**hit["knobs"])
            return hit["knobs"], hit["ms_per_step"], []
    snap = _Snapshot(ctx)
    best = ctx.tuning()
    trials = []

    def run(knobs):
        ctx.set_tuning(**knobs)
        ms = _time_steps(ctx, snap, steps, warmup)
        trials.append((dict(knobs), ms))
        if log:
            log(f"autotune {knobs} -> {ms:.3f} ms/step")
        return ms

    best_ms = run(best)
    improved = True
    while improved:
        improved = False
        for name, values in space.items():
            for v in values:
                if v == best[name]:
                    continue
                cand = dict(best, **{name: v})
                ms = run(cand)
                if ms < best_ms * 0.98:        # 2 %: below that it is noise
                    best, best_ms, improved = cand, ms, True
    ctx.set_tuning(**best)
    snap.restore()
    if use_cache:
        os.makedirs(os.path.dirname(cache_path), exist_ok=True)
        try:
            data = json.load(open(cache_path)) if os.path.exists(cache_path) else {}
        except (OSError, ValueError):
            data = {}
        data[key] = {"knobs": best, "ms_per_step": best_ms}
        json.dump(data, open(cache_path, "w"), indent=1, sort_keys=True)
    return best, best_ms, trials
