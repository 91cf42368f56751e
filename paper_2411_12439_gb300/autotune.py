"""Autotuner of the build's launch and sizing parameters (lcg_set_tuning).

The parse kernel's resident blocks per SM, the phrase tables' load factor and
the byte rounds' miss-queue threshold change the build's speed, never its
result.  ``autotune`` times builds of a sample collection on a context and
keeps, one parameter at a time (coordinate descent, two sweeps), the value
with the shortest median build time; the context keeps the best setting.
"""
from __future__ import annotations

import time

import numpy as np

CANDIDATES = {
    "parse_blocks_per_sm": [0, 2, 3, 4],
    "table_load": [0.4, 0.5, 0.6, 0.7],
    "miss_flush": [32, 64, 128],
}


def _time_builds(ctx, data, offsets, reps: int) -> float:
    import torch
    times = []
    for _ in range(reps):
        torch.cuda.synchronize()
        t = time.perf_counter()
        ctx.build(data, offsets).free()
        torch.cuda.synchronize()
        times.append(time.perf_counter() - t)
    return float(np.median(times))


def autotune(ctx, data, offsets, reps: int = 3, sweeps: int = 2, candidates=None) -> dict:
    """Tune ``ctx`` on the collection (``data`` on the device, ``offsets`` on
    the host).  Returns {"tuning": best setting, "ms": its median build time,
    "trials": [(setting, ms), ...]}."""
    cands = candidates or CANDIDATES
    best = ctx.tuning()
    ctx.build(data, offsets).free()  # a plan for the builds below
    best_t = _time_builds(ctx, data, offsets, reps)
    trials = [(dict(best), best_t * 1e3)]
    for _ in range(sweeps):
        changed = False
        for name, values in cands.items():
            for v in values:
                if v == best[name]:
                    continue
                trial = dict(best, **{name: v})
                try:
                    ctx.set_tuning(**trial)
                except Exception:
                    continue  # not valid on this device
                t = _time_builds(ctx, data, offsets, reps)
                trials.append((trial, t * 1e3))
                if t < best_t * 0.98:  # a change must win by 2 %
                    best, best_t, changed = trial, t, True
            ctx.set_tuning(**best)
        if not changed:
            break
    ctx.set_tuning(**best)
    return {"tuning": best, "ms": best_t * 1e3, "trials": trials}
