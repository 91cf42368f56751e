"""Autotuner of the build's launch and sizing parameters (lcg_set_tuning),
with a cache of the best setting per class of collection.

The parse tile size, the rank rounds' tile order (tiles taken in interleaved
stripes), the parse kernel's resident blocks per SM, the phrase tables' load
factor and the byte rounds' miss-queue threshold change the build's speed,
never its result.
``autotune`` times builds of a sample collection on a context and keeps, one
parameter at a time (coordinate descent, two sweeps), the value with the
shortest median build time; the context keeps the best setting.

``tuned`` looks the collection's class up in a JSON cache first (its alphabet,
its size in powers of two and its number of strings: collections of one class
share the distinct-phrase ratios and per-round sizes that the setting depends
on) and only tunes, and records the result, when the class is new.  The cache
shipped with the package, ``tuning_cache.json``, holds settings measured on a
GB300.
"""
from __future__ import annotations

import json
import math
import os
import time

import numpy as np

CANDIDATES = {
    "parse_tile": [4096, 2048, 1024],
    "parse_tile_min": [16, 4, 64],
    "tile_stripes": [1, 2, 4, 8],
    "parse_blocks_per_sm": [0, 2, 3, 4],
    "table_load": [0.3, 0.35, 0.45, 0.6],
    "miss_flush": [32, 64, 128],
}

CACHE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "tuning_cache.json")


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
            if name not in best:
                continue  # a parameter this context does not have
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


def config_class(n_bytes: int, k: int, sample: np.ndarray) -> str:
    """Class of a collection of ``k`` strings and ``n_bytes`` bytes whose
    first bytes are ``sample``: "dna" when the sample uses at most five
    distinct byte values (ACGT and N), else "bytes"; the size rounded to a
    power of two; and the number of strings in one of 1-8, 9-256, 257 or more."""
    distinct = int(np.unique(np.asarray(sample, dtype=np.uint8)).shape[0]) if len(sample) else 0
    alphabet = "dna" if distinct <= 5 else "bytes"
    size = int(round(math.log2(max(1, int(n_bytes)))))
    strings = "1-8" if k <= 8 else ("9-256" if k <= 256 else "257+")
    return f"{alphabet}/2^{size}B/{strings} strings"


def load_cache(path: str = CACHE) -> dict:
    try:
        with open(path) as fh:
            return json.load(fh)
    except (OSError, ValueError):
        return {}


def store(cls: str, setting: dict, ms: float, path: str = CACHE, note: str = "") -> None:
    cache = load_cache(path)
    cache[cls] = {"tuning": setting, "ms": ms, "note": note}
    tmp = f"{path}.{os.getpid()}.tmp"
    with open(tmp, "w") as fh:
        json.dump(cache, fh, indent=1, sort_keys=True)
        fh.write("\n")
    os.replace(tmp, path)


def tuned(ctx, data, offsets, cls: str, retune: bool = False, reps: int = 3, sweeps: int = 1,
          path: str = CACHE, note: str = "") -> dict:
    """Set ``ctx`` to the cached setting of class ``cls``; when there is none
    (or ``retune``), tune on the collection and record the result.  Returns
    {"class", "tuning", "source": "cache" | "tuned", "ms" (tuned only),
    "trials" (tuned only)}."""
    entry = None if retune else load_cache(path).get(cls)
    if entry is not None:
        try:
            ctx.set_tuning(**entry["tuning"])
            return {"class": cls, "tuning": ctx.tuning(), "source": "cache"}
        except Exception:
            pass  # a setting this device refuses: tune again
    rep = autotune(ctx, data, offsets, reps=reps, sweeps=sweeps)
    try:
        store(cls, rep["tuning"], rep["ms"], path, note)
    except OSError:
        pass  # a read-only install keeps the result for this context only
    return {"class": cls, "tuning": rep["tuning"], "source": "tuned", "ms": rep["ms"], "trials": len(rep["trials"])}
