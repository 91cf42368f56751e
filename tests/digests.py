"""SHA-256 digests of an exported grammar, level by level.

A grammar of the multi-gigabyte collections is too large to store as a
fixture, so the oracle's export is stored as digests: per level the number of
rules g, the number of right-hand-side symbols G, and one digest each of
rhs_off (uint64), rhs (uint32) and F (uint32); plus digests of F^0 and of the
roots C (c_level, c_rank as uint32).  Two exports agree exactly when all
digests and sizes agree (up to SHA-256 collisions), and the first differing
entry names the level and array that differ.
"""
from __future__ import annotations

import hashlib

import numpy as np


def _sha(*arrays) -> str:
    h = hashlib.sha256()
    for a in arrays:
        a = np.ascontiguousarray(a)
        h.update(memoryview(a).cast("B"))
    return h.hexdigest()


def grammar_digests(ex: dict) -> dict:
    """Digests of an export dict (``levels``, ``F0``, ``c_level``, ``c_rank``)."""
    levels = []
    for L in ex["levels"]:
        rhs_off = np.asarray(L["rhs_off"], dtype=np.uint64)
        rhs = np.asarray(L["rhs"], dtype=np.uint32)
        F = np.asarray(L["F"], dtype=np.uint32)
        levels.append({
            "g": int(L["g"]),
            "G": int(rhs.shape[0]),
            "rhs_off": _sha(rhs_off),
            "rhs": _sha(rhs),
            "F": _sha(F),
        })
    return {
        "F0": _sha(np.asarray(ex["F0"], dtype=np.uint32)),
        "levels": levels,
        "k": int(np.asarray(ex["c_level"]).shape[0]),
        "C": _sha(np.asarray(ex["c_level"], dtype=np.uint32), np.asarray(ex["c_rank"], dtype=np.uint32)),
    }


def first_digest_difference(got: dict, want: dict):
    """None when equal, else a short description of the first difference."""
    if got["F0"] != want["F0"]:
        return "F0"
    if len(got["levels"]) != len(want["levels"]):
        return f"levels {len(got['levels'])} != {len(want['levels'])}"
    for i, (a, b) in enumerate(zip(got["levels"], want["levels"]), start=1):
        for key in ("g", "G", "rhs_off", "rhs", "F"):
            if a[key] != b[key]:
                return f"level {i}: {key} differs ({a[key]} vs {b[key]})" if key in ("g", "G") else \
                    f"level {i}: {key} differs"
    if got["k"] != want["k"]:
        return f"k {got['k']} != {want['k']}"
    if got["C"] != want["C"]:
        return "C differs"
    return None
