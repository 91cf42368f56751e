"""Plain oracle of the grammar post-processing steps RL and Simp (Sec. 2.2,
post-processing paragraph; Sec. 4, implementation details: RL runs on the
output of BuildGram, then Simp).

TEST INFRASTRUCTURE ONLY: the tests, the smoke check and the benchmark's CPU
baseline use it; the product path never imports it.

Input: an exported level grammar (``oracle.Grammar.export()`` layout: per
level ``rhs_off`` / ``rhs`` over the ranks of the level below, bytes at level
1, and the roots ``c_level`` / ``c_rank``).

RL (run-length compression): every maximal run Y^l (l >= 2) of one symbol in
the right-hand side of one rule of level i becomes a reference to a
run-length rule (Y, l) of level i; the distinct pairs of a level are numbered
in order of first occurrence (rule rank, then position).

Simp (grammar simplification): a rule of level i >= 1 that occurs exactly
once in the right-hand sides of the rules of level i+1, is not the root of a
string and is not the base of a run-length rule, is removed and its
occurrence is replaced by its right-hand side (recursively).

Readings taken here (the paper states the two steps in one sentence each):
  - runs never cross rule boundaries, and the roots C are not run-length
    compressed (each string keeps its own root symbol);
  - a rule used only as a root, or as the base of a run-length rule, is kept;
    run-length rules are never inlined (they are constant-size);
  - output numbering: terminals are the byte values 0..255; then level by
    level, the surviving rules of the level in rank order followed by the
    level's run-length rules in their order, get the ids 256, 257, ...;
  - a run-length rule is stored as the two-entry right-hand side
    [base id, run length] with kind 1; other rules have kind 0.

Output: {"kind": uint8[R], "rhs_off": uint64[R+1], "rhs": uint32[...],
"c": uint32[k]} plus "stats".  The size of the grammar is len(rhs).
"""
from __future__ import annotations

import numpy as np

RL_FLAG = 1 << 31  # marks a run-length rule id in an RL-rewritten right-hand side


def rl_level(rhs_off: np.ndarray, rhs: np.ndarray):
    """RL of one level: (new_off, new_rhs, rl_rules) where new_rhs holds a
    plain symbol Y or RL_FLAG | id, and rl_rules[id] = (Y, l)."""
    rhs_off = np.asarray(rhs_off, dtype=np.uint64)
    rhs = np.asarray(rhs, dtype=np.uint32)
    g = rhs_off.shape[0] - 1
    ids: dict[tuple[int, int], int] = {}
    rules: list[tuple[int, int]] = []
    new_off = np.zeros(g + 1, dtype=np.uint64)
    out: list[int] = []
    for r in range(g):
        a, b = int(rhs_off[r]), int(rhs_off[r + 1])
        p = a
        while p < b:
            y = int(rhs[p])
            e = p + 1
            while e < b and int(rhs[e]) == y:
                e += 1
            length = e - p
            if length >= 2:
                key = (y, length)
                if key not in ids:
                    ids[key] = len(rules)
                    rules.append(key)
                out.append(RL_FLAG | ids[key])
            else:
                out.append(y)
            p = e
        new_off[r + 1] = len(out)
    return new_off, np.asarray(out, dtype=np.uint32), rules


def postprocess(ex: dict) -> dict:
    """RL, then Simp, of an exported level grammar."""
    levels = ex["levels"]
    nl = len(levels)
    c_level = np.asarray(ex["c_level"], dtype=np.uint32)
    c_rank = np.asarray(ex["c_rank"], dtype=np.uint32)
    size_before = int(sum(np.asarray(L["rhs"]).shape[0] for L in levels))

    # RL, level by level
    rl = [rl_level(L["rhs_off"], L["rhs"]) for L in levels]
    size_rl = int(sum(x[1].shape[0] + 2 * len(x[2]) for x in rl))

    # Simp: uses of every rule of level i in the right-hand sides of level i+1
    g = [int(L["g"]) for L in levels]
    uses = [np.zeros(gi, dtype=np.int64) for gi in g]
    pinned = [np.zeros(gi, dtype=bool) for gi in g]
    for i in range(1, nl):  # level i+1 (index i) refers to level i (index i-1)
        new_rhs = rl[i][1]
        plain = new_rhs[(new_rhs & RL_FLAG) == 0]
        np.add.at(uses[i - 1], plain.astype(np.int64), 1)
        for (y, _) in rl[i][2]:
            pinned[i - 1][y] = True
    for lv, rk in zip(c_level.tolist(), c_rank.tolist()):
        if lv > 0:
            pinned[lv - 1][rk] = True
    removable = [(uses[i] == 1) & ~pinned[i] for i in range(nl)]

    # final ids: level by level, surviving rules in rank order, then RL rules
    fid = []      # fid[i][r]: final id of surviving rule r of level i+1
    rl_fid = []   # rl_fid[i][id]: final id of run-length rule id of level i+1
    nxt = 256
    for i in range(nl):
        f = np.full(g[i], -1, dtype=np.int64)
        surv = np.nonzero(~removable[i])[0]
        f[surv] = nxt + np.arange(surv.shape[0])
        nxt += surv.shape[0]
        fid.append(f)
        rl_fid.append(nxt + np.arange(len(rl[i][2])))
        nxt += len(rl[i][2])

    def sym_id(level: int, y: int) -> int:
        """Final id of plain symbol y of `level` (0: a byte)."""
        return y if level == 0 else int(fid[level - 1][y])

    def expand(level: int, r: int, out: list):
        """Right-hand side of rule r of `level` (1-based) with removed rules
        replaced by their own right-hand sides."""
        off, new_rhs, _ = rl[level - 1]
        for p in range(int(off[r]), int(off[r + 1])):
            v = int(new_rhs[p])
            if v & RL_FLAG:
                out.append(int(rl_fid[level - 1][v & ~RL_FLAG]))
            elif level >= 2 and removable[level - 2][v]:
                expand(level - 1, v, out)
            else:
                out.append(sym_id(level - 1, v))

    kind, rhs_off, rhs = [], [0], []
    for i in range(nl):
        for r in np.nonzero(~removable[i])[0].tolist():
            expand(i + 1, r, rhs)
            kind.append(0)
            rhs_off.append(len(rhs))
        for (y, length) in rl[i][2]:
            rhs.extend([sym_id(i, y), length])
            kind.append(1)
            rhs_off.append(len(rhs))
    c = np.asarray([sym_id(int(lv), int(rk)) for lv, rk in zip(c_level, c_rank)], dtype=np.uint32)
    removed = int(sum(int(x.sum()) for x in removable))
    return {
        "kind": np.asarray(kind, dtype=np.uint8),
        "rhs_off": np.asarray(rhs_off, dtype=np.uint64),
        "rhs": np.asarray(rhs, dtype=np.uint32),
        "c": c,
        "stats": {"size_before": size_before, "size_rl": size_rl, "size": len(rhs),
                  "rl_rules": int(sum(len(x[2]) for x in rl)), "removed": removed,
                  "rules": len(kind)},
    }


def expand_symbol(pp: dict, s: int) -> bytes:
    """exp(s) in a post-processed grammar (iterative, explicit stack)."""
    out = bytearray()
    stack = [(s, 1)]
    kind, off, rhs = pp["kind"], pp["rhs_off"], pp["rhs"]
    while stack:
        x, times = stack.pop()
        if x < 256:
            out.extend(bytes([x]) * times)
            continue
        r = x - 256
        a, b = int(off[r]), int(off[r + 1])
        if kind[r] == 1:
            base, length = int(rhs[a]), int(rhs[a + 1])
            for _ in range(times):
                stack.append((base, length))
        else:
            for _ in range(times):
                for p in range(b - 1, a - 1, -1):
                    stack.append((int(rhs[p]), 1))
    return bytes(out)


def pp_equal(x: dict, y: dict) -> bool:
    return all(np.array_equal(np.asarray(x[k]), np.asarray(y[k])) for k in ("kind", "rhs_off", "rhs", "c"))
