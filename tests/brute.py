"""Brute-force formulations used to pin the oracle (tiny inputs only).

Each function restates a definition of the paper in a different form from the
oracle's, so that a mistake in either shows up as a disagreement:

* ``plateau_breaks``: a break at l >= 1 iff f[l-1] > f[l] and the first value
  to the right of l that differs from f[l] exists and is larger (the run of
  ~-equal values starting at l is a local minimum).  The oracle instead runs the
  right-to-left type recursion of Eq. rand_types.
* ``sais_lms``: the textbook induced-sorting classification (sentinel-terminated
  L/S types of Nong et al., Eq. lex_types) used for the special case where h^0
  preserves the byte order.
* ``phrases_by_enumeration``: every pair (l, r) that satisfies conditions (i)
  and (ii) of the phrase definition with no LMS position inside.
* ``fingerprint_tree``: Eq. lvl_hash evaluated recursively over the parse tree
  PT(X) with Python integers and explicit powers c^(j-1), as opposed to the
  F-array shortcut of Eq. fast_hash with a running power.
* ``build``: a complete BuildGram with a Python dict for the phrase set.
"""
from __future__ import annotations

import math

P61 = (1 << 61) - 1


def plateau_breaks(f):
    n = len(f)
    out = [0] * n
    if n:
        out[0] = 1
    for l in range(1, n):
        if not f[l - 1] > f[l]:
            continue
        r = l + 1
        while r < n and f[r] == f[l]:
            r += 1
        if r < n and f[r] > f[l]:
            out[l] = 1
    return out


def sais_lms(t):
    """LMS positions in [1, n-1] of t followed by a unique smallest sentinel."""
    n = len(t)
    typ = [None] * (n + 1)
    typ[n] = "S"  # sentinel
    if n:
        typ[n - 1] = "L"  # t[n-1] > sentinel
    for i in range(n - 2, -1, -1):
        if t[i] < t[i + 1] or (t[i] == t[i + 1] and typ[i + 1] == "S"):
            typ[i] = "S"
        else:
            typ[i] = "L"
    return [i for i in range(1, n) if typ[i] == "S" and typ[i - 1] == "L"]


def phrases_by_enumeration(is_lms, n):
    """All (l, r) with (i) l = 0 or LMS(l), (ii) r = n-1 or LMS(r+1), and no LMS
    position in (l, r]."""
    out = []
    for l in range(n):
        if not (l == 0 or is_lms[l]):
            continue
        for r in range(l, n):
            if not (r == n - 1 or is_lms[r + 1]):
                continue
            if any(is_lms[x] for x in range(l + 1, r + 1)):
                continue
            out.append((l, r))
    return out


def h0(hf, s):
    m = 1 << hf.m_bits
    return ((int(hf.a[0]) * s + int(hf.b[0])) % P61) % m


def level_hash(hf, i, child_fps):
    a, b, c = int(hf.a[i]), int(hf.b[i]), int(hf.c[i])
    m = 1 << hf.m_bits
    poly = sum(v * pow(c, j, P61) for j, v in enumerate(child_fps))
    return ((a * poly + b) % P61) % m


def fingerprint_tree(hf, levels, i, r, memo=None):
    """h^i(rhs(X)) for the rank-r rule of level i, evaluated through PT(X)."""
    if memo is None:
        memo = {}
    key = (i, r)
    if key in memo:
        return memo[key]
    if i == 0:
        v = h0(hf, r)
    else:
        L = levels[i - 1]
        s, e = int(L["rhs_off"][r]), int(L["rhs_off"][r + 1])
        kids = [fingerprint_tree(hf, levels, i - 1, int(x), memo) for x in L["rhs"][s:e]]
        v = level_hash(hf, i, kids)
    memo[key] = v
    return v


def build(strings, hf):
    """BuildGram with plateau breaks and a dict, ranks in first-occurrence order."""
    levels = []
    F = [h0(hf, s) for s in range(256)]
    C = [None] * len(strings)
    active = []
    for j, s in enumerate(strings):
        s = list(s)
        if len(s) == 1:
            C[j] = (0, s[0])
        else:
            active.append((j, s))
    i = 1
    while active:
        rank = {}
        rules = []
        Fi = []
        nxt = []
        for j, seq in active:
            f = [F[x] for x in seq]
            brk = plateau_breaks(f)
            starts = [l for l in range(len(seq)) if brk[l]] + [len(seq)]
            out = []
            for a, b in zip(starts[:-1], starts[1:]):
                q = tuple(seq[a:b])
                if q not in rank:
                    rank[q] = len(rules)
                    rules.append(q)
                    Fi.append(level_hash(hf, i, f[a:b]))
                out.append(rank[q])
            if len(out) == 1:
                C[j] = (i, out[0])
            else:
                nxt.append((j, out))
        levels.append({"rules": rules, "F": Fi})
        F = Fi
        active = nxt
        i += 1
    return levels, C


def expand_levels(ex, j):
    """Sequences of string j at every level, from its C entry down to bytes:
    seqs[i] is the sequence of level-i symbols (T^{i+1}_j)."""
    lev, r = int(ex["c_level"][j]), int(ex["c_rank"][j])
    seqs = {lev: [r]}
    for i in range(lev, 0, -1):
        L = ex["levels"][i - 1]
        nxt = []
        for x in seqs[i]:
            s, e = int(L["rhs_off"][x]), int(L["rhs_off"][x + 1])
            nxt.extend(int(v) for v in L["rhs"][s:e])
        seqs[i - 1] = nxt
    return seqs


def ceil_log2(n):
    return 0 if n <= 1 else math.ceil(math.log2(n))
