"""Pins of the RL / Simp oracle (oracle/postprocess.py) against things other
than itself: a grammar worked out by hand, the expansion of every string
(which post-processing must not change), the size identities of the two
steps, and the defining properties of their outputs."""
import numpy as np
import pytest

import lcg_inputs as li
from oracle import oracle as O
from oracle import postprocess as P


def level(rules):
    off = np.zeros(len(rules) + 1, dtype=np.uint64)
    off[1:] = np.cumsum([len(r) for r in rules])
    rhs = np.asarray([x for r in rules for x in r], dtype=np.uint32)
    return {"g": len(rules), "rhs_off": off, "rhs": rhs, "F": np.zeros(len(rules), dtype=np.uint32)}


def hand_grammar():
    # level 1 over bytes: 0 = AAAC, 1 = CG, 2 = GG
    # level 2 over level 1: 0 = [0 1], 1 = [1 2 2 2], 2 = [0 0]
    # level 3 over level 2: 0 = [0 1 2]
    # string 0 has root (3, 0); string 1 has root (2, 1)
    A, C, G = 65, 67, 71
    return {"F0": np.zeros(256, dtype=np.uint32),
            "levels": [level([[A, A, A, C], [C, G], [G, G]]), level([[0, 1], [1, 2, 2, 2], [0, 0]]), level([[0, 1, 2]])],
            "c_level": np.asarray([3, 2], dtype=np.uint32), "c_rank": np.asarray([0, 1], dtype=np.uint32)}


def test_hand_worked_grammar():
    """Worked by hand from the two definitions.
    RL, level 1: A^3 -> (A,3) = L1 run 0, G^2 -> (G,2) = L1 run 1;
        level 2: 2^3 -> (2,3) = L2 run 0, 0^2 -> (0,2) = L2 run 1.
    Uses in level 3: each level-2 rule once; level-2 rule 1 is a root, so
    rules 0 and 2 of level 2 are inlined.  Level-1 rules 0 and 2 are bases of
    level-2 runs and rule 1 is used twice: all kept.
    Ids: L1 rules 256 257 258, L1 runs 259 260, L2 rule 1 -> 261, L2 runs
    262 263, L3 rule 0 -> 264."""
    pp = P.postprocess(hand_grammar())
    want_rules = [(0, [259, 67]), (0, [67, 71]), (0, [260]), (1, [65, 3]), (1, [71, 2]),
                  (0, [257, 262]), (1, [258, 3]), (1, [256, 2]), (0, [256, 257, 261, 263])]
    assert pp["kind"].tolist() == [k for k, _ in want_rules]
    got = [pp["rhs"][int(pp["rhs_off"][r]):int(pp["rhs_off"][r + 1])].tolist() for r in range(len(want_rules))]
    assert got == [rhs for _, rhs in want_rules]
    assert pp["c"].tolist() == [264, 261]
    assert P.expand_symbol(pp, 264) == b"AAACCG" + b"CG" + b"GG" * 3 + b"AAAC" * 2
    assert P.expand_symbol(pp, 261) == b"CG" + b"GG" * 3
    st = pp["stats"]
    assert (st["size_before"], st["size_rl"], st["size"], st["rl_rules"], st["removed"]) == (19, 21, 19, 4, 2)


def collections():
    rng = np.random.default_rng(21)
    yield li.from_strings([b"N" * 3000, b"ACGT" * 500 + b"N" * 777 + b"A" * 50, b"A", b"GG"])
    yield li.from_strings([li.random_dna(rng, 4000).tobytes() for _ in range(3)] * 2)  # repeated strings
    yield li.from_strings([li.zipf_text(rng, 20_000), li.zipf_text(rng, 9_000)])
    yield li.tiny_dna_collection(base_len=30_000, k=4)


def rl_runs(rhs_off, rhs):
    """(symbol, length) of every maximal run of length >= 2, rule by rule."""
    out = []
    for r in range(len(rhs_off) - 1):
        q = rhs[int(rhs_off[r]):int(rhs_off[r + 1])].tolist()
        p = 0
        while p < len(q):
            e = p
            while e < len(q) and q[e] == q[p]:
                e += 1
            if e - p >= 2:
                out.append((q[p], e - p))
            p = e
    return out


@pytest.mark.parametrize("idx", range(4))
def test_expansions_sizes_and_properties(hf, idx):
    coll = list(collections())[idx]
    ex = O.build(coll, hf).export()
    pp = P.postprocess(ex)
    # every string expands to itself
    for j in range(coll.k):
        assert P.expand_symbol(pp, int(pp["c"][j])) == coll.string(j).tobytes()
    st = pp["stats"]
    runs = [rl_runs(L["rhs_off"], np.asarray(L["rhs"])) for L in ex["levels"]]
    saved = sum(length - 1 for lv in runs for (_, length) in lv)
    distinct = sum(len(set(lv)) for lv in runs)
    # RL: each run of length l leaves one symbol; each distinct run adds a two-entry rule
    assert st["rl_rules"] == distinct
    assert st["size_rl"] == st["size_before"] - saved + 2 * distinct
    # Simp: removing a rule used once saves exactly the symbol that named it
    assert st["size"] == st["size_rl"] - st["removed"]
    assert st["rules"] == sum(L["g"] for L in ex["levels"]) - st["removed"] + distinct
    # run-length rules: length >= 2, distinct within the output
    kind, off, rhs = pp["kind"], pp["rhs_off"], pp["rhs"]
    rl = [tuple(rhs[int(off[r]):int(off[r + 1])].tolist()) for r in np.nonzero(kind == 1)[0]]
    assert all(len(t) == 2 and t[1] >= 2 for t in rl)
    assert len(set(rl)) == len(rl)  # bases of different levels are different ids
    # Simp: a regular rule left with exactly one use is a root or a run base
    uses = np.zeros(len(kind) + 256, dtype=np.int64)
    for r in np.nonzero(kind == 0)[0]:
        np.add.at(uses, rhs[int(off[r]):int(off[r + 1])].astype(np.int64), 1)
    bases = {int(rhs[int(off[r])]) for r in np.nonzero(kind == 1)[0]}
    roots = set(pp["c"].tolist())
    for r in np.nonzero(kind == 0)[0]:
        s = 256 + int(r)
        if uses[s] <= 1:
            assert s in roots or s in bases


def test_rl_level_maximal_and_exact():
    """RL of one level: no two equal plain symbols side by side, and each
    reference stands for its run."""
    rng = np.random.default_rng(5)
    rules = [rng.integers(0, 3, size=int(rng.integers(1, 12))).tolist() for _ in range(300)]
    L = level(rules)
    off, new, table = P.rl_level(L["rhs_off"], L["rhs"])
    for r, q in enumerate(rules):
        seg = new[int(off[r]):int(off[r + 1])].tolist()
        back = []
        for v in seg:
            if v & P.RL_FLAG:
                y, length = table[v & ~P.RL_FLAG]
                back += [y] * length
            else:
                back.append(v)
        assert back == q
        assert all(a != b for a, b in zip(seg, seg[1:]))  # runs are maximal
    # first-occurrence numbering
    seen = []
    for r in range(len(rules)):
        for v in new[int(off[r]):int(off[r + 1])].tolist():
            if v & P.RL_FLAG and (v & ~P.RL_FLAG) not in seen:
                seen.append(v & ~P.RL_FLAG)
    assert seen == list(range(len(table)))
