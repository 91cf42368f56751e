"""Pins of the CPU oracle against what the paper and the mathematics fix.

None of these tests compares the oracle with itself: each checks it against a
brute-force or textbook formulation (tests/brute.py), a closed form, a
published test vector, an invariant the paper proves, or the values printed in
the caption of Fig. 3.
"""
import itertools
import json
import math
import os

import numpy as np
import pytest

import lcg_inputs as li
from oracle import oracle as O
from tests import brute

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# --------------------------------------------------------------------------
# hash family
# --------------------------------------------------------------------------

def test_splitmix64_published_vector():
    # first outputs of splitmix64 started at 0 (Vigna's reference generator)
    assert li.splitmix64_stream(0, 2) == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4]


def test_hash_family_ranges(hf):
    for arr in (hf.a, hf.b, hf.c):
        assert np.all(arr >= 1) and np.all(arr < li.MERSENNE61)
    assert len(set(hf.c.tolist())) == hf.levels


@pytest.mark.parametrize("m_bits", [32, 16, 2])
def test_h0_closed_form(m_bits):
    """F^0 over all bytes equals ((a s + b) mod p) mod m (Sec. 2.4)."""
    hf = li.hash_family(m_bits=m_bits)
    g = O.build(li.from_strings([b"AC"]), hf)
    F0 = g.export()["F0"]
    for s in range(256):
        assert int(F0[s]) == brute.h0(hf, s)


def test_level_hash_matches_tree_evaluation(hf):
    """Every stored F^i equals Eq. lvl_hash evaluated recursively over PT(X)
    with explicit powers, on a collection with many levels.  A transposed
    polynomial (c^(q-j)), a dropped a_i or b_i, or the parameters of the wrong
    level all fail here."""
    coll = li.tiny_dna_collection(base_len=4000, k=3)
    ex = O.build(coll, hf).export()
    memo = {}
    assert len(ex["levels"]) >= 8
    for i, L in enumerate(ex["levels"], start=1):
        for r in range(L["g"]):
            assert int(L["F"][r]) == brute.fingerprint_tree(hf, ex["levels"], i, r, memo)


def test_level_hash_order_sensitive(hf):
    """h^i of Q and of its reverse differ (the polynomial gives Q[1] the power
    c^0); checked on level-1 rules whose reverse is also a rule."""
    coll = li.tiny_dna_collection(base_len=20000, k=1)
    ex = O.build(coll, hf).export()
    L = ex["levels"][0]
    rules = {tuple(L["rhs"][int(L["rhs_off"][r]):int(L["rhs_off"][r + 1])].tolist()): r for r in range(L["g"])}
    pairs = [(q, q[::-1]) for q in rules if q[::-1] in rules and q != q[::-1]]
    assert pairs
    for q, rq in pairs:
        assert L["F"][rules[q]] != L["F"][rules[rq]]


# --------------------------------------------------------------------------
# RandLMSPar breaks
# --------------------------------------------------------------------------

def test_breaks_exhaustive_small_alphabet():
    """Type recursion (oracle) == plateau-minimum formulation, on every
    sequence of length <= 7 over {0,1,2}."""
    for n in range(1, 8):
        for f in itertools.product(range(3), repeat=n):
            assert O.breaks(np.array(f)).tolist() == brute.plateau_breaks(list(f)), f


def test_breaks_random_with_runs():
    rng = np.random.default_rng(11)
    for _ in range(300):
        n = int(rng.integers(1, 200))
        f = rng.integers(0, int(rng.integers(1, 6)), size=n).astype(np.uint32)
        f = np.repeat(f, rng.integers(1, 4, size=n))
        assert O.breaks(f).tolist() == brute.plateau_breaks(f.tolist())


def test_breaks_extreme_values():
    f = np.array([0xFFFFFFFF, 0, 0xFFFFFFFF, 0, 0, 0xFFFFFFFF, 5, 5], dtype=np.uint32)
    assert O.breaks(f).tolist() == brute.plateau_breaks(f.tolist()) == [1, 1, 0, 1, 0, 0, 0, 0]


def test_breaks_reduce_to_nong_lms():
    """With an order-preserving h^0 (identity), the phrase starts other than
    position 0 are exactly the LMS positions of the textbook induced-sorting
    classification (Eq. lex_types), away from the sentinel."""
    rng = np.random.default_rng(5)
    for _ in range(400):
        n = int(rng.integers(2, 120))
        t = rng.integers(0, int(rng.integers(2, 8)), size=n)
        brk = O.breaks(t.astype(np.uint32))
        got = [l for l in range(1, n) if brk[l]]
        assert got == brute.sais_lms(t.tolist()), t.tolist()


def test_trailing_run_never_breaks():
    """The suffix that is one ~-run has undefined types: no break inside."""
    f = np.array([9, 3, 1, 1, 1, 1], dtype=np.uint32)
    assert O.breaks(f).tolist() == [1, 0, 0, 0, 0, 0]
    f = np.array([9, 3, 7, 1, 1, 1], dtype=np.uint32)
    assert O.breaks(f).tolist() == [1, 1, 0, 0, 0, 0]


# --------------------------------------------------------------------------
# phrases, naming, whole build
# --------------------------------------------------------------------------

def _level1_phrases(ex, j):
    seqs = brute.expand_levels(ex, j)
    if min(seqs) > 0 or 1 not in seqs:
        return None
    L = ex["levels"][0]
    out, pos = [], 0
    for r in seqs[1]:
        ln = int(L["rhs_off"][r + 1] - L["rhs_off"][r])
        out.append((pos, pos + ln - 1))
        pos += ln
    return out


def test_phrases_equal_enumeration(hf):
    rng = np.random.default_rng(3)
    strings = [li.random_dna(rng, int(rng.integers(2, 40))).tobytes() for _ in range(60)]
    strings += [b"AAAAAAAC", b"CAAAAAAA", b"ACACACAC", b"TTTTAAAATTTT"]
    coll = li.from_strings(strings)
    ex = O.build(coll, hf).export()
    F0 = ex["F0"]
    for j, s in enumerate(strings):
        f = [int(F0[x]) for x in s]
        brk = brute.plateau_breaks(f)
        is_lms = [bool(brk[l]) and l > 0 for l in range(len(s))]
        assert _level1_phrases(ex, j) == brute.phrases_by_enumeration(is_lms, len(s)), s


def test_build_matches_bruteforce_build(hf):
    """Whole grammar (rules in rank order, F, C) equals the dict-based Python
    build, on random tiny collections and on every ACGT string of length <= 5."""
    rng = np.random.default_rng(17)
    cases = []
    for _ in range(40):
        k = int(rng.integers(1, 6))
        cases.append([li.random_dna(rng, int(rng.integers(1, 60))).tobytes() for _ in range(k)])
    for n in range(1, 6):
        cases.append([bytes(p) for p in itertools.product(b"ACGT", repeat=n)])
    for strings in cases:
        ex = O.build(li.from_strings(strings), hf).export()
        levels, C = brute.build(strings, hf)
        assert len(ex["levels"]) == len(levels)
        for L, B in zip(ex["levels"], levels):
            rules = [tuple(L["rhs"][int(L["rhs_off"][r]):int(L["rhs_off"][r + 1])].tolist()) for r in range(L["g"])]
            assert rules == B["rules"]
            assert L["F"].tolist() == B["F"]
        assert list(zip(ex["c_level"].tolist(), ex["c_rank"].tolist())) == C


def _check_invariants(coll, ex):
    g_prev = 256
    for L in ex["levels"]:
        ro = L["rhs_off"]
        assert ro[0] == 0 and np.all(np.diff(ro.astype(np.int64)) >= 1)
        assert int(ro[-1]) == L["rhs"].shape[0]
        assert L["rhs"].size == 0 or int(L["rhs"].max()) < g_prev  # full balance
        # distinct right-hand sides within a level
        rules = {L["rhs"][int(ro[r]):int(ro[r + 1])].tobytes() for r in range(L["g"])}
        assert len(rules) == L["g"]
        g_prev = L["g"]
    for j in range(coll.k):
        nj = int(coll.offsets[j + 1] - coll.offsets[j])
        lev = int(ex["c_level"][j])
        assert lev <= brute.ceil_log2(nj)  # O(log n) rounds: |T^{i+1}| <= ceil(|T^i|/2)
        seqs = brute.expand_levels(ex, j)
        assert bytes(seqs[0]) == coll.string(j).tobytes()
        for i in range(1, lev + 1):
            assert len(seqs[i]) <= math.ceil(len(seqs[i - 1]) / 2)
            # every phrase but the first of a string has length >= 2
            L = ex["levels"][i - 1]
            lens = [int(L["rhs_off"][x + 1] - L["rhs_off"][x]) for x in seqs[i]]
            assert all(ln >= 2 for ln in lens[1:])


def test_invariants_dna_and_edge(hf):
    for coll in (li.tiny_dna_collection(base_len=30000, k=4), li.edge_collection()):
        g = O.build(coll, hf)
        ex = g.export()
        _check_invariants(coll, ex)
        for j in range(coll.k):
            assert g.decompress(j) == coll.string(j).tobytes()


def test_invariants_text(hf):
    rng = np.random.default_rng(2)
    coll = li.from_strings([li.zipf_text(rng, 20000, copy_frac=0.3), li.zipf_text(rng, 7000, copy_frac=0.0)])
    ex = O.build(coll, hf).export()
    _check_invariants(coll, ex)


def test_empty_string_rejected(hf):
    coll = li.Collection(data=np.frombuffer(b"ACGT", dtype=np.uint8),
                         offsets=np.array([0, 2, 2, 4], dtype=np.uint64))
    with pytest.raises(O.OracleError):
        O.build(coll, hf)


def test_worked_example_strings_roundtrip(hf):
    """The strings of Fig. 2 and Fig. 3 (Sec. 3.3, Sec. 3.6).  Their grammars
    depend on the paper's unknown hash draws: only the round trip and the
    invariants are checked here (values unpinned)."""
    strings = [b"agtagtagtgtagtaggagatcggag", b"agtagtagtgtagtaggtcag"]
    coll = li.from_strings(strings)
    g = O.build(coll, hf)
    _check_invariants(coll, g.export())


# --------------------------------------------------------------------------
# collisions (Sec. 3.4, note on collisions)
# --------------------------------------------------------------------------

@pytest.mark.parametrize("m_bits", [1, 2, 3])
def test_colliding_fingerprints_stay_exact(m_bits):
    """With tiny m nearly all fingerprints collide: ~-runs merge and phrases get
    long, but distinct contents must still get distinct ranks and every string
    must decompress exactly."""
    hf = li.hash_family(m_bits=m_bits)
    rng = np.random.default_rng(m_bits)
    strings = [li.random_dna(rng, int(rng.integers(1, 300))).tobytes() for _ in range(12)]
    coll = li.from_strings(strings)
    g = O.build(coll, hf)
    ex = g.export()
    _check_invariants(coll, ex)
    levels, C = brute.build(strings, hf)
    for L, B in zip(ex["levels"], levels):
        assert L["F"].tolist() == B["F"]


# --------------------------------------------------------------------------
# MergeGrams (Sec. 3.5-3.6)
# --------------------------------------------------------------------------

def test_merge_equals_build_of_union_exhaustive(hf):
    """MergeGrams(Build(A), Build(B)) == Build(A o B), bit for bit, for all
    pairs of ACGT strings of lengths 1..4 (a sample of pairs) and larger ones."""
    words = [bytes(p) for n in range(1, 5) for p in itertools.product(b"ACGT", repeat=n)]
    rng = np.random.default_rng(0)
    idx = rng.choice(len(words), size=(400, 2))
    for x, y in idx.tolist():
        A, B = [words[x]], [words[y]]
        ga = O.build(li.from_strings(A), hf)
        ga.merge(O.build(li.from_strings(B), hf))
        assert O.grammars_equal(ga.export(), O.build(li.from_strings(A + B), hf).export())


def test_merge_equals_build_of_union_dna(hf):
    coll = li.tiny_dna_collection(base_len=20000, k=6)
    ga = O.build(coll.subset(range(0, 2)), hf)
    gb = O.build(coll.subset(range(2, 6)), hf)
    ga.merge(gb)
    assert O.grammars_equal(ga.export(), O.build(coll, hf).export())


def test_merge_fold_and_associativity(hf):
    rng = np.random.default_rng(9)
    strings = [li.random_dna(rng, int(rng.integers(1, 400))).tobytes() for _ in range(7)]
    whole = O.build(li.from_strings(strings), hf).export()
    fold = O.build(li.from_strings(strings[:1]), hf)
    for s in strings[1:]:
        fold.merge(O.build(li.from_strings([s]), hf))
    assert O.grammars_equal(fold.export(), whole)
    left = O.build(li.from_strings(strings[:3]), hf).merge(O.build(li.from_strings(strings[3:5]), hf))
    left.merge(O.build(li.from_strings(strings[5:]), hf))
    right = O.build(li.from_strings(strings[3:5]), hf).merge(O.build(li.from_strings(strings[5:]), hf))
    left2 = O.build(li.from_strings(strings[:3]), hf).merge(right)
    assert O.grammars_equal(left.export(), left2.export())
    assert O.grammars_equal(left.export(), whole)


@pytest.mark.parametrize("threads", [1, 2, 3, 5, 8, 16])
def test_parallel_build_equals_build(hf, threads):
    """The threaded construction (parts built on separate threads, merged in a
    tree) is the build of the whole collection, for any number of parts,
    including more threads than strings."""
    rng = np.random.default_rng(21)
    strings = [li.random_dna(rng, int(rng.integers(1, 3000))).tobytes() for _ in range(9)]
    coll = li.from_strings(strings)
    assert O.grammars_equal(O.build_parallel(coll, hf, threads).export(), O.build(coll, hf).export())


def test_merge_refuses_other_hash_family(hf):
    g1 = O.build(li.from_strings([b"ACGTACGT"]), hf)
    g2 = O.build(li.from_strings([b"ACGTACGT"]), li.hash_family(seed=99))
    with pytest.raises(O.OracleError):
        g1.merge(g2)


def test_merge_fig3_caption_values():
    """Fig. 3 (Sec. 3.6) prints the rank map of its merge example: level-1 rule
    5 -> agg of G_b matches 1 -> agg of G_a, tc is new and becomes rule 6, and
    the level-2 rules of G_b, 1 -> 1 1 4 3 1 and 2 -> 5 2 4, are rewritten to
    1 -> 2 2 3 4 2 and 2 -> 1 6 3.  The fixture rebuilds grammars consistent
    with that caption (1-based there, 0-based ranks here) and checks that the
    merge reproduces the printed values."""
    with open(os.path.join(GOLDEN, "merge_fig3.json")) as fh:
        fx = json.load(fh)

    def mk(spec):
        levels = []
        for L in spec["levels"]:
            rules = L["rules"]
            ro = np.zeros(len(rules) + 1, dtype=np.uint64)
            ro[1:] = np.cumsum([len(q) for q in rules])
            rhs = np.array([x for q in rules for x in q], dtype=np.uint32)
            levels.append({"g": len(rules), "rhs_off": ro, "rhs": rhs, "F": np.array(L["F"], dtype=np.uint32)})
        return {"F0": np.arange(256, dtype=np.uint32), "levels": levels,
                "c_level": np.array(spec["c_level"], dtype=np.uint32),
                "c_rank": np.array(spec["c_rank"], dtype=np.uint32)}

    ga = O.from_export(mk(fx["G_a"]), 7)
    gb = O.from_export(mk(fx["G_b"]), 7)
    ga.merge(gb)
    ex = ga.export()
    L1, L2 = ex["levels"][0], ex["levels"][1]
    exp = fx["expected"]
    assert L1["g"] == exp["level1_g"]
    new1 = L1["rhs"][int(L1["rhs_off"][exp["new_level1_rank"]]):int(L1["rhs_off"][exp["new_level1_rank"] + 1])]
    assert bytes(new1.tolist()) == exp["new_level1_rhs"].encode()
    got2 = [L2["rhs"][int(L2["rhs_off"][r]):int(L2["rhs_off"][r + 1])].tolist() for r in range(L2["g"])]
    assert got2[-2:] == exp["appended_level2_rules"]
    assert ex["c_level"].tolist() == exp["c_level"] and ex["c_rank"].tolist() == exp["c_rank"]


# --------------------------------------------------------------------------
# stable local consistency (Definition 1)
# --------------------------------------------------------------------------

def _breaks_terminal(ex, j):
    """Per level i >= 1: set of terminal offsets where a level-i phrase starts,
    plus per level the terminal span and fingerprint of every level-i symbol."""
    seqs = brute.expand_levels(ex, j)
    lev = int(ex["c_level"][j])
    # terminal length of each symbol, bottom-up
    spans = {0: [(p, p + 1) for p in range(len(seqs[0]))]}
    for i in range(1, lev + 1):
        L = ex["levels"][i - 1]
        out, pos = [], 0
        for x in seqs[i]:
            cnt = int(L["rhs_off"][x + 1] - L["rhs_off"][x])
            out.append((spans[i - 1][pos][0], spans[i - 1][pos + cnt - 1][1]))
            pos += cnt
        spans[i] = out
    fps = {0: [int(ex["F0"][x]) for x in seqs[0]]}
    for i in range(1, lev + 1):
        fps[i] = [int(ex["levels"][i - 1]["F"][x]) for x in seqs[i]]
    return seqs, spans, fps


def test_stable_cores(hf):
    """A pattern P built inside two unrelated contexts, independently: at every
    level, each symbol whose break decision only sees symbols inside the core
    (one to its left, its ~-run and one more to its right) breaks identically,
    and the core symbols carry identical fingerprints (Def. 1, Sec. 3.3)."""
    rng = np.random.default_rng(21)
    checked_levels = 0
    for trial in range(6):
        P = li.random_dna(rng, 3000).tobytes()
        ctx = [(li.random_dna(rng, int(rng.integers(50, 400))).tobytes(),
                li.random_dna(rng, int(rng.integers(50, 400))).tobytes()) for _ in range(2)]
        views = []
        for X, Y in ctx:
            ex = O.build(li.from_strings([X + P + Y]), hf).export()
            views.append((len(X), _breaks_terminal(ex, 0)))
        # core in terminal coordinates relative to P, level by level
        lo, hi = 0, len(P)
        for i in range(0, 12):
            # symbols of level i fully inside [lo, hi) (relative to P), per view
            per_view = []
            for off, (seqs, spans, fps) in views:
                if i not in spans:
                    per_view.append(None)
                    continue
                syms = [(s - off, e - off, fps[i][t]) for t, (s, e) in enumerate(spans[i])
                        if s - off >= lo and e - off <= hi]
                per_view.append(syms)
            if None in per_view or not per_view[0]:
                break
            a, b = per_view
            # fingerprints of the core symbols are context independent
            assert a == b, (trial, i)
            # break decisions of the next round at symbols whose window (one to
            # the left, the ~-run, one to the right) lies inside the core
            fp = [x[2] for x in a]
            safe = []
            for t in range(1, len(fp)):
                r = t
                while r < len(fp) and fp[r] == fp[t]:
                    r += 1
                if r < len(fp):
                    safe.append(t)
            if not safe or i + 1 not in views[0][1][1]:
                break
            starts = []
            for off, (seqs, spans, fps) in views:
                st = {s - off for (s, e) in spans[i + 1]}
                starts.append([a[t][0] in st for t in safe])
            assert starts[0] == starts[1], (trial, i)
            # shrink the core to the next level's complete phrases inside it
            cut = [a[t][0] for t, s in zip(safe, starts[0]) if s]
            if len(cut) < 2:
                break
            lo, hi = cut[0], cut[-1]
            checked_levels = max(checked_levels, i + 1)
    assert checked_levels >= 4


def test_grammar_digests_locate_differences(hf):
    """The digests the full-size GPU tests compare: equal for equal grammars,
    and a change anywhere (one rule symbol, one fingerprint, one root) names
    its level and array."""
    from tests.digests import first_digest_difference, grammar_digests
    coll = li.tiny_dna_collection(base_len=20_000, k=3)
    ex = O.build(coll, hf).export()
    a = grammar_digests(ex)
    assert first_digest_difference(a, grammar_digests(O.build(coll, hf).export())) is None
    ex["levels"][1]["rhs"] = ex["levels"][1]["rhs"].copy()
    ex["levels"][1]["rhs"][5] ^= 1
    assert first_digest_difference(grammar_digests(ex), a) == "level 2: rhs differs"
    ex = O.build(coll, hf).export()
    ex["levels"][0]["F"] = ex["levels"][0]["F"].copy()
    ex["levels"][0]["F"][0] ^= 1
    assert first_digest_difference(grammar_digests(ex), a) == "level 1: F differs"
    ex = O.build(coll, hf).export()
    ex["c_rank"] = ex["c_rank"].copy()
    ex["c_rank"][2] += 1
    assert first_digest_difference(grammar_digests(ex), a) == "C differs"
