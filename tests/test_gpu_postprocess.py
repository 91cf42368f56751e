"""Parity of the GPU post-processing (lcg_postprocess: RL, then Simp) with the
oracle, array for array, through the C ABI."""
import numpy as np
import pytest

import lcg_inputs as li
from oracle import oracle as O
from oracle import postprocess as P

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx(hf):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2411_12439_gb300 import Context
    return Context(hf, device=0)


def assert_pp_same(got, want):
    for key in ("kind", "rhs_off", "rhs", "c"):
        x, y = np.asarray(got[key]), np.asarray(want[key])
        assert x.shape == y.shape, f"{key}: shape {x.shape} != {y.shape}"
        bad = np.nonzero(x != y)[0]
        assert bad.size == 0, f"{key}[{bad[0]}] {x[bad[0]]} != {y[bad[0]]} ({bad.size} differ)"


def check(ctx, g, ex):
    want = P.postprocess(ex)
    pp = ctx.postprocess(g)
    got = pp.export()
    assert_pp_same(got, want)
    st = pp.stats()
    for key in ("size_before", "size_rl", "size", "rl_rules", "removed", "rules"):
        assert st[key] == want["stats"][key], key
    assert st["strings"] == want["c"].shape[0]
    pp.free()
    return got


def runs_collection(rng):
    # long equal-symbol runs inside rules at several levels (N-runs, tandem repeats)
    s = [li.random_dna(rng, 3000).tobytes() + b"N" * 20_000 + li.random_dna(rng, 3000).tobytes(),
         b"N" * 50_000, (b"ACGTTG" * 4000), b"A" * 7 + b"C" + b"A" * 7, b"G"]
    return li.from_strings(s)


def test_small_collections(ctx, hf):
    rng = np.random.default_rng(31)
    colls = [li.edge_collection(), runs_collection(rng),
             li.from_strings([li.random_dna(rng, 5000).tobytes() for _ in range(4)] * 3),
             li.from_strings([li.zipf_text(rng, 60_000), li.zipf_text(rng, 20_000, copy_frac=0.0)]),
             li.from_strings([b"A", b"C", b"AC"])]
    for coll in colls:
        g = ctx.build(coll.data, coll.offsets)
        ex = O.build(coll, hf).export()
        before = g.export()
        got = check(ctx, g, ex)
        assert O.grammars_equal(g.export(), before)  # the level grammar is unchanged
        for j in range(coll.k):
            assert P.expand_symbol(got, int(got["c"][j])) == coll.string(j).tobytes()


def test_dna_variants(ctx, hf):
    coll = li.tiny_dna_collection()
    check(ctx, ctx.build(coll.data, coll.offsets), O.build(coll, hf).export())


def test_bacterial_subset(ctx, hf):
    """8 of the benchmark's strings (40 MB): the grammar the benchmark post-processes, in part."""
    coll = li.bacterial_collection().subset(range(8))
    check(ctx, ctx.build(coll.data, coll.offsets), O.build(coll, hf).export())


def test_merged_grammar(ctx, hf):
    coll = li.tiny_dna_collection(base_len=200_000, k=6)
    A, B = coll.subset(range(0, 3)), coll.subset(range(3, 6))
    ga, gb = ctx.build(A.data, A.offsets), ctx.build(B.data, B.offsets)
    ctx.merge(ga, gb)
    check(ctx, ga, O.build(A, hf).merge(O.build(B, hf)).export())


def test_only_single_bytes(ctx, hf):
    coll = li.from_strings([b"x", b"y", b"x"])
    got = check(ctx, ctx.build(coll.data, coll.offsets), O.build(coll, hf).export())
    assert got["c"].tolist() == [ord("x"), ord("y"), ord("x")] and got["kind"].shape[0] == 0
