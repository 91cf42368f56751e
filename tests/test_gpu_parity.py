"""Parity of the CUDA path with the oracle, through the C ABI.

Every comparison is exact: the grammar is integer data (ranks, offsets,
fingerprints), so the GPU export must equal the oracle's byte for byte.
"""
import numpy as np
import pytest

import lcg_inputs as li
from oracle import oracle as O

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx(hf):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2411_12439_gb300 import Context
    return Context(hf, device=0)


def first_difference(got, want):
    if not np.array_equal(got["F0"], want["F0"]):
        return "F0"
    if len(got["levels"]) != len(want["levels"]):
        return f"levels {len(got['levels'])} != {len(want['levels'])}"
    for i, (a, b) in enumerate(zip(got["levels"], want["levels"]), start=1):
        if a["g"] != b["g"]:
            return f"level {i}: g {a['g']} != {b['g']}"
        for key in ("rhs_off", "rhs", "F"):
            x, y = np.asarray(a[key]), np.asarray(b[key])
            if x.shape != y.shape:
                return f"level {i}: {key} shape {x.shape} != {y.shape}"
            bad = np.nonzero(x != y)[0]
            if bad.size:
                return f"level {i}: {key}[{bad[0]}] {x[bad[0]]} != {y[bad[0]]} ({bad.size} differ)"
    for key in ("c_level", "c_rank"):
        bad = np.nonzero(got[key] != want[key])[0]
        if bad.size:
            return f"{key}[{bad[0]}] {got[key][bad[0]]} != {want[key][bad[0]]}"
    return None


def assert_same(got, want):
    diff = first_difference(got, want)
    assert diff is None, diff


def check_build(ctx, hf, coll, device_input=True):
    import torch
    data = torch.from_numpy(coll.data).to("cuda:0") if device_input else coll.data
    g = ctx.build(data, coll.offsets)
    assert_same(g.export(), O.build(coll, hf).export())
    return g


def test_tiny_and_edge_cases(ctx, hf):
    check_build(ctx, hf, li.edge_collection())
    check_build(ctx, hf, li.from_strings([b"agtagtagtgtagtaggagatcggag", b"agtagtagtgtagtaggtcag"]))
    check_build(ctx, hf, li.from_strings([b"A"]))
    check_build(ctx, hf, li.from_strings([b"AC", b"G", b"TT"]))


def test_random_small_collections(ctx, hf):
    rng = np.random.default_rng(1)
    for _ in range(20):
        k = int(rng.integers(1, 12))
        strings = [li.random_dna(rng, int(rng.integers(1, 3000))).tobytes() for _ in range(k)]
        check_build(ctx, hf, li.from_strings(strings), device_input=bool(rng.integers(0, 2)))


def test_tiles_and_ragged_tails(ctx, hf):
    """Strings spanning several 8192-position tiles, with ragged ends and
    string boundaries inside bitmap words."""
    rng = np.random.default_rng(2)
    lens = [8192, 8191, 8193, 40000, 33, 31, 2, 70001, 16384 * 3 + 5]
    coll = li.from_strings([li.random_dna(rng, n) for n in lens])
    check_build(ctx, hf, coll)


def test_runs_longer_than_tiles(ctx, hf):
    rng = np.random.default_rng(3)
    s1 = li.random_dna(rng, 5000).tobytes() + b"N" * 100_000 + li.random_dna(rng, 5000).tobytes()
    s2 = b"N" * 50_000
    s3 = b"A" * 20_000 + b"C" + b"A" * 20_000
    s4 = (b"AC" * 30_000) + b"G" * 9000
    check_build(ctx, hf, li.from_strings([s1, s2, s3, s4]))


@pytest.mark.parametrize("tp", [1024, 2048, 4096])
def test_every_parse_tile(hf, tp):
    """Every parse tile size (lcg_tuning.parse_tile) gives the oracle's
    grammar: ragged tiles, string starts inside tiles, runs over many tiles,
    text with long phrases, many short strings; as launches, from a plan and
    as a CUDA graph launch."""
    import torch
    from paper_2411_12439_gb300 import Context
    ctx = Context(hf, device=0)
    ctx.set_tuning(parse_tile=tp, parse_tile_min=0)  # every round at tp, however short
    assert ctx.tuning()["parse_tile"] == tp
    rng = np.random.default_rng(tp)
    lens = [tp, tp - 1, tp + 1, 5 * tp + 3, 33, 31, 2, 1, 70001]
    check_build(ctx, hf, li.from_strings([li.random_dna(rng, n) for n in lens]))
    check_build(ctx, hf, li.edge_collection())
    s1 = li.random_dna(rng, 3000).tobytes() + b"N" * 60_000 + li.random_dna(rng, 3000).tobytes()
    check_build(ctx, hf, li.from_strings([s1, b"A" * 9000 + b"C" + b"A" * 9000, li.zipf_text(rng, 80_000)]))
    check_build(ctx, hf, li.from_strings([li.random_dna(rng, int(rng.integers(1, 400))) for _ in range(600)]))
    coll = li.tiny_dna_collection(seed=tp, base_len=300_000, k=4)
    want = O.build(coll, hf).export()
    d = torch.from_numpy(coll.data).cuda()
    ctx.build(d, coll.offsets).free()
    g = ctx.build(d, coll.offsets)  # planned rounds
    assert ctx.last_build_stats()["async_rounds"] > 0
    assert_same(g.export(), want)
    g.free()
    ctx.set_graph(True)
    try:
        for _ in range(2):
            g = ctx.build(d, coll.offsets)
            assert_same(g.export(), want)
            g.free()
        assert ctx.last_build_stats()["graph"] == 2
    finally:
        ctx.set_graph(False)


def test_text_bytes(ctx, hf):
    rng = np.random.default_rng(4)
    coll = li.from_strings([li.zipf_text(rng, 200_000), li.zipf_text(rng, 50_000, copy_frac=0.0),
                            bytes(range(256)) * 40])
    check_build(ctx, hf, coll)


@pytest.mark.parametrize("m_bits", [2, 8])
def test_colliding_fingerprints(m_bits):
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2411_12439_gb300 import Context
    hf = li.hash_family(m_bits=m_bits)
    ctx = Context(hf, device=0)
    rng = np.random.default_rng(m_bits)
    coll = li.from_strings([li.random_dna(rng, int(rng.integers(1, 5000))) for _ in range(10)])
    g = check_build(ctx, hf, coll)
    for j in range(coll.k):
        assert g.decompress(j) == coll.string(j).tobytes()


def test_dna_variants_full(ctx, hf):
    """8 variants of a 1 Mbp genome (0.1% SNPs, 0.01% indels), one call."""
    check_build(ctx, hf, li.tiny_dna_collection())


def test_decompress_roundtrip(ctx, hf):
    import torch
    coll = li.tiny_dna_collection(base_len=200_000, k=3)
    g = ctx.build(coll.data, coll.offsets)
    for j in range(coll.k):
        assert g.decompress(j) == coll.string(j).tobytes()
        out = torch.zeros(coll.string(j).shape[0], dtype=torch.uint8, device="cuda:0")
        n = g.decompress(j, out)
        assert n == out.numel() and bytes(out.cpu().numpy()) == coll.string(j).tobytes()


def test_merge_matches_oracle_and_union(ctx, hf):
    coll = li.tiny_dna_collection(base_len=100_000, k=6)
    A, B = coll.subset(range(0, 3)), coll.subset(range(3, 6))
    ga = ctx.build(A.data, A.offsets)
    gb = ctx.build(B.data, B.offsets)
    ctx.merge(ga, gb)
    oa = O.build(A, hf).merge(O.build(B, hf)).export()
    got = ga.export()
    assert_same(got, oa)
    assert_same(got, O.build(coll, hf).export())


def test_build_into_resident(ctx, hf):
    coll = li.tiny_dna_collection(base_len=100_000, k=6)
    R = ctx.build(coll.subset([0, 1]).data, coll.subset([0, 1]).offsets)
    rest = coll.subset(range(2, 6))
    ctx.build_into(R, rest.data, rest.offsets)
    assert_same(R.export(), O.build(coll, hf).export())
    # a second request on the same resident grammar
    again = coll.subset([5, 0])
    ctx.build_into(R, again.data, again.offsets)
    want = O.build(coll, hf).merge(O.build(again, hf)).export()
    assert_same(R.export(), want)


def test_bacterial_batch_full_size(ctx, hf):
    """The benchmark's workload: 64 strings of ~5 Mbp (4 base genomes, 1% SNPs,
    0.02% indels, 5 rearrangements), all in one batched build; then, as the
    benchmark times it, later builds of the same shape as a captured CUDA
    graph and its launches."""
    import torch
    coll = li.bacterial_collection()
    want = O.build(coll, hf).export()
    d = torch.from_numpy(coll.data).to("cuda:0")
    g = ctx.build(d, coll.offsets)
    assert_same(g.export(), want)
    g.free()
    ctx.set_graph(True)
    modes = []
    try:
        for _ in range(3):
            g = ctx.build(d, coll.offsets)
            modes.append(ctx.last_build_stats()["graph"])
            assert_same(g.export(), want)
            g.free()
    finally:
        ctx.set_graph(False)
    assert 2 in modes, modes  # at least one build was a launch of the captured graph


def test_repeated_builds_on_one_context(hf):
    """A context's second build enqueues all rounds without host syncs, sized
    from the first build; when the data differ the planned rounds are too many,
    too few or too small, and the build must still equal the oracle."""
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2411_12439_gb300 import Context
    ctx = Context(hf, device=0)
    small = li.tiny_dna_collection(base_len=20_000, k=3)
    big = li.tiny_dna_collection(base_len=300_000, k=5, snp=1e-2)
    rng = np.random.default_rng(8)
    text = li.from_strings([li.zipf_text(rng, 150_000), li.zipf_text(rng, 90_000)])
    seen = []
    for coll in (big, big, small, big, text, text, small, small):
        check_build(ctx, hf, coll)
        st = ctx.last_build_stats()
        seen.append((st["async_rounds"], st["redone"]))
    # the first build has no plan; a repeat of the same collection fits its plan
    assert seen[0] == (0, False)
    assert seen[1][0] > 0 and not seen[1][1]
    assert seen[5][0] > 0 and not seen[5][1]
