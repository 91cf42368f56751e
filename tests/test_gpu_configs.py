"""Full-size runs of the uneven batch (2000 strings, ~8 GB) and the large
repetitive strings (4 x 3.1 Gbp over ACGTN, ~12.4 GB), each in one batched
build, compared with the oracle's grammar of the same collection in full:
every level's rhs_off, rhs and F, and the roots C, through SHA-256 digests
that tests/golden/make_config_digests.py wrote from the oracle alone (the
grammars are gigabytes; the oracle takes minutes on them).  The second build
of each runs as a launch of its captured CUDA graph, as the benchmark times
it.  The repetitive generator is also checked bit for bit against the oracle
at a size the oracle finishes in seconds."""
import json
import os

import numpy as np
import pytest

import lcg_inputs as li
from oracle import oracle as O
from tests.digests import first_digest_difference, grammar_digests

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "config_digests.json")


@pytest.fixture(scope="module")
def ctx(hf):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2411_12439_gb300 import Context
    return Context(hf, device=0)


def _golden(name):
    with open(GOLDEN) as fh:
        return json.load(fh)[name]


def _expands(g, j, dev_data, off):
    import torch
    n = int(off[j + 1] - off[j])
    out = torch.empty(n, dtype=torch.uint8, device=dev_data.device)
    assert g.decompress(j, out) == n
    return torch.equal(out, dev_data[int(off[j]):int(off[j + 1])])


def _check_full(ctx, coll, want, samples):
    import torch
    assert coll.n == want["n"] and coll.k == want["k"]
    d = torch.from_numpy(coll.data).cuda()
    g = ctx.build(d, coll.offsets)
    diff = first_digest_difference(grammar_digests(g.export()), want)
    assert diff is None, diff
    for j in samples:
        assert _expands(g, j, d, coll.offsets), j
    g.free()
    # again, all rounds enqueued at once from the plan of the build before
    g = ctx.build(d, coll.offsets)
    assert ctx.last_build_stats()["async_rounds"] > 0
    diff = first_digest_difference(grammar_digests(g.export()), want)
    assert diff is None, f"planned rounds: {diff}"
    g.free()
    # the same shape again as one captured CUDA graph, then its launch
    ctx.set_graph(True)
    try:
        modes = []
        for _ in range(2):
            g = ctx.build(d, coll.offsets)
            modes.append(ctx.last_build_stats()["graph"])
            if modes[-1] == 2:
                diff = first_digest_difference(grammar_digests(g.export()), want)
                assert diff is None, f"graph launch: {diff}"
            g.free()
    finally:
        ctx.set_graph(False)
    assert modes[-1] == 2, modes


def test_uneven_batch_8gb(ctx):
    coll = li.uneven_collection()
    rng = np.random.default_rng(0)
    samples = sorted(set(rng.integers(0, coll.k, size=4).tolist()) | {0, coll.k - 1})
    _check_full(ctx, coll, _golden("uneven"), samples)


def test_repetitive_12gb(ctx):
    coll = li.repetitive_collection()
    assert coll.k == 4 and coll.n == 4 * 3_100_000_000
    _check_full(ctx, coll, _golden("repetitive"), range(coll.k))


def test_repetitive_structure_against_oracle(ctx, hf):
    coll = li.repetitive_collection(length=1_500_000, copies=3000, n_run_max=20_000)
    g = ctx.build(coll.data, coll.offsets)
    assert O.grammars_equal(g.export(), O.build(coll, hf).export())
