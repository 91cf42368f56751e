"""Full-size runs of the uneven batch (2000 strings, ~8 GB) and the large
repetitive strings (4 x 3.1 Gbp over ACGTN, ~12.4 GB), in one batched build
each, checked where the oracle can follow: the root of a string (its level and
the fingerprint of its expansion) depends on that string only, so sampled
strings are built alone by the oracle and their roots compared; every sampled
string expands to its bytes.  The repetitive generator is also checked bit for
bit against the oracle at a size the oracle finishes in seconds."""
import numpy as np
import pytest

import lcg_inputs as li
from oracle import oracle as O

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


@pytest.fixture(scope="module")
def ctx(hf):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2411_12439_gb300 import Context
    return Context(hf, device=0)


def _oracle_root(hf, s):
    ex = O.build(li.from_strings([s]), hf).export()
    lvl, r = int(ex["c_level"][0]), int(ex["c_rank"][0])
    return lvl, int(ex["F0"][r] if lvl == 0 else ex["levels"][lvl - 1]["F"][r])


def _expands(g, j, dev_data, off):
    import torch
    n = int(off[j + 1] - off[j])
    out = torch.empty(n, dtype=torch.uint8, device=dev_data.device)
    assert g.decompress(j, out) == n
    return torch.equal(out, dev_data[int(off[j]):int(off[j + 1])])


def test_uneven_batch_8gb(ctx, hf):
    import torch
    coll = li.uneven_collection()
    assert coll.k == 2000 and 7.5e9 < coll.n < 8.5e9
    d = torch.from_numpy(coll.data).cuda()
    g = ctx.build(d, coll.offsets)
    lv, _, fp = g.roots()
    rng = np.random.default_rng(0)
    for j in sorted(set(rng.integers(0, coll.k, size=6).tolist()) | {0, coll.k - 1}):
        assert (int(lv[j]), int(fp[j])) == _oracle_root(hf, coll.string(j)), j
        assert _expands(g, j, d, coll.offsets), j
    print("uneven batch: levels", g.shape[1], "packed grammar bytes", g.packed_size())


def test_repetitive_12gb(ctx, hf):
    import torch
    from paper_2411_12439_gb300 import Context
    coll = li.repetitive_collection()
    assert coll.k == 4 and coll.n == 4 * 3_100_000_000
    d = torch.from_numpy(coll.data).cuda()
    g = ctx.build(d, coll.offsets)
    lv, _, fp = g.roots()
    for j in range(coll.k):
        assert _expands(g, j, d, coll.offsets), j
    # each string parsed alone has the same root (the oracle is too slow at 3.1 Gbp)
    alone = Context(hf, device=0)
    for j in range(coll.k):
        sub = d[int(coll.offsets[j]):int(coll.offsets[j + 1])]
        ga = alone.build(sub, np.array([0, sub.numel()], dtype=np.uint64))
        la, _, fa = ga.roots()
        assert (int(la[0]), int(fa[0])) == (int(lv[j]), int(fp[j])), j
        ga.free()


def test_repetitive_structure_against_oracle(ctx, hf):
    coll = li.repetitive_collection(length=1_500_000, copies=3000, n_run_max=20_000)
    g = ctx.build(coll.data, coll.offsets)
    assert O.grammars_equal(g.export(), O.build(coll, hf).export())
