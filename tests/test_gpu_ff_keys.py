"""Inputs rich in 0xFF bytes, through every table of the CUDA path.

Phrase tables mark an empty slot with a key whose high word is all ones.  A
phrase of 15 bytes of 0xFF, packed exactly, would have had that very key; the
key layout keeps inline keys to 14 symbols so that no phrase can.  These tests
drive such phrases through the round tables (build), the level tables of a
merge (Sec. 3.6) and of a resident grammar (lcg_build_into), and the serving
loop, and compare each result with the oracle.
"""
import numpy as np
import pytest

import lcg_inputs as li
from oracle import oracle as O

pytestmark = pytest.mark.gpu


def _ff_heavy(rng, n, p_ff=0.7):
    """Bytes that are 0xFF with probability p_ff, else uniform: runs of 0xFF of
    every length, and phrases that start with several 0xFF bytes."""
    x = rng.integers(0, 256, size=n, dtype=np.uint8)
    x[rng.random(n) < p_ff] = 0xFF
    return x


def _strings(seed):
    rng = np.random.default_rng(seed)
    out = [b"\xff" * 15, b"\x01" + b"\xff" * 15 + b"\x01", b"\xff" * 14, b"\xff" * 16, b"\xff" * 31]
    # 15-byte blocks whose first 7 bytes are 0xFF, between separators
    blocks = [b"\xff" * 7 + bytes(rng.integers(0, 256, size=8, dtype=np.uint8).tolist()) for _ in range(200)]
    out.append(b"\x00".join(blocks))
    out.append(b"".join(b + b"\x02\x01" for b in blocks[:50]))
    out.append(_ff_heavy(rng, 1_000_000).tobytes())
    out.append(_ff_heavy(rng, 300_000, p_ff=0.9).tobytes())
    return out


@pytest.fixture(scope="module")
def ctx(hf):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2411_12439_gb300 import Context
    return Context(hf, device=0)


def test_build(ctx, hf):
    coll = li.from_strings(_strings(1))
    g = ctx.build(coll.data, coll.offsets)
    assert O.grammars_equal(g.export(), O.build(coll, hf).export())
    for j in range(coll.k):
        assert g.decompress(j) == coll.string(j).tobytes()
    g.free()


def test_each_string_alone(ctx, hf):
    for s in _strings(2)[:7]:
        coll = li.from_strings([s])
        g = ctx.build(coll.data, coll.offsets)
        assert O.grammars_equal(g.export(), O.build(coll, hf).export()), s[:20]
        g.free()


def test_merge(ctx, hf):
    strings = _strings(3)
    coll = li.from_strings(strings)
    A, B = coll.subset(range(0, 4)), coll.subset(range(4, coll.k))
    ga, gb = ctx.build(A.data, A.offsets), ctx.build(B.data, B.offsets)
    ctx.merge(ga, gb)
    assert O.grammars_equal(ga.export(), O.build(A, hf).merge(O.build(B, hf)).export())
    assert O.grammars_equal(ga.export(), O.build(coll, hf).export())
    # merging the same strings again finds every rule (nothing is appended)
    gc = ctx.build(B.data, B.offsets)
    ctx.merge(ga, gc)
    want = O.build(coll, hf).merge(O.build(B, hf)).export()
    assert O.grammars_equal(ga.export(), want)
    for g in (ga, gb, gc):
        g.free()


def test_build_into_resident(ctx, hf):
    coll = li.from_strings(_strings(4))
    first = coll.subset(range(0, 5))
    R = ctx.build(first.data, first.offsets)
    rest = coll.subset(range(5, coll.k))
    ctx.build_into(R, rest.data, rest.offsets)
    assert O.grammars_equal(R.export(), O.build(coll, hf).export())
    again = coll.subset([0, 7, 1])
    ctx.build_into(R, again.data, again.offsets)
    assert O.grammars_equal(R.export(), O.build(coll, hf).merge(O.build(again, hf)).export())
    R.free()


@pytest.mark.parametrize("mode", ["merge", "resident"])
def test_serving(hf, mode):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2411_12439_gb300 import Context, serving
    strings = _strings(5) + _strings(6)[5:]
    stream = [li.Request(0.001 * i, np.frombuffer(s, dtype=np.uint8).copy(), "ff") for i, s in enumerate(strings)]
    srv = serving.Server(serving.CudaBackend(hf, device=0, lanes=2), lanes=2, max_batch_bytes=1 << 20, mode=mode)
    srv.start()
    reqs = serving.replay(srv, stream)
    assert srv.drain(reqs, timeout=300)
    srv.stop()
    assert not srv.errors, srv.errors
    alone = Context(hf, device=0)
    for r in reqs:
        g = alone.build(r.data, np.array([0, r.n], dtype=np.uint64))
        lv, _, fp = g.roots()
        assert r.result == (int(lv[0]), int(fp[0]))
        g.free()
    order = sorted(reqs, key=lambda r: r.index)
    want = O.build(li.from_strings([r.data for r in order]), hf).export()
    assert O.grammars_equal(srv.resident.export(), want)
