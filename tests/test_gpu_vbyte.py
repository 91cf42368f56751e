"""GPU parity of the VByte codec and of the VByte form of a grammar (Sec. 4,
resource usage) with the oracle (oracle/vbyte.py): byte for byte on the
encode side, value for value on the decode side, across several tiles, ragged
tails, unaligned buffers and every value length; malformed streams and
buffers give LCG_EINVAL."""
import numpy as np
import pytest

import lcg_inputs as li
from oracle import oracle as O
from oracle import vbyte as V

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
from paper_2411_12439_gb300 import Context, LCGError  # noqa: E402

EINVAL, EMISMATCH = -1, -4


@pytest.fixture(scope="module")
def ctx():
    return Context(li.hash_family(), device=0)


def _values(n, seed):
    """Values of every VByte length, with the boundaries of each length."""
    rng = np.random.default_rng(seed)
    v = rng.integers(0, 1 << 32, size=n, dtype=np.uint64) >> rng.integers(0, 32, size=n).astype(np.uint64)
    edges = [0, 1, 127, 128, 16383, 16384, (1 << 21) - 1, 1 << 21, (1 << 28) - 1, 1 << 28, (1 << 32) - 1]
    if n:
        at = rng.integers(0, n, size=min(n, 64))
        v[at] = np.array(edges * 6, dtype=np.uint64)[:at.size]
    return v.astype(np.uint32)


def _dev(v):
    return torch.from_numpy(v.view(np.int32)).cuda()


@pytest.mark.parametrize("n", [1, 7, 2047, 2048, 2049, 4096 * 3 + 5, 250_001])
def test_encode_decode_match_oracle(ctx, n):
    v = _values(n, n)
    want = V.encode_np(v)
    got = ctx.vbyte_encode(_dev(v)).cpu().numpy().tobytes()
    assert got == want
    stream = torch.from_numpy(np.frombuffer(want, dtype=np.uint8).copy()).cuda()
    back = ctx.vbyte_decode(stream, n).cpu().numpy().view(np.uint32)
    assert np.array_equal(back, v)


@pytest.mark.parametrize("shift", [1, 2, 3, 5])
def test_unaligned_buffers(ctx, shift):
    v = _values(9000, 100 + shift)
    want = V.encode_np(v)
    big = torch.zeros(len(want) + 64, dtype=torch.uint8, device="cuda")
    got = ctx.vbyte_encode(_dev(v), out=big[shift:])
    assert got.cpu().numpy().tobytes() == want
    assert int(big[:shift].sum()) == 0 and int(big[shift + len(want):].sum()) == 0  # nothing outside the stream
    src = torch.zeros(len(want) + 16, dtype=torch.uint8, device="cuda")
    src[shift:shift + len(want)] = torch.from_numpy(np.frombuffer(want, dtype=np.uint8).copy()).cuda()
    back = ctx.vbyte_decode(src[shift:shift + len(want)], v.size).cpu().numpy().view(np.uint32)
    assert np.array_equal(back, v)


def test_empty(ctx):
    assert ctx.vbyte_encode(torch.zeros(0, dtype=torch.int32, device="cuda")).numel() == 0
    assert ctx.vbyte_decode(torch.zeros(0, dtype=torch.uint8, device="cuda"), 0).numel() == 0


@pytest.mark.parametrize("bad,n", [
    ("80", 1),                      # ends inside a value
    ("0180", 2),                    # ends inside its second value
    ("ffffffff10", 1),              # five bytes, more than 32 bits
    ("808080808001", 1),            # six bytes
    ("010203", 2),                  # three values, two expected
    ("0102", 3),                    # fewer bytes than values (host check)
])
def test_decode_rejects_malformed(ctx, bad, n):
    buf = torch.from_numpy(np.frombuffer(bytes.fromhex(bad), dtype=np.uint8).copy()).cuda()
    with pytest.raises(LCGError) as e:
        ctx.vbyte_decode(buf, n)
    assert e.value.code == EINVAL


def test_decode_rejects_damage_in_a_long_stream(ctx):
    v = _values(20000, 3)
    want = bytearray(V.encode_np(v))
    want[len(want) // 2] |= 0x80  # two values become one: one value short
    with pytest.raises(LCGError):
        ctx.vbyte_decode(torch.from_numpy(np.frombuffer(bytes(want), dtype=np.uint8).copy()).cuda(), v.size)
    # the context stays usable
    ok = ctx.vbyte_encode(_dev(v)).cpu().numpy().tobytes()
    assert ok == V.encode_np(v)


def _collections():
    rng = np.random.default_rng(17)
    text = [bytes(rng.integers(32, 127, 3000, dtype=np.uint8)) * 4, b"x", b"abcabcabcabd" * 300]
    return {
        "dna": li.tiny_dna_collection(base_len=60_000, k=6),
        "text": li.from_strings(text),
    }


@pytest.mark.parametrize("kind", ["dna", "text"])
def test_grammar_form_matches_oracle(ctx, kind):
    hf = li.hash_family()
    coll = _collections()[kind]
    want_ex = O.build(coll, hf).export()
    want = V.export_vbyte(want_ex)
    g = ctx.build(torch.from_numpy(coll.data).cuda(), coll.offsets)
    assert g.vbyte_size() == len(want)
    host = g.export_vbyte()
    assert host.tobytes() == want
    dev = g.export_vbyte(device=True)
    assert dev.cpu().numpy().tobytes() == want
    for buf in (host, dev):
        h = ctx.import_vbyte(buf)
        assert O.grammars_equal(h.export(), want_ex)
        for j in range(coll.k):
            assert h.decompress(j) == coll.string(j).tobytes()
        h.free()
    g.free()


def test_grammar_form_of_benchmark_strings(ctx):
    """4 of the benchmark's strings (~20 MB): ranks up to millions (3- and
    4-byte VBytes), many tiles per level."""
    hf = li.hash_family()
    coll = li.bacterial_collection().subset(range(4))
    want_ex = O.build(coll, hf).export()
    want = V.export_vbyte(want_ex)
    g = ctx.build(torch.from_numpy(coll.data).cuda(), coll.offsets)
    got = g.export_vbyte(device=True)
    assert got.cpu().numpy().tobytes() == want
    h = ctx.import_vbyte(got)
    assert O.grammars_equal(h.export(), want_ex)
    h.free()
    g.free()


def test_grammar_without_levels(ctx):
    """Strings of one byte each: no level, only C and F^0."""
    hf = li.hash_family()
    coll = li.from_strings([b"A", b"C", b"\x00"])
    want_ex = O.build(coll, hf).export()
    want = V.export_vbyte(want_ex)
    g = ctx.build(torch.from_numpy(coll.data).cuda(), coll.offsets)
    assert g.export_vbyte().tobytes() == want
    h = ctx.import_vbyte(np.frombuffer(want, dtype=np.uint8).copy())
    assert O.grammars_equal(h.export(), want_ex)
    h.free()
    g.free()


def test_import_rejects_damage(ctx):
    hf = li.hash_family()
    coll = _collections()["dna"]
    want = bytearray(V.export_vbyte(O.build(coll, hf).export()))
    nl = int(np.frombuffer(bytes(want[16:24]), dtype=np.uint64)[0])
    first_stream = 24 + 32 * nl

    def expect(buf, code):
        with pytest.raises(LCGError) as e:
            ctx.import_vbyte(np.frombuffer(bytes(buf), dtype=np.uint8).copy())
        assert e.value.code == code

    bad = bytearray(want)
    bad[0] ^= 1
    expect(bad, EINVAL)                       # magic
    expect(want[:-8], EINVAL)                 # truncated
    bad = bytearray(want)
    bad[first_stream] = 0
    expect(bad, EINVAL)                       # an empty rule
    bad = bytearray(want)
    bad[first_stream] ^= 0x01                 # a rule length off by one: the lengths miss G
    expect(bad, EINVAL)
    bad = bytearray(want)
    Fpos = first_stream + 8 * ((int(np.frombuffer(bytes(want[24 + 16:24 + 24]), dtype=np.uint64)[0]) + 7) // 8) \
        + 8 * ((int(np.frombuffer(bytes(want[24 + 24:24 + 32]), dtype=np.uint64)[0]) + 7) // 8)
    bad[Fpos] ^= 0x01                         # a fingerprint of level 1
    expect(bad, EMISMATCH)
    # a grammar of another hash family
    other = Context(li.hash_family(seed=99), device=0)
    with pytest.raises(LCGError) as e:
        other.import_vbyte(np.frombuffer(bytes(want), dtype=np.uint8).copy())
    assert e.value.code == EMISMATCH
    other.close()
    # still usable
    h = ctx.import_vbyte(np.frombuffer(bytes(want), dtype=np.uint8).copy())
    h.free()
