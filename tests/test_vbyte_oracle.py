"""Pins of the VByte oracle (Sec. 4, resource usage: VByte rules and keys).

The byte layout of a VByte is fixed by published examples of the LEB128 /
varint form (tests/golden/vbyte_vectors.json), its lengths by a closed form,
the codec by brute force, and the grammar layout by a hand-worked buffer
(tests/golden/vbyte_layout.json)."""
import json
import math
import os

import numpy as np
import pytest

import lcg_inputs as li
from oracle import oracle as O
from oracle import vbyte as V

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _load(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return json.load(f)


def test_published_vectors():
    for vec in _load("vbyte_vectors.json")["vectors"]:
        want = bytes.fromhex(vec["hex"])
        assert V.encode([vec["value"]]) == want, vec
        assert V.decode(want) == [vec["value"]], vec


def test_lengths_closed_form():
    # a value of b significant bits takes ceil(b / 7) bytes (one for zero)
    vals = [0, 1]
    for t in range(1, 5):
        vals += [(1 << (7 * t)) - 1, 1 << (7 * t)]
    vals += [(1 << 32) - 1]
    for v in vals:
        want = max(1, math.ceil(v.bit_length() / 7))
        assert V.encoded_length(v) == want == len(V.encode([v])), v
    assert V.encode([(1 << 32) - 1]) == bytes.fromhex("ffffffff0f")


def test_roundtrip_brute_and_random():
    vals = list(range(0, 70000))
    rng = np.random.default_rng(5)
    vals += [int(x) for x in rng.integers(0, 1 << 32, size=20000, dtype=np.uint64)]
    vals += [int(x) >> int(s) for x, s in zip(rng.integers(0, 1 << 32, size=5000, dtype=np.uint64),
                                              rng.integers(0, 32, size=5000))]
    buf = V.encode(vals)
    assert len(buf) == sum(V.encoded_length(v) for v in vals)
    assert V.decode(buf, len(vals)) == vals


def test_numpy_forms_equal_loops():
    rng = np.random.default_rng(8)
    for n in [0, 1, 5, 1000, 30000]:
        v = rng.integers(0, 1 << 32, size=n, dtype=np.uint64) >> rng.integers(0, 32, size=n).astype(np.uint64)
        v = v.astype(np.uint32)
        buf = V.encode(v.tolist())
        assert V.encode_np(v) == buf
        assert V.decode_np(buf, n).tolist() == V.decode(buf, n) == v.tolist()
    for vec in _load("vbyte_vectors.json")["vectors"]:
        assert V.encode_np([vec["value"]]) == bytes.fromhex(vec["hex"])


@pytest.mark.parametrize("bad", ["80", "ff", "0180", "ffffffff10", "ffffffffff01", "8080808080800"])
def test_decode_rejects_malformed(bad):
    buf = bytes.fromhex(bad if len(bad) % 2 == 0 else bad + "0")
    with pytest.raises(ValueError):
        V.decode(buf)
    with pytest.raises(ValueError):
        V.decode_np(buf)


def test_decode_rejects_wrong_count():
    with pytest.raises(ValueError):
        V.decode(V.encode([1, 2, 3]), 2)


def _hand_export(fx):
    levels = []
    for L in fx["grammar"]["levels"]:
        lens = [len(r) for r in L["rules"]]
        ro = np.zeros(len(lens) + 1, dtype=np.uint64)
        ro[1:] = np.cumsum(lens)
        levels.append({"g": len(lens), "rhs_off": ro,
                       "rhs": np.array([s for r in L["rules"] for s in r], dtype=np.uint32),
                       "F": np.array(L["F"], dtype=np.uint32)})
    return {"F0": np.arange(256, dtype=np.uint32), "levels": levels,
            "c_level": np.array(fx["grammar"]["c_level"], dtype=np.uint32),
            "c_rank": np.array(fx["grammar"]["c_rank"], dtype=np.uint32)}


def test_layout_hand_example():
    fx = _load("vbyte_layout.json")
    ex = _hand_export(fx)
    buf = V.export_vbyte(ex)
    want = bytes.fromhex(fx["header_hex"].replace(" ", "") + fx["body_hex"].replace(" ", ""))
    assert len(buf) == fx["size"]
    assert buf[:len(want)] == want
    assert buf[len(want):] == np.arange(256, dtype="<u4").tobytes()
    back = V.import_vbyte(buf)
    assert O.grammars_equal(back, ex)


def test_import_rejects_damage():
    ex = _hand_export(_load("vbyte_layout.json"))
    buf = bytearray(V.export_vbyte(ex))
    with pytest.raises(ValueError):
        V.import_vbyte(bytes(buf[:-4]))  # truncated
    bad = bytearray(buf)
    bad[0] ^= 1  # magic
    with pytest.raises(ValueError):
        V.import_vbyte(bytes(bad))
    bad = bytearray(buf)
    bad[24 + 64] = 0  # first rule length 2 -> 0: empty rule
    with pytest.raises(ValueError):
        V.import_vbyte(bytes(bad))
    bad = bytearray(buf)
    bad[24 + 64] = 3  # lengths no longer sum to G
    with pytest.raises(ValueError):
        V.import_vbyte(bytes(bad))


@pytest.mark.parametrize("kind", ["dna", "text"])
def test_grammar_roundtrip_and_size(kind):
    hf = li.hash_family()
    coll = (li.tiny_dna_collection(base_len=30000, k=5) if kind == "dna"
            else li.from_strings([bytes(np.random.default_rng(3).integers(0, 256, 5000, dtype=np.uint8)) * 3]))
    ex = O.build(coll, hf).export()
    buf = V.export_vbyte(ex)
    assert O.grammars_equal(V.import_vbyte(buf), ex)
    # each symbol takes encoded_length(value) bytes, each rule length likewise
    syms = sum(V.encoded_length(int(x)) for L in ex["levels"] for x in L["rhs"])
    lens = sum(V.encoded_length(int(b - a)) for L in ex["levels"]
               for a, b in zip(L["rhs_off"][:-1], L["rhs_off"][1:]))
    words = sum(4 * int(L["rhs_off"][-1]) + 8 * (int(L["g"]) + 1) for L in ex["levels"])
    assert syms + lens < words
