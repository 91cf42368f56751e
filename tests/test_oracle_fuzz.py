"""Property-based tests of the oracle (hypothesis): collections drawn from
small alphabets, so that runs, repeats and collisions of short phrases are
common.  Properties from the paper: every string expands to itself (Sec. 2.2);
MergeGrams of two parts equals BuildGram of the whole collection under
first-occurrence naming (Sec. 3.6); post-processing (RL, Simp) keeps every
expansion and obeys its size identities; the VByte codec and the VByte form of
a grammar (Sec. 4) give back what they were given."""
import numpy as np
import pytest

hypothesis = pytest.importorskip("hypothesis")
from hypothesis import HealthCheck, given, settings  # noqa: E402
from hypothesis import strategies as st  # noqa: E402

import lcg_inputs as li  # noqa: E402
from oracle import oracle as O  # noqa: E402
from oracle import postprocess as P  # noqa: E402

alphabets = st.sampled_from([b"A", b"AC", b"ACGT", b"ACGTN", bytes(range(256))])


@st.composite
def collections(draw, max_k=6, max_len=400):
    sigma = draw(alphabets)
    k = draw(st.integers(1, max_k))
    out = []
    for _ in range(k):
        n = draw(st.integers(1, max_len))
        idx = draw(st.lists(st.integers(0, len(sigma) - 1), min_size=n, max_size=n))
        out.append(bytes(sigma[i] for i in idx))
    return out


settings_ = settings(max_examples=60, deadline=None, suppress_health_check=[HealthCheck.too_slow])


@settings_
@given(collections())
def test_expansion_is_the_input(strings):
    hf = li.hash_family()
    g = O.build(li.from_strings(strings), hf)
    for j, s in enumerate(strings):
        assert g.decompress(j) == s


@settings_
@given(collections(), st.integers(0, 6))
def test_merge_equals_build_of_the_whole(strings, cut):
    hf = li.hash_family()
    cut = min(cut, len(strings))
    whole = O.build(li.from_strings(strings), hf).export()
    if cut in (0, len(strings)):
        return
    a = O.build(li.from_strings(strings[:cut]), hf)
    b = O.build(li.from_strings(strings[cut:]), hf)
    assert O.grammars_equal(a.merge(b).export(), whole)


@settings_
@given(collections())
def test_postprocess_keeps_expansions(strings):
    hf = li.hash_family()
    ex = O.build(li.from_strings(strings), hf).export()
    pp = P.postprocess(ex)
    for j, s in enumerate(strings):
        assert P.expand_symbol(pp, int(pp["c"][j])) == s
    stt = pp["stats"]
    assert stt["size"] == stt["size_rl"] - stt["removed"]
    assert np.all(pp["rhs_off"][1:] >= pp["rhs_off"][:-1])


@settings_
@given(st.lists(st.integers(0, (1 << 32) - 1), max_size=300))
def test_vbyte_codec_roundtrip(values):
    from oracle import vbyte as V
    buf = V.encode(values)
    assert V.encode_np(np.array(values, dtype=np.uint64)) == buf
    assert len(buf) == sum(V.encoded_length(v) for v in values)
    assert V.decode(buf, len(values)) == values
    assert V.decode_np(buf, len(values)).tolist() == values


@settings_
@given(collections())
def test_vbyte_form_roundtrip(strings):
    from oracle import vbyte as V
    hf = li.hash_family()
    ex = O.build(li.from_strings(strings), hf).export()
    assert O.grammars_equal(V.import_vbyte(V.export_vbyte(ex)), ex)
