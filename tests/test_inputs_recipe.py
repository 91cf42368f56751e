"""The seeded synthetic inputs follow their stated recipes (small instances of
each generator): alphabets, sizes, mutation rates, rearrangements that keep
the base composition, the N fraction of the repetitive strings, the serving
stream's arrival process, length range and DNA / text mix, and determinism."""
import numpy as np
import pytest

import lcg_inputs as li


def _rng(seed=0):
    return np.random.Generator(np.random.PCG64(seed))


def test_same_seed_same_bytes():
    a, b = li.bacterial_collection(base_len=50_000, n_bases=2, per_base=2), \
        li.bacterial_collection(base_len=50_000, n_bases=2, per_base=2)
    assert np.array_equal(a.data, b.data) and np.array_equal(a.offsets, b.offsets)
    c = li.bacterial_collection(seed=9, base_len=50_000, n_bases=2, per_base=2)
    assert not np.array_equal(a.data[:1000], c.data[:1000])


def test_snp_rate_and_substitution():
    base = li.random_dna(_rng(1), 200_000)
    s = li.apply_snps(_rng(2), base, 0.01)
    diff = np.count_nonzero(s != base)
    # 2000 draws with replacement: a few collide; every drawn position changes
    assert 1900 <= diff <= 2000
    assert set(np.unique(s).tolist()) <= set(b"ACGT")


def test_snps_leave_n_untouched():
    seq = np.frombuffer(b"N" * 1000 + b"ACGT" * 250, dtype=np.uint8).copy()
    s = li.apply_snps(_rng(3), seq, 0.2)
    assert np.all(s[:1000] == ord("N"))
    assert np.count_nonzero(s[1000:] != seq[1000:]) > 0


def test_indels_change_the_length_by_their_sizes():
    base = li.random_dna(_rng(4), 100_000)
    s = li.apply_indels(_rng(5), base, 2e-4, 50)  # 20 indels of U[1, 50]
    assert abs(s.shape[0] - base.shape[0]) <= 20 * 50
    assert set(np.unique(s).tolist()) <= set(b"ACGT")


def test_rearrangements_keep_length_and_composition():
    base = li.random_dna(_rng(6), 300_000)
    s = li.apply_rearrangements(_rng(7), base, 5, 10_000, 60_000)
    assert s.shape[0] == base.shape[0]
    # transpositions move blocks; inversions complement them: A+T and C+G stay
    count = lambda x, cs: sum(int(np.count_nonzero(x == ord(c))) for c in cs)  # noqa: E731
    assert count(s, "AT") == count(base, "AT") and count(s, "CG") == count(base, "CG")
    assert not np.array_equal(s, base)
    assert np.array_equal(li.revcomp(li.revcomp(base)), base)


def test_bacterial_shape():
    c = li.bacterial_collection(base_len=100_000, n_bases=3, per_base=4)
    assert c.k == 12
    lens = np.diff(c.offsets.astype(np.int64))
    assert np.all(np.abs(lens - 100_000) < 100_000 * 0.05)
    assert set(np.unique(c.data).tolist()) <= set(b"ACGT")


def test_uneven_lengths():
    # the recipe's clip range [0.5, 12] Mbp around the lognormal's median of 3.5 Mbp, 20 strings
    c = li.uneven_collection(k=20, n_bases=2, total=7e7)
    lens = np.diff(c.offsets.astype(np.int64))
    assert c.k == 20
    assert lens.min() >= 5e5 * 0.9 and lens.max() <= 12e6 * 1.05
    assert abs(lens.sum() - 7e7) < 0.1 * 7e7
    assert lens.std() > 0.2 * lens.mean()  # lognormal spread, not equal lengths


def test_repetitive_n_fraction_and_repeats():
    c = li.repetitive_collection(k=2, length=2_000_000, copies=2_000, n_run_max=20_000)
    s0, s1 = c.string(0), c.string(1)
    n_frac = np.count_nonzero(s0 == ord("N")) / s0.shape[0]
    assert 0.005 <= n_frac <= 0.03
    assert set(np.unique(s0).tolist()) <= set(b"ACGTN")
    # string 2 = string 1 with SNPs over ACGT only: the N positions agree
    assert np.array_equal(s0 == ord("N"), s1 == ord("N"))
    assert 0 < np.count_nonzero(s0 != s1) < 0.002 * s0.shape[0]


def test_serving_stream_recipe():
    reqs = li.serving_stream(count=300, rate_hz=50.0, n_bases=4, base_len=3_000_000, len_min=10_000,
                             len_max=2_000_000)
    t = np.array([r.arrival_s for r in reqs])
    assert np.all(np.diff(t) > 0)
    gaps = np.diff(np.concatenate([[0.0], t]))
    assert gaps.mean() == pytest.approx(1 / 50.0, rel=0.25)  # exponential gaps
    lens = np.array([r.data.shape[0] for r in reqs])
    assert lens.min() >= 10_000 and lens.max() <= 2_000_000
    dna = sum(r.kind == "dna" for r in reqs) / len(reqs)
    assert 0.7 <= dna <= 0.9
    for r in reqs:
        if r.kind == "dna":
            assert set(np.unique(r.data).tolist()) <= set(b"ACGT")


def test_zipf_text_is_skewed():
    t = li.zipf_text(_rng(8), 200_000, copy_frac=0.0)
    counts = np.sort(np.bincount(t, minlength=256))[::-1]
    assert counts[0] > 10 * counts[50]  # Zipf(1.1): the top symbol dominates the 51st
