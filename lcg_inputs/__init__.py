"""Seeded synthetic inputs shared by the oracle, the tests and the benchmark.

This module holds no arithmetic of the grammar method itself: it only draws
random numbers and builds byte strings.  Two kinds of input live here:

* the random parameters of the hash family H = {h^0, ..., h^l} (Sec. 3.2: the
  method draws a_i, b_i, c_i uniformly from [p]_+ for a prime p).  The method's
  random draws are inputs to both implementations, so they are generated once
  here and passed to each side;
* synthetic string collections with the shapes of the paper's workloads
  (bacterial/human DNA over {A,C,G,T,N}, byte text), standing in for the
  ATB / HUM / COVID / KERNEL datasets of Sec. 4, which are not available.

Every generator is seeded (numpy PCG64 for the strings, splitmix64 for the hash
parameters) and returns a ``Collection``: one flat uint8 array plus uint64
offsets, string j being ``data[off[j]:off[j+1]]``.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

# Prime modulus used for every level (2^61 - 1).  The paper draws a random
# prime p_i > m_{i-1} per level (Sec. 3.2); this build fixes the Mersenne prime
# 2^61-1 > 2^32 >= m for all levels.
MERSENNE61 = (1 << 61) - 1
DEFAULT_SEED = 0x4C4347  # "LCG"
_MASK64 = (1 << 64) - 1
_GOLDEN = 0x9E3779B97F4A7C15

DNA = np.frombuffer(b"ACGT", dtype=np.uint8)
_COMP = np.zeros(256, dtype=np.uint8)
for _x, _y in zip(b"ACGTN", b"TGCAN"):
    _COMP[_x] = _y
_BASE_INDEX = np.zeros(256, dtype=np.uint8)
for _i, _x in enumerate(b"ACGT"):
    _BASE_INDEX[_x] = _i


# --------------------------------------------------------------------------
# hash-family parameters
# --------------------------------------------------------------------------

def splitmix64_stream(seed: int, count: int) -> list[int]:
    """``count`` outputs of Vigna's splitmix64 generator started at ``seed``."""
    x = seed & _MASK64
    out = []
    for _ in range(count):
        x = (x + _GOLDEN) & _MASK64
        z = x
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _MASK64
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _MASK64
        out.append(z ^ (z >> 31))
    return out


@dataclasses.dataclass(frozen=True)
class HashFamily:
    """Random parameters (a_i, b_i, c_i), i = 0..levels-1, and m = 2^m_bits.

    Level 0 uses (a_0, b_0) for the terminal hash; level i >= 1 uses
    (a_i, b_i, c_i).  All values lie in [1, p-1] with p = 2^61-1.
    """
    a: np.ndarray
    b: np.ndarray
    c: np.ndarray
    m_bits: int
    seed: int

    @property
    def levels(self) -> int:
        return int(self.a.shape[0])


def hash_family(seed: int = DEFAULT_SEED, levels: int = 64, m_bits: int = 32) -> HashFamily:
    """Draw the parameters of H.  Level i takes the first three splitmix64
    outputs (rejecting values that reduce to 0 mod p) of the stream seeded with
    seed XOR (i * 0x9E3779B97F4A7C15)."""
    if not 1 <= m_bits <= 32:
        raise ValueError("m_bits must be in [1, 32]")
    if levels < 1:
        raise ValueError("levels must be >= 1")
    a = np.zeros(levels, dtype=np.uint64)
    b = np.zeros(levels, dtype=np.uint64)
    c = np.zeros(levels, dtype=np.uint64)
    for i in range(levels):
        stream = splitmix64_stream(seed ^ ((i * _GOLDEN) & _MASK64), 16)
        vals = [v % MERSENNE61 for v in stream if v % MERSENNE61 != 0][:3]
        a[i], b[i], c[i] = vals
    return HashFamily(a=a, b=b, c=c, m_bits=m_bits, seed=seed)


# --------------------------------------------------------------------------
# collections
# --------------------------------------------------------------------------

@dataclasses.dataclass
class Collection:
    data: np.ndarray      # uint8, all strings concatenated
    offsets: np.ndarray   # uint64, k+1 entries
    name: str = ""

    @property
    def k(self) -> int:
        return int(self.offsets.shape[0] - 1)

    @property
    def n(self) -> int:
        return int(self.offsets[-1])

    def string(self, j: int) -> np.ndarray:
        return self.data[int(self.offsets[j]):int(self.offsets[j + 1])]

    def subset(self, idx) -> "Collection":
        return from_strings([self.string(int(j)) for j in idx], name=f"{self.name}[subset]")


def from_strings(strings, name: str = "") -> Collection:
    arrs = [np.frombuffer(s, dtype=np.uint8) if isinstance(s, (bytes, bytearray)) else np.asarray(s, dtype=np.uint8)
            for s in strings]
    lens = np.array([a.shape[0] for a in arrs], dtype=np.uint64)
    off = np.zeros(len(arrs) + 1, dtype=np.uint64)
    np.cumsum(lens, out=off[1:])
    data = np.concatenate(arrs) if arrs else np.zeros(0, dtype=np.uint8)
    return Collection(data=np.ascontiguousarray(data, dtype=np.uint8), offsets=off, name=name)


def random_dna(rng: np.random.Generator, n: int) -> np.ndarray:
    return DNA[rng.integers(0, 4, size=n, dtype=np.uint8)]


def apply_snps(rng, seq: np.ndarray, rate: float, protect_n: bool = True) -> np.ndarray:
    """Replace about ``rate * len`` uniformly chosen positions by a different
    base (N positions are left untouched when ``protect_n``)."""
    seq = seq.copy()
    cnt = int(round(rate * seq.shape[0]))
    if cnt == 0 or seq.shape[0] == 0:
        return seq
    pos = rng.integers(0, seq.shape[0], size=cnt)
    if protect_n:
        pos = pos[seq[pos] != ord("N")]
    shift = rng.integers(1, 4, size=pos.shape[0], dtype=np.uint8)
    seq[pos] = DNA[(_BASE_INDEX[seq[pos]] + shift) % 4]
    return seq


def apply_indels(rng, seq: np.ndarray, rate: float, max_len: int) -> np.ndarray:
    """About ``rate * len`` indels, half insertions of random bases and half
    deletions, each of length U[1, max_len]."""
    cnt = int(round(rate * seq.shape[0]))
    if cnt == 0 or seq.shape[0] < 2:
        return seq.copy()
    pos = np.sort(rng.integers(0, seq.shape[0], size=cnt))
    lens = rng.integers(1, max_len + 1, size=cnt)
    ins = rng.integers(0, 2, size=cnt).astype(bool)
    pieces = []
    cur = 0
    for p, ln, is_ins in zip(pos.tolist(), lens.tolist(), ins.tolist()):
        if p < cur:
            continue
        pieces.append(seq[cur:p])
        if is_ins:
            pieces.append(random_dna(rng, ln))
            cur = p
        else:
            cur = min(seq.shape[0], p + ln)
    pieces.append(seq[cur:])
    out = np.concatenate(pieces)
    if out.shape[0] == 0:
        out = random_dna(rng, 1)
    return out


def revcomp(seq: np.ndarray) -> np.ndarray:
    return _COMP[seq[::-1]]


def apply_rearrangements(rng, seq: np.ndarray, count: int, bmin: int, bmax: int) -> np.ndarray:
    """``count`` block rearrangements, alternating a transposition (a block of
    U[bmin, bmax] bases moved elsewhere) and an inversion (the block replaced by
    its reverse complement)."""
    seq = seq.copy()
    for r in range(count):
        n = seq.shape[0]
        bl = int(rng.integers(bmin, bmax + 1))
        if bl >= n:
            continue
        s = int(rng.integers(0, n - bl))
        block = seq[s:s + bl].copy()
        if r % 2 == 0:
            rest = np.concatenate([seq[:s], seq[s + bl:]])
            t = int(rng.integers(0, rest.shape[0] + 1))
            seq = np.concatenate([rest[:t], block, rest[t:]])
        else:
            seq[s:s + bl] = revcomp(block)
    return seq


def tiny_dna_collection(seed: int = 1, base_len: int = 1_000_000, k: int = 8,
                        snp: float = 1e-3, indel: float = 1e-4, indel_max: int = 20) -> Collection:
    """Plain-method collection: k variants of one uniform random base, each with
    ``snp`` SNPs and ``indel`` indels of U[1, indel_max] bp."""
    rng = np.random.Generator(np.random.PCG64(seed))
    base = random_dna(rng, base_len)
    strings = []
    for _ in range(k):
        s = apply_snps(rng, base, snp)
        s = apply_indels(rng, s, indel, indel_max)
        strings.append(s)
    return from_strings(strings, name=f"dna-variants k={k} base={base_len}")


def bacterial_collection(seed: int = 2, n_bases: int = 4, per_base: int = 16, base_len: int = 5_000_000,
                         snp: float = 1e-2, indel: float = 2e-4, indel_max: int = 50,
                         rearr: int = 5, block_min: int = 10_000, block_max: int = 100_000) -> Collection:
    """Bacterial-like batch: ``n_bases`` random genomes, ``per_base`` variants of
    each with SNPs, indels and block rearrangements.  Strings are ordered
    round-robin over the bases."""
    rng = np.random.Generator(np.random.PCG64(seed))
    bases = [random_dna(rng, base_len) for _ in range(n_bases)]
    strings = []
    for v in range(per_base):
        for b in range(n_bases):
            s = apply_snps(rng, bases[b], snp)
            s = apply_indels(rng, s, indel, indel_max)
            s = apply_rearrangements(rng, s, rearr, min(block_min, base_len // 10 + 1),
                                     min(block_max, base_len // 5 + 1))
            strings.append(s)
    return from_strings(strings, name=f"bacterial {n_bases}x{per_base}x{base_len}")


def uneven_collection(seed: int = 3, k: int = 2000, n_bases: int = 50, base_len: int = 12_000_000,
                      total: float = 8e9, len_min: float = 5e5, len_max: float = 12e6) -> Collection:
    """Uneven batch: lognormal lengths clipped to [len_min, len_max] and rescaled
    so that the sum is about ``total``; each string is a window of one of
    ``n_bases`` random genomes with divergence U[0.5%, 3%] (SNPs, and indels at
    1/20 of that rate of length U[1, 50])."""
    rng = np.random.Generator(np.random.PCG64(seed))
    bases = [random_dna(rng, base_len) for _ in range(n_bases)]
    lens = rng.lognormal(mean=math.log(3.5e6), sigma=0.6, size=k)
    lens = np.clip(lens, len_min, len_max)
    lens = np.clip(lens * (total / lens.sum()), len_min, min(len_max, base_len))
    strings = []
    for j in range(k):
        ln = int(lens[j])
        b = int(rng.integers(0, n_bases))
        s0 = int(rng.integers(0, base_len - ln + 1))
        div = float(rng.uniform(0.005, 0.03))
        s = apply_snps(rng, bases[b][s0:s0 + ln], div)
        s = apply_indels(rng, s, div / 20, 50)
        strings.append(s)
    return from_strings(strings, name=f"uneven k={k} total={total:.3g}")


def repetitive_collection(seed: int = 4, k: int = 4, length: int = 3_100_000_000, families: int = 10,
                          copies: int = 1_000_000, cons_min: int = 300, cons_max: int = 6000,
                          n_fraction: float = 0.01, n_run_max: int = 50_000, snp: float = 1e-3) -> Collection:
    """Large repetitive strings over {A,C,G,T,N}: a random base seeded with
    ``copies`` mutated fragments of ``families`` repeat consensus sequences
    (log-spaced lengths, 10-20% divergence, weight ~ 1/length), plus N-runs of
    log-uniform length in [1, n_run_max] covering about ``n_fraction`` of the
    string.  Strings 2..k are string 1 with ``snp`` SNPs over ACGT."""
    rng = np.random.Generator(np.random.PCG64(seed))
    base = random_dna(rng, length)
    cons_lens = np.unique(np.round(np.geomspace(cons_min, cons_max, families)).astype(np.int64))
    cons = [random_dna(rng, int(c)) for c in cons_lens]
    w = 1.0 / cons_lens.astype(np.float64)
    w /= w.sum()
    fam = rng.choice(len(cons), size=copies, p=w)
    starts = rng.integers(0, max(1, length - cons_max), size=copies)
    for f, st in zip(fam.tolist(), starts.tolist()):
        c = cons[f]
        fl = int(rng.integers(min(100, c.shape[0]), c.shape[0] + 1))
        fs = int(rng.integers(0, c.shape[0] - fl + 1))
        frag = c[fs:fs + fl].copy()
        div = float(rng.uniform(0.10, 0.20))
        m = rng.random(fl) < div
        frag[m] = DNA[rng.integers(0, 4, size=int(m.sum()))]
        base[st:st + fl] = frag
    covered = 0
    target = int(n_fraction * length)
    while covered < target:
        rl = int(math.exp(rng.uniform(0.0, math.log(n_run_max))))
        st = int(rng.integers(0, length - rl))
        base[st:st + rl] = ord("N")
        covered += rl
    strings = [base] + [apply_snps(rng, base, snp, protect_n=True) for _ in range(k - 1)]
    return from_strings(strings, name=f"repetitive k={k} len={length}")


def zipf_text(rng: np.random.Generator, n: int, s: float = 1.1, copy_frac: float = 0.3,
              pool: np.ndarray | None = None) -> np.ndarray:
    """Byte text: i.i.d. Zipf(s) over 256 symbols, with about ``copy_frac`` of
    the bytes overwritten by copies of 1-64 KB blocks taken from earlier in the
    same string or from ``pool``."""
    ranks = np.arange(1, 257, dtype=np.float64)
    p = ranks ** (-s)
    p /= p.sum()
    perm = rng.permutation(256).astype(np.uint8)
    t = perm[rng.choice(256, size=n, p=p)]
    copied = 0
    target = int(copy_frac * n)
    while copied < target and n > 2048:
        bl = int(rng.integers(1024, min(65536, n // 2) + 1))
        dst = int(rng.integers(bl, n - bl + 1)) if n - bl >= bl else 0
        if pool is not None and rng.random() < 0.5 and pool.shape[0] > bl:
            src = int(rng.integers(0, pool.shape[0] - bl))
            t[dst:dst + bl] = pool[src:src + bl]
        else:
            src = int(rng.integers(0, max(1, dst - bl + 1)))
            t[dst:dst + bl] = t[src:src + bl]
        copied += bl
    return t


@dataclasses.dataclass
class Request:
    arrival_s: float
    data: np.ndarray
    kind: str


def serving_stream(seed: int = 5, count: int = 2000, rate_hz: float = 100.0, n_bases: int = 100,
                   base_len: int = 50_000_000, len_min: int = 10_000, len_max: int = 50_000_000,
                   dna_frac: float = 0.8):
    """Poisson arrivals of strings with lognormal lengths clipped to
    [len_min, len_max] (median 1 Mbp, sigma 1.5); ``dna_frac`` of them are
    windows of seeded random genomes with 0.1-1% SNPs, the rest Zipf byte text
    with copied blocks.  Returns a list of ``Request``."""
    rng = np.random.Generator(np.random.PCG64(seed))
    pool = zipf_text(rng, min(4 * 1024 * 1024, 4 * len_max), copy_frac=0.0)
    bases = {}
    t = 0.0
    out = []
    for _ in range(count):
        t += float(rng.exponential(1.0 / rate_hz))
        ln = int(np.clip(rng.lognormal(math.log(1e6), 1.5), len_min, len_max))
        if rng.random() < dna_frac:
            b = int(rng.integers(0, n_bases))
            if b not in bases:
                bases[b] = random_dna(np.random.Generator(np.random.PCG64(seed * 1000 + b)), base_len)
            ln = min(ln, base_len)
            s0 = int(rng.integers(0, base_len - ln + 1))
            s = apply_snps(rng, bases[b][s0:s0 + ln], float(rng.uniform(0.001, 0.01)))
            out.append(Request(t, s, "dna"))
        else:
            out.append(Request(t, zipf_text(rng, ln, pool=pool), "text"))
    return out


def edge_collection(seed: int = 7) -> Collection:
    """Degenerate strings: length 1 and 2, single long runs, alternating
    patterns, strictly increasing / decreasing bytes, and runs at both ends."""
    rng = np.random.Generator(np.random.PCG64(seed))
    strings = [
        b"A", b"AC", b"CA", b"AA", b"N" * 1000, b"ACGT" * 300, b"AC" * 500,
        bytes(range(256)), bytes(range(255, -1, -1)), b"N" * 70 + b"ACGTTGCA" * 20 + b"N" * 90,
        b"\x00\xff" * 64, bytes([7]) * 3, random_dna(rng, 5000).tobytes(),
        b"GATTACA", b"Z",
    ]
    return from_strings(strings, name="edge")
