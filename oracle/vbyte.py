"""VByte form of a grammar: the plain oracle.

TEST INFRASTRUCTURE ONLY: the tests and the benchmark use it; the product
path never imports it.

Sec. 4 (resource usage) proposes VBytes for the grammar's rules and phrase
keys: a symbol takes as many bytes as its value needs instead of a 32-bit
cell, which its preliminary tests found to shrink the sink grammar by 39-47 %.
The paper does not fix the byte layout of a VByte; the reading taken here is
the common one (LEB128, the varint of Protocol Buffers): a value is cut into
groups of 7 bits, least significant group first, one group per byte, and the
high bit of a byte is set when another byte of the same value follows.

Layout of a grammar's VByte form ("LCGV"; little-endian; every section starts
at a multiple of 8 bytes and is zero-padded):
    u64 magic 0x4C434756, u64 k, u64 nlevels,
    per level: u64 g, u64 G, u64 bytes of the lengths, u64 bytes of the symbols;
    per level: VByte of |rhs(X)| for the g rules in rank order,
               VByte of the G right-hand-side symbols, u32 F[g];
    u32 c_level[k], u32 c_rank[k], u32 F0[256].
``encode`` / ``decode`` take one value at a time in plain Python; ``encode_np``
/ ``decode_np`` state the same definition over numpy arrays, one byte
position at a time, and are checked against them.
"""
from __future__ import annotations

import struct

import numpy as np

MAGIC = 0x4C434756  # "LCGV"


def encode(values) -> bytes:
    """VByte of each value (0 <= v < 2^32), concatenated."""
    out = bytearray()
    for v in values:
        v = int(v)
        if v < 0 or v >= 1 << 32:
            raise ValueError("value outside 32 bits")
        while True:
            group = v & 0x7F
            v >>= 7
            if v:
                out.append(group | 0x80)
            else:
                out.append(group)
                break
    return bytes(out)


def encoded_length(v: int) -> int:
    """Bytes of one value's VByte."""
    n = 1
    while v >= 0x80:
        v >>= 7
        n += 1
    return n


def decode(buf: bytes, count: int | None = None) -> list:
    """Values of a VByte stream.  Raises ValueError on a stream that ends
    inside a value, a value of more than 32 bits, or (when ``count`` is given)
    a different number of values."""
    vals = []
    v = 0
    shift = 0
    for b in bytes(buf):
        v |= (b & 0x7F) << shift
        shift += 7
        if v >= 1 << 32 or shift > 35:
            raise ValueError("value of more than 32 bits")
        if not b & 0x80:
            vals.append(v)
            v = 0
            shift = 0
    if shift:
        raise ValueError("stream ends inside a value")
    if count is not None and len(vals) != count:
        raise ValueError(f"{len(vals)} values, expected {count}")
    return vals


def encode_np(values) -> bytes:
    """``encode`` over a numpy array, one byte position at a time: value p
    starts at the sum of the lengths before it, and its byte t holds bits
    7t .. 7t+6, with the high bit set when t is not its last byte."""
    v = np.asarray(values, dtype=np.uint64)
    if v.size and int(v.max()) >= 1 << 32:
        raise ValueError("value outside 32 bits")
    lens = np.ones(v.shape, dtype=np.int64)
    for t in range(1, 5):
        lens += v >= (1 << (7 * t))
    start = np.cumsum(lens) - lens
    out = np.zeros(int(lens.sum()), dtype=np.uint8)
    for t in range(5):
        m = lens > t
        group = (v[m] >> np.uint64(7 * t)) & np.uint64(0x7F)
        more = np.where(lens[m] > t + 1, 0x80, 0).astype(np.uint64)
        out[start[m] + t] = (group | more).astype(np.uint8)
    return out.tobytes()


def decode_np(buf, count: int | None = None) -> np.ndarray:
    """``decode`` over a numpy array: a value ends at every byte without the
    high bit and starts after the previous such byte."""
    b = np.frombuffer(bytes(buf), dtype=np.uint8)
    if b.size == 0:
        vals = np.zeros(0, dtype=np.uint32)
    else:
        if b[-1] & 0x80:
            raise ValueError("stream ends inside a value")
        ends = np.flatnonzero((b & 0x80) == 0)
        starts = np.concatenate(([0], ends[:-1] + 1))
        lens = ends - starts + 1
        if lens.max() > 5:
            raise ValueError("value of more than 32 bits")
        acc = np.zeros(ends.shape, dtype=np.uint64)
        for t in range(5):
            m = lens > t
            acc[m] |= (b[starts[m] + t] & 0x7F).astype(np.uint64) << np.uint64(7 * t)
        if acc.size and int(acc.max()) >= 1 << 32:
            raise ValueError("value of more than 32 bits")
        vals = acc.astype(np.uint32)
    if count is not None and vals.size != count:
        raise ValueError(f"{vals.size} values, expected {count}")
    return vals


def _pad8(b: bytes) -> bytes:
    return b + bytes((-len(b)) % 8)


def export_vbyte(ex: dict) -> bytes:
    """The LCGV form of an exported grammar (the oracle's ``export()`` dict)."""
    levels = ex["levels"]
    k = len(ex["c_level"])
    head = struct.pack("<3Q", MAGIC, k, len(levels))
    body = b""
    for L in levels:
        ro = np.asarray(L["rhs_off"], dtype=np.uint64)
        lens = encode_np(np.diff(ro))
        syms = encode_np(L["rhs"])
        head += struct.pack("<4Q", int(L["g"]), int(ro[-1]), len(lens), len(syms))
        body += _pad8(lens) + _pad8(syms) + _pad8(np.asarray(L["F"], dtype="<u4").tobytes())
    body += _pad8(np.asarray(ex["c_level"], dtype="<u4").tobytes())
    body += _pad8(np.asarray(ex["c_rank"], dtype="<u4").tobytes())
    body += np.asarray(ex["F0"], dtype="<u4").tobytes()
    return head + body


def import_vbyte(buf: bytes) -> dict:
    """The exported-grammar dict of an LCGV buffer (ValueError if malformed)."""
    buf = bytes(buf)
    if len(buf) < 24:
        raise ValueError("short buffer")
    magic, k, nl = struct.unpack_from("<3Q", buf, 0)
    if magic != MAGIC:
        raise ValueError("not an LCGV buffer")
    pos = 24 + 32 * nl
    sizes = [struct.unpack_from("<4Q", buf, 24 + 32 * i) for i in range(nl)]
    levels = []

    def take(n):
        nonlocal pos
        if pos + n > len(buf):
            raise ValueError("truncated")
        s = buf[pos:pos + n]
        pos += n + (-n) % 8
        return s

    for g, G, nb_len, nb_rhs in sizes:
        lens = decode_np(take(nb_len), g)
        syms = decode_np(take(nb_rhs), G)
        F = np.frombuffer(take(4 * g), dtype="<u4").astype(np.uint32)
        if lens.size and int(lens.min()) == 0:
            raise ValueError("empty rule")
        ro = np.zeros(g + 1, dtype=np.uint64)
        np.cumsum(lens, out=ro[1:])
        if int(ro[-1]) != G:
            raise ValueError("rule lengths disagree with G")
        levels.append({"g": g, "rhs_off": ro, "rhs": syms, "F": F})
    c_level = np.frombuffer(take(4 * k), dtype="<u4").astype(np.uint32)
    c_rank = np.frombuffer(take(4 * k), dtype="<u4").astype(np.uint32)
    F0 = np.frombuffer(take(4 * 256), dtype="<u4").astype(np.uint32)
    if pos != len(buf):
        raise ValueError("wrong size")
    return {"F0": F0, "levels": levels, "c_level": c_level, "c_rank": c_rank}
