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
Everything here is plain Python / numpy, one value at a time.
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


def _pad8(b: bytes) -> bytes:
    return b + bytes((-len(b)) % 8)


def export_vbyte(ex: dict) -> bytes:
    """The LCGV form of an exported grammar (the oracle's ``export()`` dict)."""
    levels = ex["levels"]
    k = len(ex["c_level"])
    head = struct.pack("<3Q", MAGIC, k, len(levels))
    body = b""
    for L in levels:
        ro = [int(x) for x in L["rhs_off"]]
        lens = encode(ro[r + 1] - ro[r] for r in range(int(L["g"])))
        syms = encode(int(x) for x in L["rhs"])
        head += struct.pack("<4Q", int(L["g"]), ro[-1], len(lens), len(syms))
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
        lens = decode(take(nb_len), g)
        syms = decode(take(nb_rhs), G)
        F = np.frombuffer(take(4 * g), dtype="<u4").astype(np.uint32)
        ro = np.zeros(g + 1, dtype=np.uint64)
        for r, ln in enumerate(lens):
            if ln == 0:
                raise ValueError("empty rule")
            ro[r + 1] = ro[r] + ln
        if int(ro[-1]) != G:
            raise ValueError("rule lengths disagree with G")
        levels.append({"g": g, "rhs_off": ro, "rhs": np.array(syms, dtype=np.uint32), "F": F})
    c_level = np.frombuffer(take(4 * k), dtype="<u4").astype(np.uint32)
    c_rank = np.frombuffer(take(4 * k), dtype="<u4").astype(np.uint32)
    F0 = np.frombuffer(take(4 * 256), dtype="<u4").astype(np.uint32)
    if pos != len(buf):
        raise ValueError("wrong size")
    return {"F0": F0, "levels": levels, "c_level": c_level, "c_rank": c_rank}
