"""A collection sharded over processes (one per GPU), and the merge tree that
joins their grammars.

BuildGram with one hash family over disjoint parts of a collection gives
grammars that MergeGrams joins into the grammar of the whole collection
(stable property, Sec. 3.1; MergeGrams, Sec. 3.6).  Because ranks within a
level follow the first occurrence in collection order, merging the parts in
collection order gives exactly the grammar a single BuildGram over all strings
gives: every rank's part is a contiguous range of strings, and at each merge
the lower-ranked part absorbs the higher-ranked one.

The exchange is the one step that moves data between processes: log2(P) stages
in which half of the remaining ranks send their grammar (exported to host
arrays, a small fraction of the input) to a partner that imports and merges it.
Rank 0 ends with the grammar of the collection.

The grammar operations come from a ``backend`` with ``build(data, offsets)``,
``pack(g)`` / ``unpack(buf)`` (a grammar as one byte buffer) and
``merge(a, b)`` (a absorbs b; returns a), and the transport from a ``comm``
with ``send(buf, dst)`` / ``recv(src)`` of uint8 arrays.  ``CudaBackend`` and
``TorchComm`` are the ones for GPUs; ``CudaBackend`` sends the packed form of
lcg_export_packed, or the VByte form of lcg_export_vbyte (about half the
bytes: rule lengths and right-hand sides as VBytes, Sec. 4) for links slower
than the encode and decode.
"""
from __future__ import annotations

import numpy as np

_MAGIC = 0x4C434753  # "LCGS": the packed form of lcg_export_packed


def shard_by_bytes(offsets, world: int) -> list[tuple[int, int]]:
    """Contiguous string ranges [lo, hi), one per rank, with about the same
    number of bytes each (a rank may get none when there are fewer strings
    than ranks).  String j goes to the rank whose byte interval holds the
    middle of the string."""
    off = np.asarray(offsets, dtype=np.uint64).astype(np.float64)
    k = off.shape[0] - 1
    if world < 1:
        raise ValueError("world must be >= 1")
    total = off[-1] - off[0]
    if k == 0 or total == 0:
        return [(0, k)] + [(k, k)] * (world - 1)
    mid = (off[:-1] + off[1:]) / 2.0 - off[0]
    owner = np.minimum((mid * world / total).astype(np.int64), world - 1)
    cuts = np.searchsorted(owner, np.arange(world + 1), side="left")
    return [(int(cuts[r]), int(cuts[r + 1])) for r in range(world)]


def _pad8(a: np.ndarray) -> np.ndarray:
    b = a.view(np.uint8)
    r = (-b.size) % 8
    return np.concatenate([b, np.zeros(r, dtype=np.uint8)]) if r else b


def pack(ex: dict | None) -> np.ndarray:
    """The packed form (the layout of lcg_export_packed: a u64 header, then
    per level rhs_off, rhs and F, then C and F0, every array starting at a
    multiple of 8 bytes) of an exported grammar; None gives an empty buffer
    (a rank without strings)."""
    if ex is None:
        return np.zeros(0, dtype=np.uint8)
    levels = ex["levels"]
    k = int(np.asarray(ex["c_level"]).shape[0])
    head = [_MAGIC, k, len(levels)]
    for L in levels:
        head += [int(L["g"]), int(np.asarray(L["rhs"]).shape[0])]
    parts = [np.asarray(head, dtype=np.uint64).view(np.uint8)]
    for L in levels:
        parts.append(np.ascontiguousarray(L["rhs_off"], dtype=np.uint64).view(np.uint8))
        parts.append(_pad8(np.ascontiguousarray(L["rhs"], dtype=np.uint32)))
        parts.append(_pad8(np.ascontiguousarray(L["F"], dtype=np.uint32)))
    parts.append(_pad8(np.ascontiguousarray(ex["c_level"], dtype=np.uint32)))
    parts.append(_pad8(np.ascontiguousarray(ex["c_rank"], dtype=np.uint32)))
    parts.append(np.ascontiguousarray(ex["F0"], dtype=np.uint32).view(np.uint8))
    return np.concatenate(parts)


def unpack(buf) -> dict | None:
    """Inverse of ``pack`` (also reads the buffers of lcg_export_packed)."""
    buf = np.ascontiguousarray(buf, dtype=np.uint8)
    if buf.size == 0:
        return None
    pos = 0

    def take(n, dt):
        nonlocal pos
        nb = n * np.dtype(dt).itemsize
        if pos + nb > buf.size:
            raise ValueError("truncated grammar buffer")
        a = buf[pos:pos + nb].copy().view(dt)
        pos += nb + (-nb) % 8
        return a

    magic, k, nl = (int(x) for x in take(3, np.uint64))
    if magic != _MAGIC:
        raise ValueError("not a packed grammar")
    sizes = take(2 * nl, np.uint64).reshape(nl, 2) if nl else np.zeros((0, 2), dtype=np.uint64)
    levels = []
    for g, G in sizes:
        g, G = int(g), int(G)
        levels.append({"g": g, "rhs_off": take(g + 1, np.uint64), "rhs": take(G, np.uint32),
                       "F": take(g, np.uint32)})
    ex = {"levels": levels, "c_level": take(k, np.uint32), "c_rank": take(k, np.uint32),
          "F0": take(256, np.uint32)}
    if pos != buf.size:
        raise ValueError("trailing bytes after a packed grammar")
    return ex


def merge_tree(grammar, rank: int, world: int, backend, comm):
    """Join the ranks' grammars (rank r holding the r-th part of the
    collection) by a binary tree of MergeGrams.  Returns the grammar of the
    whole collection on rank 0, None on the other ranks.  ``grammar`` may be
    None for a rank without strings."""
    stride = 1
    while stride < world:
        if rank % (2 * stride) == stride:
            comm.send(np.zeros(0, dtype=np.uint8) if grammar is None else backend.pack(grammar), rank - stride)
            return None
        if rank % (2 * stride) == 0 and rank + stride < world:
            buf = comm.recv(rank + stride)
            if buf.size:
                other = backend.unpack(buf)
                grammar = other if grammar is None else backend.merge(grammar, other)
        stride *= 2
    return grammar if rank == 0 else None


def build_sharded(data, offsets, rank: int, world: int, backend, comm):
    """BuildGram of a collection whose strings are split over ``world``
    ranks by ``shard_by_bytes``: each rank builds its part, then the merge
    tree joins them.  ``data`` and ``offsets`` describe the whole collection
    (``offsets`` on the host); only this rank's strings are parsed here.
    Returns the collection's grammar on rank 0, None elsewhere."""
    off = np.asarray(offsets, dtype=np.uint64)
    lo, hi = shard_by_bytes(off, world)[rank]
    g = None
    if hi > lo:
        base = int(off[lo])
        part = (off[lo:hi + 1] - np.uint64(base)).astype(np.uint64)
        g = backend.build(data[base:int(off[hi])], part)
    return merge_tree(g, rank, world, backend, comm)


class CudaBackend:
    """Grammar operations of a ``Context`` (the CUDA path).  ``form``: the
    exchange format, "packed" (lcg_export_packed) or "vbyte"
    (lcg_export_vbyte)."""

    def __init__(self, ctx, form: str = "packed"):
        if form not in ("packed", "vbyte"):
            raise ValueError("form is 'packed' or 'vbyte'")
        self.ctx = ctx
        self.form = form

    def build(self, data, offsets):
        return self.ctx.build(data, offsets)

    def pack(self, g) -> np.ndarray:
        return np.asarray(g.export_packed() if self.form == "packed" else g.export_vbyte())

    def unpack(self, buf):
        buf = np.ascontiguousarray(buf, dtype=np.uint8)
        return self.ctx.import_packed(buf) if self.form == "packed" else self.ctx.import_vbyte(buf)

    def merge(self, a, b):
        self.ctx.merge(a, b)
        b.free()
        return a


class TorchComm:
    """send / recv of uint8 arrays over the default torch.distributed group.
    With NCCL the buffers travel through ``device`` (a CUDA device); with
    gloo they stay on the host."""

    def __init__(self, device=None):
        import torch
        self.torch = torch
        self.device = torch.device(device) if device is not None else torch.device("cpu")

    def send(self, buf: np.ndarray, dst: int) -> None:
        import torch.distributed as dist
        t = self.torch
        n = t.tensor([int(buf.size)], dtype=t.int64, device=self.device)
        dist.send(n, dst)
        if buf.size:
            dist.send(t.from_numpy(np.ascontiguousarray(buf)).to(self.device), dst)

    def recv(self, src: int) -> np.ndarray:
        import torch.distributed as dist
        t = self.torch
        n = t.zeros(1, dtype=t.int64, device=self.device)
        dist.recv(n, src)
        size = int(n.item())
        if size == 0:
            return np.zeros(0, dtype=np.uint8)
        b = t.empty(size, dtype=t.uint8, device=self.device)
        dist.recv(b, src)
        return b.cpu().numpy()
