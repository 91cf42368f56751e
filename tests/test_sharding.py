"""The multi-process path on the CPU: sharding by bytes, the packed exchange
format, and the MergeGrams tree over gloo ranks (world sizes 2 and 3).  Each
rank builds its part with the oracle; rank 0's merged grammar must equal the
oracle's BuildGram of the whole collection bit for bit (first-occurrence
ranks make Merge(Build(A), Build(B)) == Build(A.B), Sec. 3.6)."""
import multiprocessing as mp
import os
import socket

import numpy as np
import pytest

import lcg_inputs as li
from oracle import oracle as O
from paper_2411_12439_gb300 import sharding

import sharding_worker


def test_shard_by_bytes_contiguous_and_balanced():
    rng = np.random.default_rng(5)
    for world in (1, 2, 3, 4, 7):
        for _ in range(20):
            k = int(rng.integers(1, 40))
            lens = rng.integers(1, 1000, size=k)
            off = np.zeros(k + 1, dtype=np.uint64)
            np.cumsum(lens, out=off[1:])
            parts = sharding.shard_by_bytes(off, world)
            assert len(parts) == world
            assert parts[0][0] == 0 and parts[-1][1] == k
            for (a, b), (c, d) in zip(parts, parts[1:]):
                assert b == c and a <= b
            total = int(off[-1])
            for lo, hi in parts:
                # a part exceeds its share by at most one string
                assert int(off[hi] - off[lo]) <= total / world + int(lens.max())


def test_shard_by_bytes_fewer_strings_than_ranks():
    off = np.array([0, 10, 25], dtype=np.uint64)
    parts = sharding.shard_by_bytes(off, 4)
    assert sum(hi - lo for lo, hi in parts) == 2
    assert [p for p in parts if p[1] > p[0]] == [(0, 1), (1, 2)] or parts[0] == (0, 2)


def test_pack_roundtrip(hf):
    coll = li.tiny_dna_collection(base_len=5000, k=3)
    ex = O.build(coll, hf).export()
    back = sharding.unpack(sharding.pack(ex))
    assert O.grammars_equal(ex, back)
    assert sharding.unpack(sharding.pack(None)) is None
    with pytest.raises(ValueError):
        sharding.unpack(sharding.pack(ex)[:-3])


class _LocalComm:
    """In-process transport for a sequential run of the merge tree."""

    def __init__(self, boxes, rank):
        self.boxes, self.rank = boxes, rank

    def send(self, buf, dst):
        self.boxes[(self.rank, dst)] = buf

    def recv(self, src):
        return self.boxes.pop((src, self.rank))


def test_merge_tree_in_process(hf):
    """The tree's schedule without processes: ranks run from the highest to
    the lowest, so every send happens before its receive."""
    coll = li.tiny_dna_collection(base_len=8000, k=7)
    backend = sharding_worker.OracleBackend(hf)
    for world in (1, 2, 3, 5, 8):
        boxes = {}
        results = {}
        for rank in reversed(range(world)):
            results[rank] = sharding.build_sharded(coll.data, coll.offsets, rank, world, backend,
                                                   _LocalComm(boxes, rank))
        assert not boxes
        assert all(results[r] is None for r in range(1, world))
        assert O.grammars_equal(results[0].export(), O.build(coll, hf).export()), world


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _run_ranks(world, strings, out, fail_ranks=(), timeout_s=60, form="packed"):
    ctx = mp.get_context("spawn")
    port = _free_port()
    procs = [ctx.Process(target=sharding_worker.run,
                         args=(r, world, port, strings, out, fail_ranks, timeout_s, form))
             for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=180)
    codes = []
    for p in procs:
        if p.is_alive():
            p.kill()
            p.join()
        codes.append(p.exitcode)
    return codes


@pytest.mark.parametrize("world,form", [(2, "packed"), (3, "packed"), (2, "vbyte")])
def test_merge_tree_gloo(tmp_path, hf, world, form):
    rng = np.random.default_rng(40 + world)
    base = li.random_dna(rng, 6000)
    strings = [li.apply_snps(rng, base, 0.01).tobytes() for _ in range(5)] + [b"AC", b"G"]
    out = str(tmp_path / "merged.npy")
    codes = _run_ranks(world, strings, out, form=form)
    assert codes == [0] * world
    got = sharding.unpack(np.load(out))
    want = O.build(li.from_strings(strings), hf).export()
    assert O.grammars_equal(got, want)


def test_rank_failure_is_reported(tmp_path):
    """A rank that stops before the exchange: its partner's receive ends with
    an error (the gloo timeout or the closed connection), no rank hangs."""
    strings = [b"ACGTACGTTGCA" * 50, b"TTGACCA" * 80]
    out = str(tmp_path / "merged.npy")
    codes = _run_ranks(2, strings, out, fail_ranks=(1,), timeout_s=10)
    assert codes[1] != 0
    assert codes[0] != 0
    assert not os.path.exists(out)
