"""The serving loop's host logic on the CPU, with the oracle standing in for
the GPU's build / merge: continuous batching over two lanes, admission by the
batch-size and memory limits, results that are the same alone and in the mix,
and a resident grammar equal to BuildGram over the strings in the order they
were merged (Sec. 3.6)."""
import numpy as np
import pytest

import lcg_inputs as li
from oracle import oracle as O
from paper_2411_12439_gb300 import serving


class OracleBackend:
    def __init__(self, hf):
        self.hf = hf
        self.tag = O.family_tag(hf)
        self.F0 = O.build(li.from_strings([b"A"]), hf).export()["F0"]
        self.builds = 0

    def empty(self):
        return O.from_export({"levels": [], "c_level": np.zeros(0, np.uint32), "c_rank": np.zeros(0, np.uint32),
                              "F0": self.F0}, self.tag)

    def gather(self, lane, parts, total):
        return np.concatenate(parts)

    def build(self, lane, data, offsets):
        self.builds += 1
        return O.build(li.Collection(data=data, offsets=offsets), self.hf)

    def roots(self, lane, g):
        ex = g.export()
        lv = ex["c_level"]
        fp = np.array([ex["F0"][r] if l == 0 else ex["levels"][l - 1]["F"][r] for l, r in zip(lv, ex["c_rank"])],
                      dtype=np.uint32)
        return lv, fp

    def merge(self, resident, g):
        return resident.merge(g)

    def build_info(self, lane):
        return {}

    def size(self, g):
        return g.k

    def free(self, g):
        pass

    def memory_budget(self, fraction):
        return 1 << 40

    def pack(self, g):
        from paper_2411_12439_gb300 import sharding
        return sharding.pack(g.export())

    def unpack(self, buf):
        from paper_2411_12439_gb300 import sharding
        return O.from_export(sharding.unpack(buf), self.tag)


def _requests(seed, count):
    rng = np.random.default_rng(seed)
    base = li.random_dna(rng, 40_000)
    out, t = [], 0.0
    for i in range(count):
        t += float(rng.exponential(0.002))
        n = int(rng.integers(1, 6000))
        if i % 5 == 4:
            data = np.frombuffer(li.zipf_text(rng, n).tobytes(), dtype=np.uint8)
        else:
            s0 = int(rng.integers(0, base.shape[0] - n))
            data = li.apply_snps(rng, base[s0:s0 + n], 0.01)
        out.append(li.Request(t, data, "x"))
    return out


def _alone(hf, data):
    g = O.build(li.from_strings([data]), hf)
    lv, fp = OracleBackend(hf).roots(0, g)
    return int(lv[0]), int(fp[0])


def test_results_alone_and_in_the_mix(hf):
    stream = _requests(11, 40)
    backend = OracleBackend(hf)
    srv = serving.Server(backend, lanes=2, max_batch_bytes=20_000)
    srv.start()
    reqs = serving.replay(srv, stream)
    assert srv.drain(reqs, timeout=120)
    srv.stop()
    assert not srv.errors
    for r in reqs:
        assert r.error is None
        assert r.result == _alone(hf, r.data)
    # every batch within the size limit (a single request may exceed it)
    for lane, cnt, nbytes, t0, t1 in srv.batches:
        assert cnt == 1 or nbytes <= 20_000
    assert len(srv.batches) > 1 and {b[0] for b in srv.batches} == {0, 1}
    # the resident grammar is BuildGram over the strings in merge order
    order = sorted(reqs, key=lambda r: r.index)
    assert [r.index for r in order] == list(range(len(reqs)))
    want = O.build(li.from_strings([r.data for r in order]), hf).export()
    assert O.grammars_equal(srv.resident.export(), want)
    st = serving.latency_stats(reqs)
    assert st["requests"] == len(reqs) and 0 < st["p50_s"] <= st["p99_s"]


def test_memory_admission(hf):
    """With a budget of two strings' worth, no more than two strings are in
    flight at once, and a string larger than the budget still runs alone."""
    rng = np.random.default_rng(3)
    datas = [li.random_dna(rng, 3000) for _ in range(8)] + [li.random_dna(rng, 9000)]
    backend = OracleBackend(hf)
    srv = serving.Server(backend, lanes=3, max_batch_bytes=1 << 30, mem_factor=1.0, budget_bytes=6000)
    for d in datas:
        srv.submit(d)
    srv.start()
    reqs = list(srv._pending)
    assert srv.drain(reqs, timeout=120)
    srv.stop()
    for r in reqs:
        assert r.result == _alone(hf, r.data)
    # batches that run at the same time hold at most the budget; the oversized
    # string runs with nothing beside it
    spans = srv.batches
    for i, (_, c1, b1, s1, e1) in enumerate(spans):
        overlap = sum(b2 for j, (_, c2, b2, s2, e2) in enumerate(spans) if j != i and s2 < e1 and s1 < e2)
        if b1 > 6000:
            assert c1 == 1 and overlap == 0
        else:
            assert b1 + overlap <= 6000
    assert any(b == 9000 for _, _, b, _, _ in spans)


def test_empty_request_fails_alone(hf):
    srv = serving.Server(OracleBackend(hf), lanes=1)
    r = srv.submit(b"")
    assert r.wait(1) and r.error


def test_snapshot_and_restore(hf):
    """A snapshot of the resident grammar, restored into a new server, lets it
    continue: the result is the grammar of all strings in merge order."""
    backend = OracleBackend(hf)
    first = serving.Server(backend, lanes=1, max_batch_bytes=30_000)
    first.start()
    reqs = serving.replay(first, _requests(41, 8))
    assert first.drain(reqs, timeout=120)
    first.stop()
    snap = first.snapshot()
    second = serving.Server(backend, lanes=2, max_batch_bytes=30_000)
    second.restore(snap)
    second.start()
    more = serving.replay(second, _requests(42, 6))
    assert second.drain(more, timeout=120)
    second.stop()
    assert not first.errors and not second.errors
    order = sorted(reqs, key=lambda r: r.index) + sorted(more, key=lambda r: r.index)
    assert [r.index for r in order] == list(range(len(order)))
    want = O.build(li.from_strings([r.data for r in order]), hf).export()
    assert O.grammars_equal(second.resident.export(), want)



def test_merges_run_off_the_requests_path(hf):
    """Requests complete when their roots are known; their batches are merged
    afterwards by the merge thread, in hand-over order, while the lanes build
    the next batches (a slow merge does not hold the lanes up)."""
    import time

    class SlowMerge(OracleBackend):
        def __init__(self, hf):
            super().__init__(hf)
            self.merges = []

        def merge(self, resident, g):
            t0 = time.perf_counter()
            time.sleep(0.05)
            out = super().merge(resident, g)
            self.merges.append((t0, time.perf_counter()))
            return out

    backend = SlowMerge(hf)
    srv = serving.Server(backend, lanes=2, max_batch_bytes=6_000)
    srv.start()
    reqs = serving.replay(srv, _requests(12, 30))
    assert srv.drain(reqs, timeout=120)
    srv.stop()
    assert not srv.errors
    for r in reqs:
        assert r.t_done <= r.t_merged
        assert r.result == _alone(hf, r.data)
    # some batch was taken by a lane while an earlier batch was being merged
    starts = [t0 for _, _, _, t0, _ in srv.batches]
    assert any(m0 < s < m1 for s in starts for m0, m1 in backend.merges)
    order = sorted(reqs, key=lambda r: r.index)
    assert [r.index for r in order] == list(range(len(reqs)))
    want = O.build(li.from_strings([r.data for r in order]), hf).export()
    assert O.grammars_equal(srv.resident.export(), want)
    assert all("merge" in p and "merge_wait" in p for p in srv.phases)
