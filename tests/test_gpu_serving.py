"""The serving loop on the GPU: two lanes (contexts on their own streams)
build batches of requests that arrive while other batches run, merge them into
the device-resident grammar, and every request's root (level and fingerprint
of its expansion) equals the root of the same string parsed alone.  The
resident grammar equals the oracle's BuildGram over the strings in merge order,
and strings expand from it to their bytes."""
import numpy as np
import pytest

import lcg_inputs as li
from oracle import oracle as O

pytestmark = pytest.mark.gpu


def _stream(seed, count):
    rng = np.random.default_rng(seed)
    bases = [li.random_dna(rng, 2_000_000) for _ in range(3)]
    out, t = [], 0.0
    for i in range(count):
        t += float(rng.exponential(0.003))
        n = int(np.clip(rng.lognormal(np.log(60_000), 1.2), 2, 1_500_000))
        if i % 5 == 4:
            data = np.frombuffer(li.zipf_text(rng, n).tobytes(), dtype=np.uint8)
        else:
            b = bases[int(rng.integers(0, 3))]
            s0 = int(rng.integers(0, b.shape[0] - n))
            data = li.apply_snps(rng, b[s0:s0 + n], float(rng.uniform(0.001, 0.01)))
        out.append(li.Request(t, data, "x"))
    return out


@pytest.mark.parametrize("mode", ["merge", "resident"])
def test_serving_alone_and_in_the_mix(hf, mode):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2411_12439_gb300 import Context, serving
    stream = _stream(21, 36)
    if mode == "resident":  # requests received into page-locked memory: the device-side gather
        for item in stream:
            item.data = torch.from_numpy(np.ascontiguousarray(item.data)).pin_memory().numpy()
    backend = serving.CudaBackend(hf, device=0, lanes=2)
    srv = serving.Server(backend, lanes=2, max_batch_bytes=3 << 20, mode=mode)
    srv.start()
    reqs = serving.replay(srv, stream)
    assert srv.drain(reqs, timeout=300)
    srv.stop()
    assert not srv.errors, srv.errors
    assert len(srv.batches) > 2
    alone_ctx = Context(hf, device=0)
    for r in reqs:
        g = alone_ctx.build(r.data, np.array([0, r.n], dtype=np.uint64))
        lv, _, fp = g.roots()
        assert r.result == (int(lv[0]), int(fp[0]))
        g.free()
    order = sorted(reqs, key=lambda r: r.index)
    assert [r.index for r in order] == list(range(len(reqs)))
    want = O.build(li.from_strings([r.data for r in order]), hf).export()
    assert O.grammars_equal(srv.resident.export(), want)
    for r in order[::7]:
        assert srv.resident.decompress(r.index) == r.data.tobytes()
    st = serving.latency_stats(reqs)
    assert st["requests"] == len(reqs) and st["p99_s"] >= st["p50_s"] > 0


def test_snapshot_restore_on_the_gpu(hf):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2411_12439_gb300 import serving
    stream = _stream(23, 16)
    backend = serving.CudaBackend(hf, device=0, lanes=2)
    first = serving.Server(backend, lanes=2, max_batch_bytes=3 << 20)
    first.start()
    a = serving.replay(first, stream[:8])
    assert first.drain(a, timeout=300)
    first.stop()
    snap = first.snapshot()
    second = serving.Server(serving.CudaBackend(hf, device=0, lanes=2), lanes=2, max_batch_bytes=3 << 20)
    second.restore(snap)
    second.start()
    b = serving.replay(second, stream[8:])
    assert second.drain(b, timeout=300)
    second.stop()
    assert not first.errors and not second.errors
    order = sorted(a, key=lambda r: r.index) + sorted(b, key=lambda r: r.index)
    assert [r.index for r in order] == list(range(len(order)))
    want = O.build(li.from_strings([r.data for r in order]), hf).export()
    assert O.grammars_equal(second.resident.export(), want)



def test_lanes_overlap_on_the_device(hf):
    """Two lanes build batches at the same time: their builds' CUDA-event
    intervals (on the device's clock) overlap, each request's root equals the
    root of its string built alone, and the resident grammar equals the
    oracle's."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2411_12439_gb300 import Context, serving
    rng = np.random.default_rng(61)
    base = li.random_dna(rng, 6_000_000)
    stream = []
    for i in range(12):
        s0 = int(rng.integers(0, base.shape[0] - 4_000_000))
        stream.append(li.Request(0.0, li.apply_snps(rng, base[s0:s0 + 4_000_000], 0.005), "dna"))
    backend = serving.CudaBackend(hf, device=0, lanes=2)
    backend.record_events = True
    srv = serving.Server(backend, lanes=2, max_batch_bytes=8 << 20)
    for item in stream:  # a burst: both lanes get work at once
        srv.submit(item.data)
    reqs = list(srv._pending)
    srv.start()
    assert srv.drain(reqs, timeout=300)
    srv.stop()
    assert not srv.errors, srv.errors
    iv = backend.device_intervals()
    assert {lane for lane, _, _ in iv} == {0, 1}
    overlap = [(a, b) for a in iv for b in iv if a[0] == 0 and b[0] == 1 and a[1] < b[2] and b[1] < a[2]]
    assert overlap, iv
    alone = Context(hf, device=0)
    for r in reqs:
        g = alone.build(r.data, np.array([0, r.n], dtype=np.uint64))
        lv, _, fp = g.roots()
        assert r.result == (int(lv[0]), int(fp[0]))
        g.free()
    order = sorted(reqs, key=lambda r: r.index)
    want = O.build(li.from_strings([r.data for r in order]), hf).export()
    assert O.grammars_equal(srv.resident.export(), want)
