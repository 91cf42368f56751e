"""Serving loop: continuous batching of string-compression requests on one GPU.

Requests (strings) arrive at any time.  ``lanes`` workers, each with its own
context and CUDA stream, take batches from the queue of pending requests: a
worker that becomes free admits pending requests, oldest first, while the
batch stays under ``max_batch_bytes`` and the device-memory estimate of all
running batches stays under the budget, and runs the batch's BuildGram
(Sec. 3.3) at once, so that requests arriving while other batches are on the
GPU start as soon as a lane and memory are free, and their work overlaps on
the device.  A batch's requests complete as soon as their roots are read;
the batch's grammar then goes to a merge thread, which merges the batches
(MergeGrams, Sec. 3.6) into the grammar kept resident on the device in the
order they were handed over, on a context of its own, while the lanes build
the next batches.

A request's result is the root of its string: the level of its C entry and
the fingerprint of its expansion (F^level[rank], Eq. fast_hash), which depend
on the string's content only and are therefore the same whether the string
was parsed alone or in any mix; plus the string's index in the resident
grammar (fixed when its batch is handed to the merge thread), from which it
can be expanded once the batch is merged (``Request.wait_merged``).

Memory admission: the context's allocations come from a stream-ordered pool
that keeps freed memory, so the free memory the driver reports does not come
back after a batch.  The server therefore keeps its own account: a budget
(a fraction of the device memory free when it starts) and, per running batch,
``mem_factor`` times its input bytes.
"""
from __future__ import annotations

import collections
import threading
import time
import warnings

import numpy as np


class Request:
    """One string to compress.  ``result`` is (level, fingerprint) of its
    root, ``index`` its string index in the resident grammar, ``latency`` the
    seconds from submission to completion."""

    def __init__(self, data, t_submit: float):
        self.data = np.ascontiguousarray(np.frombuffer(data, dtype=np.uint8) if isinstance(data, (bytes, bytearray))
                                         else data, dtype=np.uint8)
        self.t_submit = t_submit
        self.t_start = None
        self.t_done = None
        self.result = None
        self.index = None
        self.error = None
        self.batch = None
        self._done = threading.Event()
        self._merged = threading.Event()

    @property
    def n(self) -> int:
        return int(self.data.shape[0])

    @property
    def latency(self) -> float:
        return self.t_done - self.t_submit

    def wait(self, timeout=None) -> bool:
        return self._done.wait(timeout)

    def wait_merged(self, timeout=None) -> bool:
        """Wait until the request's string is in the resident grammar (or failed)."""
        return self._merged.wait(timeout)


class CudaBackend:
    """Grammar operations on the GPU: one context per lane (each with its own
    stream) for builds, and one context that owns the resident grammar."""

    def __init__(self, hash_family, device: int = 0, lanes: int = 2):
        import torch
        from .lcg import Context
        self.device = device
        self.res_ctx = Context(hash_family, device=device)
        # every lane's context launches on a stream of its own
        self.lane_streams = [torch.cuda.Stream(device=device) for _ in range(lanes)]
        self.ctxs = [Context(hash_family, device=device, stream=s.cuda_stream) for s in self.lane_streams]
        self.staging = [None] * lanes
        self.dev_staging = [None] * lanes
        self.record_events = False
        self.events = []
        self._ev_lock = threading.Lock()
        self.ref = torch.cuda.Event(enable_timing=True)
        self.ref.record(torch.cuda.current_stream(device))
        torch.cuda.synchronize(device)

    def empty(self):
        return self.res_ctx.import_grammar({"levels": [], "c_level": np.zeros(0, np.uint32),
                                            "c_rank": np.zeros(0, np.uint32), "F0": np.zeros(256, np.uint32)})

    def gather(self, lane: int, parts, total: int):
        """The batch's strings back to back.  Requests received into
        page-locked memory are copied straight into the lane's device buffer
        (one asynchronous copy each, on the lane's stream, which the host then
        waits for); others are first gathered into the
        lane's page-locked host buffer, so that the build's upload runs at
        link speed.  Buffers grow as needed."""
        import torch
        with warnings.catch_warnings():  # read-only request bytes are only read here
            warnings.filterwarnings("ignore", message="The given NumPy array is not writable")
            ts = [torch.from_numpy(x) for x in parts]
        if all(t.is_pinned() for t in ts):
            # on the lane's own stream (the buffer belongs to that stream's
            # pool, so replacing it is ordered too); the host waits for the
            # copies, as a resident-mode build reads the buffer on the resident
            # grammar's stream
            ls = self.lane_streams[lane]
            with torch.cuda.stream(ls):
                dev = self.dev_staging[lane]
                if dev is None or dev.numel() < total:
                    self.dev_staging[lane] = None
                    dev = torch.empty(max(total, 1 << 20) * 5 // 4, dtype=torch.uint8, device=self.device)
                    self.dev_staging[lane] = dev
                off = 0
                for t in ts:
                    n = t.numel()
                    dev[off:off + n].copy_(t, non_blocking=True)
                    off += n
            ls.synchronize()
            return dev[:total]
        buf = self.staging[lane]
        if buf is None or buf.numel() < total:
            buf = torch.empty(max(total, 1 << 20) * 5 // 4, dtype=torch.uint8).pin_memory()
            self.staging[lane] = buf
        torch.cat(ts, out=buf[:total])
        return buf[:total]

    def build(self, lane: int, data, offsets: np.ndarray):
        """BuildGram on the lane's context; with ``record_events`` the build is
        bracketed by CUDA events on the lane's stream (device_intervals)."""
        if not self.record_events:
            return self.ctxs[lane].build(data, offsets)
        import torch
        ev = [torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)]
        s = self.lane_streams[lane]
        ev[0].record(s)
        g = self.ctxs[lane].build(data, offsets)
        ev[1].record(s)
        with self._ev_lock:
            self.events.append((lane, ev))
        return g

    def device_intervals(self):
        """(lane, start ms, end ms) of every recorded build, on the device's
        clock, relative to the backend's reference event."""
        import torch
        torch.cuda.synchronize(self.device)
        with self._ev_lock:
            evs = list(self.events)
        return [(lane, self.ref.elapsed_time(a), self.ref.elapsed_time(b)) for lane, (a, b) in evs]

    def roots(self, lane: int, g):
        lv, _, fp = g.roots()
        return lv, fp

    def build_info(self, lane: int) -> dict:
        st = self.ctxs[lane].last_build_stats()
        return {"rounds": st["rounds"], "async_rounds": st["async_rounds"], "redone": int(st["redone"]),
                "retries": sum(r["retries"] for r in st["per_round"])}

    def merge(self, resident, g):
        self.res_ctx.merge(resident, g)
        return resident

    def build_into(self, resident, data, offsets):
        """The batch parsed against the resident grammar (App. A.2), on the
        context that owns it."""
        self.res_ctx.build_into(resident, data, offsets)

    def roots_of(self, g, j0: int, count: int):
        lv, _, fp = g.roots(j0, count)
        return lv, fp

    def size(self, g) -> int:
        return g.shape[0]

    def pack(self, g) -> np.ndarray:
        return np.asarray(g.export_packed())

    def unpack(self, buf):
        return self.res_ctx.import_packed(np.ascontiguousarray(buf, dtype=np.uint8))

    def free(self, g):
        g.free()

    def memory_budget(self, fraction: float) -> int:
        import torch
        free, _ = torch.cuda.mem_get_info(self.device)
        return int(free * fraction)


class Server:
    """Continuous-batching request loop over a grammar kept resident on the
    device.  ``submit`` may be called from any thread; ``start`` runs the
    lanes (and the merge thread) in background threads, ``stop`` ends them
    after the pending work.  ``mode``: "merge" builds each batch on its lane
    (lanes in parallel), completes its requests, and hands the batch's grammar
    to the merge thread, which merges batches into the resident grammar
    (MergeGrams) in hand-over order while the lanes go on; "resident" parses
    each batch against the resident grammar itself (App. A.2, one at a time)
    after gathering it on its lane."""

    def __init__(self, backend, lanes: int = 2, max_batch_bytes: int = 64 << 20, mem_factor: float = 12.0,
                 budget_bytes: int | None = None, budget_fraction: float = 0.5, mode: str = "merge"):
        if mode not in ("merge", "resident"):
            raise ValueError("mode is 'merge' or 'resident'")
        self.mode = mode
        self.backend = backend
        self.lanes = lanes
        self.max_batch_bytes = max_batch_bytes
        self.mem_factor = mem_factor
        self.budget = budget_bytes if budget_bytes is not None else backend.memory_budget(budget_fraction)
        self.resident = backend.empty()
        self._pending = collections.deque()
        self._cv = threading.Condition()
        self._merge_lock = threading.Lock()  # held while the resident grammar changes
        self._mq = collections.deque()       # (base index, grammar, requests, bytes estimate, t handed over, phases)
        self._mcv = threading.Condition()
        self._assigned = 0                   # strings handed to the merge thread so far
        self._merging = False
        self._inflight = 0.0
        self._running = False
        self._threads = []
        self.batches = []  # (lane, number of requests, input bytes, t_start, t_end)
        self.phases = []   # per batch: seconds spent gathering, building, reading roots, waiting, merging
        self.errors = []

    # -- requests -------------------------------------------------------------
    def submit(self, data) -> Request:
        r = Request(data, time.perf_counter())
        if r.n == 0:
            r.error = "empty string"
            r.t_done = r.t_submit
            r._done.set()
            return r
        with self._cv:
            self._pending.append(r)
            self._cv.notify_all()
        return r

    # -- checkpoint -----------------------------------------------------------
    def snapshot(self) -> np.ndarray:
        """The resident grammar in its packed form (lcg_export_packed layout),
        taken once every batch handed over so far is merged: a checkpoint of
        everything served so far."""
        self.flush()
        with self._merge_lock:
            return self.backend.pack(self.resident)

    def restore(self, buf) -> None:
        """Continue from a snapshot: the resident grammar becomes the packed
        grammar ``buf`` (later requests get indexes after its strings)."""
        g = self.backend.unpack(buf)
        self.flush()
        with self._merge_lock, self._mcv:
            old, self.resident = self.resident, g
            self._assigned = self.backend.size(g)
        self.backend.free(old)

    def flush(self, timeout: float | None = None) -> bool:
        """Wait until every batch handed to the merge thread is merged."""
        end = None if timeout is None else time.perf_counter() + timeout
        with self._mcv:
            while self._mq or self._merging:
                left = None if end is None else end - time.perf_counter()
                if left is not None and left <= 0:
                    return False
                self._mcv.wait(0.05 if left is None else min(0.05, left))
        return True

    # -- lanes ----------------------------------------------------------------
    def start(self):
        self._running = True
        if self.mode == "merge":
            self._assigned = self.backend.size(self.resident)
        for lane in range(self.lanes):
            t = threading.Thread(target=self._lane, args=(lane,), daemon=True)
            t.start()
            self._threads.append(t)
        if self.mode == "merge":
            self._mthread = threading.Thread(target=self._merger, daemon=True)
            self._mthread.start()

    def stop(self, timeout: float | None = None):
        with self._cv:
            self._running = False
            self._cv.notify_all()
        for t in self._threads:
            t.join(timeout)
        self._threads = []
        if self.mode == "merge" and getattr(self, "_mthread", None) is not None:
            with self._mcv:
                self._mcv.notify_all()
            self._mthread.join(timeout)
            self._mthread = None

    def drain(self, requests, timeout: float | None = None, merged: bool = True) -> bool:
        """Wait until every request in ``requests`` has its result and, with
        ``merged``, its string is in the resident grammar."""
        end = None if timeout is None else time.perf_counter() + timeout
        for r in requests:
            left = None if end is None else max(0.0, end - time.perf_counter())
            if not (r.wait_merged(left) if merged else r.wait(left)):
                return False
        return True

    def _take_batch(self):
        """Admit pending requests, oldest first, into a batch (under the lock)."""
        batch, nbytes = [], 0
        while self._pending:
            r = self._pending[0]
            need = self.mem_factor * (nbytes + r.n)
            if batch and (nbytes + r.n > self.max_batch_bytes or self._inflight + need > self.budget):
                break
            if not batch and self._inflight > 0 and self._inflight + need > self.budget:
                break  # wait for memory: another batch is running
            self._pending.popleft()
            batch.append(r)
            nbytes += r.n
        return batch, nbytes

    def _lane(self, lane: int):
        while True:
            with self._cv:
                while True:
                    batch, nbytes = self._take_batch() if self._pending else ([], 0)
                    if batch:
                        est = self.mem_factor * nbytes
                        self._inflight += est
                        break
                    if not self._running and not self._pending:
                        return
                    self._cv.wait(0.05)
            t0 = time.perf_counter()
            for r in batch:
                r.t_start = t0
            try:
                offsets = np.zeros(len(batch) + 1, dtype=np.uint64)
                np.cumsum([r.n for r in batch], out=offsets[1:])
                data = self.backend.gather(lane, [r.data for r in batch], int(offsets[-1]))
                ta = time.perf_counter()
                if self.mode == "resident":
                    # parse against the resident grammar itself: new rules are
                    # appended to it, no merge step (one batch at a time)
                    with self._merge_lock:
                        tq = time.perf_counter()
                        base = self.backend.size(self.resident)
                        self.backend.build_into(self.resident, data, offsets)
                        tb = time.perf_counter()
                        levels, fps = self.backend.roots_of(self.resident, base, len(batch))
                    tc = t1 = time.perf_counter()
                    ph = {"gather": ta - t0, "build": tb - tq, "roots": tc - tb, "merge": 0.0, "wait": tq - ta}
                else:
                    g = self.backend.build(lane, data, offsets)
                    tb = time.perf_counter()
                    levels, fps = self.backend.roots(lane, g)
                    t1 = time.perf_counter()
                    ph = {"gather": ta - t0, "build": tb - ta, "roots": t1 - tb}
                    ph.update(self.backend.build_info(lane))
                    # hand the grammar to the merge thread: the batch's strings
                    # take the next indexes of the resident grammar
                    with self._mcv:
                        base = self._assigned
                        self._assigned += len(batch)
                        self._mq.append((base, g, batch, est, t1, ph))
                        self._mcv.notify_all()
                self.phases.append(ph)
                for j, r in enumerate(batch):
                    r.result = (int(levels[j]), int(fps[j]))
                    r.index = base + j
                    r.batch = len(self.batches)
                    r.t_done = t1
            except Exception as e:  # the batch's requests fail; the lane goes on
                t1 = time.perf_counter()
                self.errors.append(repr(e))
                for r in batch:
                    r.error = repr(e)
                    r.t_done = t1
                    r._merged.set()
                with self._cv:
                    self._inflight -= est
                    self._cv.notify_all()
                est = 0.0
            with self._cv:
                if self.mode == "resident":
                    self._inflight -= est  # merge mode: released by the merge thread
                self.batches.append((lane, len(batch), nbytes, t0, t1))
                self._cv.notify_all()
            for r in batch:
                if self.mode == "resident":
                    r._merged.set()
                r._done.set()

    def _merger(self):
        """Merges handed-over batch grammars into the resident grammar, in
        hand-over order, on the resident grammar's context; releases each
        batch's memory estimate once its grammar is freed."""
        while True:
            with self._mcv:
                while not self._mq:
                    if not self._running and not self._threads_alive():
                        return
                    self._mcv.wait(0.05)
                base, g, batch, est, t_handed, ph = self._mq.popleft()
                self._merging = True
            t0 = time.perf_counter()
            try:
                with self._merge_lock:
                    self.resident = self.backend.merge(self.resident, g)
                self.backend.free(g)
            except Exception as e:  # the batch's strings are not in the resident grammar
                self.errors.append(repr(e))
                for r in batch:
                    r.error = repr(e)
            t1 = time.perf_counter()
            ph["merge_wait"] = t0 - t_handed
            ph["merge"] = t1 - t0
            with self._cv:
                self._inflight -= est
                self._cv.notify_all()
            with self._mcv:
                self._merging = False
                self._mcv.notify_all()
            for r in batch:
                r.t_merged = t1
                r._merged.set()

    def _threads_alive(self) -> bool:
        return any(t.is_alive() for t in self._threads)


def latency_stats(requests) -> dict:
    """p50 / p99 / mean latency (seconds) and input GB/s over the span from the
    first submission to the last completion."""
    done = [r for r in requests if r.t_done is not None and r.error is None]
    if not done:
        return {"requests": 0}
    lat = np.array([r.latency for r in done])
    span = max(r.t_done for r in done) - min(r.t_submit for r in done)
    nbytes = sum(r.n for r in done)
    return {"requests": len(done), "p50_s": float(np.percentile(lat, 50)), "p99_s": float(np.percentile(lat, 99)),
            "mean_s": float(lat.mean()), "input_bytes": int(nbytes), "span_s": float(span),
            "gbs": nbytes / span / 1e9 if span > 0 else None}


def replay(server: Server, stream, time_scale: float = 1.0):
    """Submit the requests of ``stream`` (objects with ``arrival_s`` and
    ``data``) at their arrival times, scaled by ``time_scale``; returns the
    Request objects."""
    t0 = time.perf_counter()
    out = []
    for item in stream:
        delay = item.arrival_s * time_scale - (time.perf_counter() - t0)
        if delay > 0:
            time.sleep(delay)
        out.append(server.submit(item.data))
    return out
