"""Benchmark of the batched LCG build on one GB300 (or N GPUs, one process each).

Metric: input GB/s of BuildGram (lcg_build) over the largest single-GPU
configuration, the large repetitive strings: 4 strings of 3.1 Gbp over ACGTN
(12.4 GB), all parsed together in one call per step; results are checked
bit-exact against the oracle in the test suite (full-grammar digests).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--workload c4|c3|c2]

One JSON line is printed by rank 0.  ``value`` is the whole-job input
throughput with the inputs resident in HBM (every timed build one launch of
the build's CUDA graph); ``e2e`` is the same metric through the public API
from page-locked host memory, with the whole grammar copied back to the host
every step; ``roofline`` rates the parse kernel (the kernel with most device
time) on its algorithmic bytes against the measured HBM bandwidth;
``path_roofline`` rates the whole step; ``plain`` is the one-string-per-build
form on the same GPU; ``extra_configs`` gives the same figures for the uneven
batch (2000 strings, 8 GB) and the bacterial-like batch (64 strings, 320 MB);
``cpu_baseline`` times the CPU oracle on a bounded sample of the workload, on
one thread and (``cpu_baseline_threaded``) on several with the parts merged;
``serving`` runs the request loop on the serving stream at three offered loads.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import lcg_inputs as li  # noqa: E402

METRIC = "LCG build input GB/s on 1 GB300 (batched vs plain), bit-exact; % of HBM peak"
FALLBACK_HBM_GBS = 6800.0
L2_BYTES = 126.5e6  # a round's phrase table beyond this is read from HBM

WORKLOADS = {
    "c4": {"make": li.repetitive_collection, "seed": 4,
           "desc": ("large repetitive strings: 4 strings of 3.1 Gbp over ACGTN (12.4 GB): a seeded random base with "
                    "10^6 copies of 10 repeat families (300 bp-6 kbp, 10-20% divergence) and N-runs up to 50 kbp "
                    "(about 1%); strings 2-4 are string 1 with 0.1% SNPs; all strings in one batched build per step")},
    "c3": {"make": li.uneven_collection, "seed": 3,
           "desc": ("uneven batch: 2000 strings with lognormal lengths in 0.5-12 Mbp (8.0 GB) from 50 seeded "
                    "12 Mbp genomes with 0.5-3% divergence; all strings in one batched build per step")},
    "c2": {"make": li.bacterial_collection, "seed": 2,
           "desc": ("bacterial-like batch: 64 strings of ~5 Mbp from 4 seeded random base genomes (1% SNPs, "
                    "0.02% indels of 1-50 bp, 5 block rearrangements per string), 320 MB; all strings in one "
                    "batched build per step")},
}

SERVING_WORKLOAD = ("serving stream: 2000 requests, Poisson arrivals, lognormal lengths (median 1 Mbp, sigma 1.5) "
                    "clipped to [10 kbp, 50 Mbp]; 80% windows of 100 seeded 50 Mbp genomes with 0.1-1% SNPs, "
                    "20% Zipf(1.1) byte text with copied 1-64 KB blocks; 2 lanes, merged into a device-resident "
                    "grammar")


def parse_args():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=10)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", choices=["ours", "reference"], default="ours")
    p.add_argument("--workload", choices=sorted(WORKLOADS), default="c4")
    p.add_argument("--retune", action="store_true", help="tune again even when the tuning cache has the class")
    p.add_argument("--tuning-out", default="", help="also write the tuning cache entries used to this path")
    p.add_argument("--no-plain", action="store_true")
    p.add_argument("--no-extra", action="store_true", help="skip the uneven and bacterial-like configurations")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-serving", action="store_true")
    p.add_argument("--no-graph", action="store_true", help="time the builds as separate launches")
    p.add_argument("--no-postprocess", action="store_true")
    p.add_argument("--no-vbyte", action="store_true")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--e2e-steps", type=int, default=8)
    p.add_argument("--e2e-streams", type=int, default=2, help="contexts (streams, host threads) of the e2e steps")
    p.add_argument("--serving-requests", type=int, default=2000)
    p.add_argument("--serving-lanes", type=int, default=2)
    p.add_argument("--serving-batch-mb", type=int, default=192)
    p.add_argument("--profile-builds", type=int, default=0,
                   help="only run this many batched builds of the workload inside the profiler range and exit")
    p.add_argument("--profile-warmup", type=int, default=1,
                   help="with --profile-builds: builds run before the profiler range "
                        "(cudaProfilerStart/Stop; use ncu --profile-from-start off)")
    p.add_argument("--profile-length", type=int, default=0,
                   help="with --profile-builds and --workload c4: strings of this length instead of 3.1 Gbp "
                        "(the same recipe, a capture small enough for ncu)")
    p.add_argument("--write-traffic", default="",
                   help="ncu CSV (dram__bytes_read.sum, dram__bytes_write.sum of the k_parse launches) of "
                        "--profile-builds 1 with the same --workload / --profile-length: writes "
                        "profiles/traffic.json with DRAM bytes per algorithmic byte of k_parse")
    p.add_argument("--traffic-command", default="", help="the ncu command recorded in profiles/traffic.json")
    return p.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def workload(name: str, rank: int = 0, length: int = 0):
    """The named configuration; under weak scaling every rank parses its own
    collection of the same shape (another seed)."""
    w = WORKLOADS[name]
    kw = {"seed": w["seed"] + 1000 * rank}
    if length and name == "c4":
        kw.update(length=length, copies=max(1000, length // 3100))
    return w["make"](**kw)


def measured_peak():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            return float(json.load(fh)["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


def kernel_source_hash() -> str:
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2411_12439_gb300", "csrc")
    for f in sorted(os.listdir(csrc)):
        with open(os.path.join(csrc, f), "rb") as fh:
            h.update(f.encode())
            h.update(fh.read())
    return h.hexdigest()[:16]


def profiled_traffic(kernel: str):
    """DRAM bytes per algorithmic byte of `kernel` from the committed ncu
    summary, when it was taken from the current kernel sources."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as fh:
            t = json.load(fh)
    except Exception:
        return None
    if t.get("source_hash") != kernel_source_hash():
        return None
    entry = t.get("kernels", {}).get(kernel)
    if not entry:
        return None
    return float(entry["dram_bytes_per_alg_byte"])


def parse_alg_bytes(r: dict, round_no: int, tables: bool = True) -> float:
    """Algorithmic bytes of one k_parse launch (the method's own traffic):
    the round's sequence read (1 B per symbol in round 1, a 4-byte rank
    afterwards), plus one 32-byte table sector per phrase when the round's
    phrase table is larger than L2 (`tables`)."""
    b = (1.0 if round_no == 1 else 4.0) * r["n"]
    if tables and r["table_cap"] * 32.0 > L2_BYTES:
        b += 32.0 * r["phrases"]
    return b


def path_alg_bytes(rounds: list, tables: bool = True) -> float:
    """Algorithmic bytes of a whole build: the input read, every round's
    sequence written once and read once (4 B per symbol), the new rules (4 B
    per right-hand-side symbol, 4 B of F and 8 B of offset per rule), plus one
    table sector per phrase of every round whose table exceeds L2 (`tables`)."""
    if not rounds:
        return 0.0
    b = float(rounds[0]["n"])
    for r in rounds:
        b += 8.0 * r["phrases"] + 4.0 * r["G"] + 12.0 * r["g"]
        if tables and r["table_cap"] * 32.0 > L2_BYTES:
            b += 32.0 * r["phrases"]
    return b


class ClockSampler:
    """nvidia-smi samples every 200 ms while the timed region runs."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device: int):
        self.device = device
        self.rows = []
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-lms", "200", "-i", str(self.device)], stdout=subprocess.PIPE,
                                         stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            parts = [x.strip() for x in line.split(",")]
            if len(parts) >= 9:
                self.rows.append(parts)

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        if not self.rows:
            return None
        sm = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        smax = [float(r[2]) for r in self.rows if r[2].replace(".", "").isdigit()]
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in self.rows:
            for name, v in zip(names, r[5:9]):
                if v.strip().lower() == "active":
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(self.rows)}


# --------------------------------------------------------------------------
# the oracle on the host cores (cpu_baseline and the reference arm)
# --------------------------------------------------------------------------

def oracle_sample(coll, nbytes: int):
    """A bounded sample of the workload: with at most 8 strings, the same
    prefix of every string (nbytes in total); otherwise the first strings,
    about nbytes in total.  Returns (collection, description)."""
    if coll.k <= 8:
        per = max(2, int(nbytes) // coll.k)
        sub = li.from_strings([coll.string(j)[:per] for j in range(coll.k)])
        return sub, f"the first {per / 1e6:.1f} MB of each of the {coll.k} strings ({sub.n / 1e6:.1f} MB)"
    lens = np.diff(coll.offsets.astype(np.int64))
    take = max(1, min(coll.k, int(np.searchsorted(np.cumsum(lens), nbytes)) + 1))
    sub = coll.subset(range(take))
    return sub, f"the first {take} of {coll.k} strings ({sub.n / 1e6:.1f} MB)"


def cpu_baseline(coll, hf, target_s: float = 12.0):
    """The oracle as it stands, one host thread, on a bounded sample of the
    workload (sized from a short probe to about `target_s` seconds)."""
    from oracle import oracle as O
    probe, _ = oracle_sample(coll, 4_000_000)
    t = time.perf_counter()
    O.build(probe, hf)
    rate = probe.n / max(time.perf_counter() - t, 1e-6)
    sample, desc = oracle_sample(coll, int(target_s * rate))
    t = time.perf_counter()
    O.build(sample, hf)
    dt = time.perf_counter() - t
    return {"value": sample.n / dt / 1e9, "unit": "GB/s", "cores": 1, "kind": "oracle",
            "sample": f"{desc}, one oracle build on 1 thread", "seconds": dt}


def cpu_baseline_threaded(coll, hf, rate_1t: float, target_s: float = 10.0):
    """The oracle on the host cores as the paper's implementation runs in
    parallel: contiguous parts of a bounded sample, one oracle build per
    thread, merged in a tree by the oracle's MergeGrams (the result is the
    build of the whole sample).  ``rate_1t`` (bytes/s of one thread) sizes the
    sample to about ``target_s`` seconds.  The threads used are at most the
    host's cores and at most the sample's strings."""
    from oracle import oracle as O
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else (os.cpu_count() or 1)
    threads = min(cores, coll.k)
    sample, desc = oracle_sample(coll, int(target_s * rate_1t * threads))
    subs = O.split(sample, threads)
    t = time.perf_counter()
    g = O.build_parts(subs, hf)
    dt = time.perf_counter() - t
    if g.k != sample.k:
        raise RuntimeError("threaded oracle lost strings")
    return {"value": sample.n / dt / 1e9, "unit": "GB/s", "cores": len(subs), "kind": "oracle",
            "host_cores": cores,
            "sample": f"{desc} in {len(subs)} contiguous parts, one oracle build per thread, merged by the oracle "
                      f"MergeGrams in a tree", "seconds": dt}


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    hf = li.hash_family()
    coll = workload(args.workload)
    from oracle import oracle as O
    O.build_library()
    # each step: a bounded sample of the workload (a few seconds of one thread)
    sample, desc = oracle_sample(coll, 40_000_000 if coll.k <= 8 else 20_000_000)
    del coll
    for _ in range(args.warmup):
        O.build(sample, hf)
    times = []
    for _ in range(args.steps):
        t = time.perf_counter()
        O.build(sample, hf)
        times.append(time.perf_counter() - t)
    tot = sum(times)
    value = sample.n * args.steps / tot / 1e9
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "GB/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": tot / args.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u8/u32",
        "data": "synthetic",
        "config": {"workload": WORKLOADS[args.workload]["desc"], "sample": f"{desc} per step",
                   "parallelism": "single host thread"},
        "cpu_baseline": {"value": value, "unit": "GB/s", "cores": 1, "kind": "oracle",
                         "sample": f"{desc} per step"},
        "e2e": {"value": value, "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# --------------------------------------------------------------------------
# the GPU legs
# --------------------------------------------------------------------------

def timed_builds(ctx, d, offsets, steps: int, stream, graph: bool):
    """`steps` builds bracketed by CUDA events on the context's stream, each
    freeing its grammar; only the parse launches carry events of their own
    (kernel timing mode 2).  Returns (ms per step, per-round k_parse ms
    (mean over the steps), launches of the library's kernels, graph modes)."""
    import torch
    ctx.set_kernel_timing(2)
    ctx.set_graph(graph)
    for _ in range(2):  # the plan, then the graph's capture: outside the timed region
        ctx.build(d, offsets).free()
    parse_ms = {}
    launches = 0
    modes = []
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        g = ctx.build(d, offsets)
        for rec in ctx.last_kernel_launches():
            if rec["name"] == "k_parse":
                parse_ms[rec["round"]] = parse_ms.get(rec["round"], 0.0) + rec["ms"] / steps
        st = ctx.last_build_stats()
        launches += st["kernel_launches"]
        modes.append(st["graph"])
        g.free()
    e1.record(stream)
    torch.cuda.synchronize()
    ctx.set_kernel_timing(0)
    ctx.set_graph(False)
    return e0.elapsed_time(e1) / steps, parse_ms, launches, modes


def round_breakdown(ctx, d, offsets, builds: int = 3):
    """Builds as launches with every launch timed: per round its sizes and
    device time, per kernel kind its time per build."""
    ctx.set_kernel_timing(1)
    per_round, kernels = None, {}
    for _ in range(builds):
        ctx.build(d, offsets).free()
        rs = ctx.last_build_stats()["per_round"]
        if per_round is None or len(per_round) != len(rs):
            per_round = [{k: r[k] for k in ("n", "phrases", "g", "G", "table_cap", "strings")} | {"ms": []}
                         for r in rs]
        byround = {}
        for rec in ctx.last_kernel_launches():
            byround[rec["round"]] = byround.get(rec["round"], 0.0) + rec["ms"]
            k = kernels.setdefault(rec["name"], {"launches": 0, "ms": 0.0})
            k["launches"] += 1
            k["ms"] += rec["ms"]
        for i, pr in enumerate(per_round):
            pr["ms"].append(byround.get(i + 1, 0.0))
    ctx.set_kernel_timing(0)
    for pr in per_round:
        pr["ms"] = float(np.median(pr["ms"]))
    kernels = {k: {"launches": v["launches"] // builds, "ms_per_step": v["ms"] / builds}
               for k, v in sorted(kernels.items(), key=lambda kv: -kv[1]["ms"])}
    return per_round, kernels


def plain_form(ctx, d, offsets, stream, warm: bool = True):
    """The plain form: every string built alone (one string per launch
    sequence, the same kernels), back to back, after one untimed pass.
    Returns (ms, the single-string grammars' merge time in ms or None)."""
    import torch
    offs = offsets.astype(np.int64)
    k = len(offs) - 1

    def one(j):
        sub = d[int(offs[j]):int(offs[j + 1])]
        return ctx.build(sub, np.array([0, sub.numel()], dtype=np.uint64))

    if warm:
        for j in range(k):
            one(j).free()
    torch.cuda.synchronize()
    p0 = torch.cuda.Event(enable_timing=True)
    p1 = torch.cuda.Event(enable_timing=True)
    p0.record(stream)
    gs = []
    for j in range(k):
        g = one(j)
        if k <= 8:
            gs.append(g)  # kept for the merge below
        else:
            g.free()
    p1.record(stream)
    torch.cuda.synchronize()
    ms = p0.elapsed_time(p1)
    merge_ms = None
    if gs:
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for g in gs[1:]:
            ctx.merge(gs[0], g)
        torch.cuda.synchronize()
        merge_ms = (time.perf_counter() - t0) * 1e3
        for g in gs:
            g.free()
    return ms, merge_ms


def tune(ctx, coll, d, args, note):
    from paper_2411_12439_gb300 import autotune
    cls = autotune.config_class(coll.n, coll.k, coll.data[:1 << 20])
    rep = autotune.tuned(ctx, d, coll.offsets, cls, retune=args.retune, reps=3, sweeps=1, note=note)
    if args.tuning_out:
        cache = autotune.load_cache(args.tuning_out)
        cache[cls] = autotune.load_cache().get(cls) or {"tuning": rep["tuning"], "ms": rep.get("ms"), "note": note}
        with open(args.tuning_out, "w") as fh:
            json.dump(cache, fh, indent=1, sort_keys=True)
    return rep


def extra_config(name, hf, local, stream, args):
    """Batched and plain GB/s of another configuration (inputs resident)."""
    import torch
    from paper_2411_12439_gb300 import Context
    coll = workload(name)
    d = torch.from_numpy(coll.data).to(f"cuda:{local}")
    ctx = Context(hf, device=local, stream=stream.cuda_stream)
    for _ in range(2):
        ctx.build(d, coll.offsets).free()
    tuned = tune(ctx, coll, d, args, WORKLOADS[name]["desc"])
    steps = max(3, min(args.steps, int(2000 / max(1.0, coll.n / 40e6))))
    ms, parse_ms, _, modes = timed_builds(ctx, d, coll.offsets, steps, stream, not args.no_graph)
    rounds, _ = round_breakdown(ctx, d, coll.offsets, builds=1)
    out = {"workload": WORKLOADS[name]["desc"], "strings": coll.k, "input_bytes": int(coll.n),
           "value": coll.n / (ms / 1e3) / 1e9, "unit": "GB/s", "ms_per_step": ms, "steps": steps,
           "rounds": len(rounds), "graph_modes": sorted(set(modes)), "tuning": tuned,
           "levels_g": int(sum(r["g"] for r in rounds)), "levels_G": int(sum(r["G"] for r in rounds))}
    peak, _ = measured_peak()
    out["path_frac_streams_only"] = path_alg_bytes(rounds, tables=False) / (ms / 1e3) / 1e9 / peak
    out["path_frac_with_tables"] = path_alg_bytes(rounds, tables=True) / (ms / 1e3) / 1e9 / peak
    if not args.no_plain:
        pms, _ = plain_form(ctx, d, coll.offsets, stream)
        out["plain"] = {"value": coll.n / (pms / 1e3) / 1e9, "unit": "GB/s", "ms_per_step": pms,
                        "batched_over_plain": pms / ms,
                        "form": "every string built alone (one string per launch sequence), back to back, "
                                "after one untimed pass"}
    ctx.close()
    del d
    torch.cuda.synchronize()
    torch.cuda.empty_cache()
    return out


def run_serving(hf, device: int, count: int, loads=(0.1, 0.25, 0.5), mode: str = "merge", lanes: int = 2,
                max_batch_mb: int = 192):
    """The serving loop on the seeded serving stream: first all requests at
    once (the loop's capacity: input GB/s from first submission to last
    completion), then the same requests with Poisson arrivals paced so that the
    offered input rate is ``load`` times that capacity: p50 / p99 latency and
    delivered GB/s per load.  Every run gets a fresh server (two lanes and the
    merge thread), warmed up on a stream of another seed first."""
    from paper_2411_12439_gb300 import serving

    import torch

    def make(seed, n):
        stream = li.serving_stream(seed=seed, count=n, rate_hz=1.0)
        for item in stream:  # requests arrive in page-locked receive buffers
            item.data = torch.from_numpy(np.ascontiguousarray(item.data, dtype=np.uint8)).pin_memory().numpy()
        return stream

    warm_stream = make(50, max(20, count // 20))
    stream = make(51, count)
    mean_len = float(np.mean([r.data.shape[0] for r in stream]))

    def run(time_scale):
        backend = serving.CudaBackend(hf, device=device, lanes=lanes)
        srv = serving.Server(backend, lanes=lanes, max_batch_bytes=max_batch_mb << 20, mode=mode)
        srv.start()
        warm = serving.replay(srv, warm_stream, time_scale=1e-4)
        srv.drain(warm, timeout=600)
        b0, e0 = len(srv.phases), len(srv.errors)
        reqs = serving.replay(srv, stream, time_scale=time_scale)  # arrival_s was drawn at 1 request/s
        ok = srv.drain(reqs, timeout=900, merged=False)
        srv.flush(timeout=900)
        st = serving.latency_stats(reqs)
        ph = srv.phases[b0:]
        srv.stop()
        out = {"requests": st.get("requests"), "gbs": st.get("gbs"),
               "p50_ms": 1e3 * st["p50_s"] if "p50_s" in st else None,
               "p99_ms": 1e3 * st["p99_s"] if "p99_s" in st else None, "batches": len(ph),
               "errors": len(srv.errors) - e0 + (0 if ok else 1),
               "batch_ms": {k: 1e3 * float(np.mean([p.get(k, 0.0) for p in ph]))
                            for k in ("gather", "build", "roots", "merge_wait", "merge")} if ph else None,
               "builds_redone": sum(p.get("redone", 0) for p in ph),
               "table_regrowths": sum(p.get("retries", 0) for p in ph)}
        del srv, backend
        torch.cuda.synchronize()
        torch.cuda.empty_cache()
        return out

    burst = run(0.0)
    capacity = burst["gbs"] or 1.0
    runs = []
    for load in loads:
        rate = load * capacity * 1e9 / mean_len  # requests per second
        r = run(1.0 / rate)
        r.update({"load": load, "offered_gbs": load * capacity})
        runs.append(r)
    return {"workload": SERVING_WORKLOAD, "stream_bytes": int(sum(r.data.shape[0] for r in stream)),
            "max_batch_mb": max_batch_mb, "lanes": lanes, "mode": mode, "capacity": burst,
            "loads": "fractions of the capacity (all requests submitted at once)",
            "latency": "from submission to the request's root (its batch built); batches merge into the resident "
                       "grammar afterwards (batch_ms.merge_wait, .merge)",
            "warmup": f"{len(warm_stream)} requests of another seed", "runs": runs}


def run_profile(args):
    """Only batched builds of the workload inside a profiler range (ncu)."""
    import torch
    from paper_2411_12439_gb300 import Context
    hf = li.hash_family()
    coll = workload(args.workload, 0, args.profile_length)
    d = torch.from_numpy(coll.data).cuda()
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    ctx = Context(hf, device=0, stream=stream.cuda_stream)
    for _ in range(args.profile_warmup):
        ctx.build(d, coll.offsets).free()
    torch.cuda.synchronize()
    torch.cuda.profiler.start()
    for _ in range(args.profile_builds):
        ctx.build(d, coll.offsets).free()
    torch.cuda.synchronize()
    torch.cuda.profiler.stop()
    return 0


def e2e_run(hf, local, coll, hd, tuning, lanes, args, barrier, max_over_ranks):
    """End to end through the public API: page-locked host input, the whole
    grammar to a page-locked host buffer in its packed form every step.
    Steps run on `lanes` contexts (each with its own stream and host thread,
    as a serving process would), so that one step's copies overlap another
    step's kernels.  The lanes' builds run as launches, not captured graphs:
    a graph keeps the memory of all its rounds, so two graphs of a large build
    need twice its memory, while launches return each round's buffers to the
    stream-ordered pool for the next.  Raises when the lanes do not fit in
    device memory."""
    import torch
    from paper_2411_12439_gb300 import Context
    streams = [torch.cuda.Stream(device=local) for _ in range(lanes)]
    ectx = [Context(hf, device=local, stream=s.cuda_stream) for s in streams]
    try:
        outs = []
        for c in ectx:
            c.set_tuning(**tuning)
            for _ in range(2):  # a plan, then a build from it
                g = c.build(hd, coll.offsets)
                if len(outs) < len(ectx):
                    outs.append(torch.empty(g.packed_size() * 5 // 4 + 4096, dtype=torch.uint8).pin_memory())
                g.free()
        barrier()
        torch.cuda.synchronize()
        e2e_steps = max(args.e2e_steps, lanes)
        per_lane = [e2e_steps // lanes + (1 if i < e2e_steps % lanes else 0) for i in range(lanes)]
        d2h_seen = [0] * lanes
        errors = []

        def e2e_lane(i, steps):
            try:
                for _ in range(steps):
                    g = ectx[i].build(hd, coll.offsets)
                    d2h_seen[i] = int(g.export_packed(outs[i]).numel())
                    g.free()
            except Exception as e:  # reported below
                errors.append(repr(e))

        def e2e_pass(steps):
            threads = [threading.Thread(target=e2e_lane, args=(i, steps[i])) for i in range(lanes)]
            for t in threads:
                t.start()
            for t in threads:
                t.join()
            torch.cuda.synchronize()
            if errors:
                raise RuntimeError("end-to-end step failed: " + errors[0])

        e2e_pass([1] * lanes)  # untimed: the lanes' steps running together once, as they will when timed
        barrier()
        t0 = time.perf_counter()
        e2e_pass(per_lane)
        e2e_s = max_over_ranks((time.perf_counter() - t0) / e2e_steps)
        return {"value": coll.n / e2e_s / 1e9, "unit": "GB/s", "h2d_bytes_per_step": int(coll.n),
                "d2h_bytes_per_step": max(d2h_seen), "ms_per_step": e2e_s * 1e3, "steps": e2e_steps,
                "streams": lanes,
                "result": "grammar in its packed form (lcg_export_packed) in page-locked host memory",
                "builds": "launches (no graph capture), all rounds enqueued from the context's plan",
                "timing": "host clock from the first step's start to the last step's grammar in host memory"}
    finally:
        for c in ectx:
            c.close()


def run_ours(args):
    import torch
    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    from paper_2411_12439_gb300 import Context

    hf = li.hash_family()
    coll = workload(args.workload, rank)
    d = torch.from_numpy(coll.data).to(f"cuda:{local}")
    # a stream of our own: the context launches on it and the timing events
    # are recorded on it
    torch.cuda.synchronize()
    stream = torch.cuda.Stream(device=local)
    torch.cuda.set_stream(stream)
    ctx = Context(hf, device=local, stream=stream.cuda_stream)

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()

    def max_over_ranks(x: float) -> float:
        if world == 1:
            return x
        import torch.distributed as dist
        t = torch.tensor([x], dtype=torch.float64, device=f"cuda:{local}")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        return float(t.item())

    for _ in range(args.warmup):
        ctx.build(d, coll.offsets).free()
    tuned = tune(ctx, coll, d, args, WORKLOADS[args.workload]["desc"])

    # ---- timed region: inputs resident in HBM (larger than L2, no flush needed);
    #      every build one launch of the CUDA graph of its planned rounds
    sampler = ClockSampler(local)
    barrier()
    torch.cuda.synchronize()
    sampler.start()
    ms, parse_ms, launches, modes = timed_builds(ctx, d, coll.offsets, args.steps, stream, not args.no_graph)
    barrier()
    clocks = sampler.stop()
    ms = max_over_ranks(ms)
    value = world * coll.n / (ms / 1e3) / 1e9
    stats = ctx.last_build_stats()

    # ---- per round and per kernel, every launch timed (as launches)
    rounds, kernels = round_breakdown(ctx, d, coll.offsets)
    peak, peak_kind = measured_peak()

    # ---- roofline of k_parse (the kernel with most device time) over the
    #      timed builds: algorithmic bytes per launch over its mean duration
    nl = len([r for r in parse_ms if 1 <= r <= len(rounds)])
    pb = sum(parse_alg_bytes(rounds[r - 1], r) for r in parse_ms if 1 <= r <= len(rounds))
    pb_streams = sum(parse_alg_bytes(rounds[r - 1], r, tables=False) for r in parse_ms if 1 <= r <= len(rounds))
    pt = sum(v for r, v in parse_ms.items() if 1 <= r <= len(rounds))
    roofline = None
    if nl and pt > 0:
        achieved = (pb / nl) / (pt / nl / 1e3) / 1e9
        ratio = profiled_traffic("k_parse")
        roofline = {"bound": "hbm", "kernel": "k_parse", "achieved": achieved, "peak": peak, "unit": "GB/s",
                    "frac": achieved / peak, "peak_source": f"{peak_kind} (MEASURED_PEAKS.json hbm_gbs)",
                    "traffic": (ratio * pb / nl) if ratio is not None else None,
                    "alg_bytes_per_launch": pb / nl, "launches_per_step": nl, "ms_per_step": pt,
                    "frac_streams_only": (pb_streams / nl) / (pt / nl / 1e3) / 1e9 / peak,
                    "alg_bytes": "per round: the sequence read (1 B per symbol in round 1, 4 B later) plus one "
                                 "32-byte table sector per phrase when the round's table exceeds L2 "
                                 "(frac_streams_only: without the table sectors)",
                    "timing": "CUDA events around every parse launch of the timed builds (graph event nodes)",
                    "share_of_kernel_time": (kernels["k_parse"]["ms_per_step"] /
                                             sum(v["ms_per_step"] for v in kernels.values()))
                    if "k_parse" in kernels else None}
    path_roofline = {
        "alg_bytes_streams_only": path_alg_bytes(rounds, tables=False),
        "alg_bytes_with_tables": path_alg_bytes(rounds, tables=True),
        "frac_streams_only": path_alg_bytes(rounds, tables=False) / (ms / 1e3) / 1e9 / peak,
        "frac_with_tables": path_alg_bytes(rounds, tables=True) / (ms / 1e3) / 1e9 / peak,
        "note": "all rounds' algorithmic bytes over the timed step: input read, each round's sequence written "
                "and read once (4 B per symbol), new rules (4 B per symbol, 12 B per rule), and, with tables, "
                "one 32-byte sector per phrase of every round whose table exceeds L2"}
    rounds_line = [{"round": i + 1, "symbols": int(r["n"]), "phrases": int(r["phrases"]), "g": int(r["g"]),
                    "G": int(r["G"]), "table_mb": r["table_cap"] * 32 / 1e6, "ms": r["ms"],
                    "parse_ms": parse_ms.get(i + 1),
                    "gbs": r["n"] * (1 if i == 0 else 4) / (r["ms"] / 1e3) / 1e9 if r["ms"] > 0 else None}
                   for i, r in enumerate(rounds)]

    # ---- plain form: each string built alone, back to back (and the merge of
    #      the single-string grammars, timed apart)
    plain = None
    if not args.no_plain:
        pms, merge_ms = plain_form(ctx, d, coll.offsets, stream)
        pms = max_over_ranks(pms)
        pv = world * coll.n / (pms / 1e3) / 1e9
        plain = {"value": pv, "unit": "GB/s", "ms_per_step": pms, "batched_over_plain": value / pv,
                 "merge_ms": merge_ms,
                 "form": "every string built alone (one string per launch sequence, the same kernels), back to "
                         "back, after one untimed pass; merge_ms: MergeGrams of the single-string grammars"}

    # ---- post-processing of the batch's grammar: run-length rules, then Simp
    post = None
    if not args.no_postprocess:
        g = ctx.build(d, coll.offsets)
        times = []
        for _ in range(3):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            pp = ctx.postprocess(g)
            torch.cuda.synchronize()
            times.append(time.perf_counter() - t0)
            st = pp.stats()
            pp.free()
        g.free()
        pms = float(np.median(times)) * 1e3
        post = {"ms": pms, "grammar_gbs": 4.0 * st["size_before"] / (pms / 1e3) / 1e9, **st,
                "timing": "host clock around lcg_postprocess (it synchronises between levels)"}

    # ---- the VByte form of the batch's grammar: sizes, export / import times
    vbyte_line = None
    if not args.no_vbyte:
        g = ctx.build(d, coll.offsets)
        packed = g.packed_size()
        nbytes = g.vbyte_size()
        buf = torch.empty(nbytes, dtype=torch.uint8, device=f"cuda:{local}")
        ex_t, im_t = [], []
        for _ in range(3):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            g.export_vbyte(out=buf)
            ex_t.append(time.perf_counter() - t0)
            t0 = time.perf_counter()
            ctx.import_vbyte(buf).free()
            im_t.append(time.perf_counter() - t0)
        g.free()
        del buf
        vbyte_line = {"packed_bytes": packed, "vbyte_bytes": nbytes, "ratio": nbytes / packed,
                      "export_ms": float(np.median(ex_t)) * 1e3, "import_ms": float(np.median(im_t)) * 1e3,
                      "timing": "host clock around lcg_export_vbyte / lcg_import_vbyte (device buffer; both "
                                "synchronise)"}
    ctx.close()
    del d
    torch.cuda.synchronize()
    torch.cuda.empty_cache()

    # ---- end to end through the public API: page-locked host input, the whole
    #      grammar to a page-locked host buffer in its packed form every step.
    #      Steps run on `--e2e-streams` contexts (each with its own stream and
    #      host thread, as a serving process would), so that one step's copies
    #      overlap another step's kernels.
    e2e = None
    if not args.no_e2e:
        hd = torch.from_numpy(coll.data).pin_memory()
        lanes = max(1, args.e2e_streams)
        lane_note = None
        while True:
            try:
                e2e = e2e_run(hf, local, coll, hd, tuned["tuning"], lanes, args, barrier, max_over_ranks)
                break
            except Exception as e:  # two lanes' working sets do not fit the device at once: one lane
                torch.cuda.synchronize()
                torch.cuda.empty_cache()
                if lanes == 1 or "ENOMEM" not in repr(e):
                    raise
                lane_note = f"{lanes} lanes did not fit in device memory together ({e}); one lane"
                lanes = 1
        e2e["value"] *= world
        e2e["streams_note"] = lane_note
        del hd
        torch.cuda.synchronize()
        torch.cuda.empty_cache()

    # ---- the other configurations: the uneven batch and the bacterial-like batch
    extra = None
    if not args.no_extra and world == 1:
        extra = {name: extra_config(name, hf, local, stream, args) for name in ("c3", "c2")
                 if name != args.workload}

    if rank != 0:
        return 0
    cpu = cpu_threaded = None
    if world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(coll, hf)
        cpu_threaded = cpu_baseline_threaded(coll, hf, cpu["value"] * 1e9)
    serving_line = None
    if world == 1 and not args.no_serving:
        serving_line = run_serving(hf, local, args.serving_requests, lanes=args.serving_lanes,
                                   max_batch_mb=args.serving_batch_mb)
    line = {
        "metric": METRIC, "value": value, "unit": "GB/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u8/u32", "data": "synthetic",
        "config": {"workload": WORKLOADS[args.workload]["desc"], "strings": coll.k, "input_bytes": int(coll.n),
                   "rounds": stats["rounds"],
                   "l2": f"inputs larger than L2 ({coll.n / 1e9:.1f} GB > 129 MB), no flush",
                   "autotuned": tuned,
                   "cuda_graph": ("every timed build a graph launch" if modes and min(modes) == 2
                                  else f"graph modes of the timed builds: {modes}"),
                   "parallelism": f"dp{world}" if world > 1 else "single GPU"},
        "e2e": e2e, "gpu_launches": int(launches), "clocks": clocks, "roofline": roofline,
        "path_roofline": path_roofline, "plain": plain, "extra_configs": extra,
        "cpu_baseline": cpu, "cpu_baseline_threaded": cpu_threaded, "serving": serving_line,
        "rounds": rounds_line, "kernels": kernels, "postprocess": post, "vbyte": vbyte_line,
    }
    print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


def _ncu_dram_bytes(path: str) -> dict:
    """Sum of dram__bytes_read.sum + dram__bytes_write.sum per kernel kind
    (the name before any template argument list) in an ncu --csv log."""
    import csv
    scale = {"byte": 1.0, "Kbyte": 1e3, "Mbyte": 1e6, "Gbyte": 1e9, "Tbyte": 1e12}
    with open(path) as fh:
        rows = list(csv.reader(fh))
    head = next(i for i, r in enumerate(rows) if "Kernel Name" in r and "Metric Name" in r)
    hdr = rows[head]
    ki, mi, ui, vi, ii = (hdr.index(x) for x in ("Kernel Name", "Metric Name", "Metric Unit", "Metric Value", "ID"))
    out = {}
    for r in rows[head + 1:]:
        if len(r) <= vi or r[mi] not in ("dram__bytes_read.sum", "dram__bytes_write.sum"):
            continue
        kind = r[ki].split("(")[0].split("<")[0].replace("void ", "").split("::")[-1]
        e = out.setdefault(kind, {"dram_bytes": 0.0, "launch_ids": set()})
        e["dram_bytes"] += float(r[vi].replace(",", "")) * scale.get(r[ui], 1.0)
        e["launch_ids"].add(r[ii])
    return {k: {"dram_bytes": v["dram_bytes"], "launches": len(v["launch_ids"])} for k, v in out.items()}


def write_traffic(args):
    """profiles/traffic.json from an ncu capture of the k_parse launches of
    one profiled build (--profile-builds 1): DRAM bytes over the algorithmic
    bytes (parse_alg_bytes) of the same build's rounds."""
    import torch
    from paper_2411_12439_gb300 import Context
    dram = _ncu_dram_bytes(args.write_traffic)
    hf = li.hash_family()
    coll = workload(args.workload, 0, args.profile_length)
    d = torch.from_numpy(coll.data).cuda()
    ctx = Context(hf, device=0)
    for _ in range(args.profile_warmup):
        ctx.build(d, coll.offsets).free()
    ctx.build(d, coll.offsets).free()
    rs = ctx.last_build_stats()["per_round"]
    alg = sum(parse_alg_bytes(r, i + 1) for i, r in enumerate(rs))
    kernels = {}
    if "k_parse" in dram and alg > 0:
        kernels["k_parse"] = {"launches": dram["k_parse"]["launches"], "dram_bytes": dram["k_parse"]["dram_bytes"],
                              "alg_bytes": alg, "dram_bytes_per_alg_byte": dram["k_parse"]["dram_bytes"] / alg}
    out = {"source_hash": kernel_source_hash(), "command": args.traffic_command,
           "workload": WORKLOADS[args.workload]["desc"] +
           (f" (strings of {args.profile_length} bytes)" if args.profile_length else ""),
           "input_bytes": int(coll.n), "kernels": kernels,
           "scaling": "DRAM bytes per algorithmic byte of the captured build, applied to the benchmark's "
                      "launches (traffic grows with the units processed)"}
    path = os.path.join(ROOT, "profiles", "traffic.json")
    with open(path, "w") as fh:
        json.dump(out, fh, indent=1)
    print(json.dumps(out))
    return 0


def main():
    args = parse_args()
    if args.write_traffic:
        return write_traffic(args)
    if args.impl == "reference":
        return run_reference(args)
    if args.profile_builds:
        return run_profile(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
