"""Benchmark of the batched LCG build on one GB300 (or N GPUs, one process each).

Metric: input GB/s of BuildGram (lcg_build) over a bacterial-like batch of 64
strings of ~5 Mbp (320 MB), all strings parsed together in one call per step,
with the result checked bit-exact against the oracle in the test suite.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

One JSON line is printed by rank 0.  ``value`` is the whole-job input
throughput with the inputs resident in HBM; ``e2e`` is the same metric through
the public API from pinned host memory, with the grammar copied back to the
host every step; ``roofline`` rates the kernel with the largest device time
against the measured HBM bandwidth; ``cpu_baseline`` times the CPU oracle on a
bounded sample of the same workload, on one thread and (``cpu_baseline_threaded``)
on every host core with the parts merged; ``plain`` is the one-string-at-a-time form
(each string parsed against the growing resident grammar); ``rounds`` gives per
round the symbols parsed, the device time of all its kernels and the GB/s of
its sequence (1-byte symbols in round 1, 4-byte ranks afterwards); ``vbyte``
measures the VByte form of the batch's grammar (sizes, export and import).
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
WORKLOAD = ("bacterial-like batch: 64 strings of ~5 Mbp from 4 seeded random base genomes "
            "(1% SNPs, 0.02% indels of 1-50 bp, 5 block rearrangements per string), 320 MB, "
            "all strings in one batched build per step")
FALLBACK_HBM_GBS = 6800.0


def parse_args():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=20)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", choices=["ours", "reference"], default="ours")
    p.add_argument("--no-plain", action="store_true")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-serving", action="store_true")
    p.add_argument("--no-autotune", action="store_true")
    p.add_argument("--no-graph", action="store_true", help="time the builds as separate launches")
    p.add_argument("--no-postprocess", action="store_true")
    p.add_argument("--no-vbyte", action="store_true")
    p.add_argument("--e2e-steps", type=int, default=12)
    p.add_argument("--e2e-streams", type=int, default=3, help="contexts (streams, host threads) of the e2e steps")
    p.add_argument("--profile-builds", type=int, default=0,
                   help="only run this many batched builds of the workload and exit (for profiler captures)")
    p.add_argument("--profile-vbyte", type=int, default=0,
                   help="only build the workload's grammar once, then run this many exports and imports of its "
                        "VByte form inside the profiler range (after --profile-warmup untimed ones) and exit")
    p.add_argument("--profile-strings", type=int, default=0,
                   help="with --profile-builds: only the first this many strings of the workload")
    p.add_argument("--write-traffic", default="",
                   help="ncu CSV (dram__bytes_read.sum, dram__bytes_write.sum per launch) of "
                        "--profile-builds 1 with the same --profile-strings / --profile-warmup: writes "
                        "profiles/traffic.json with DRAM bytes per algorithmic byte per kernel kind")
    p.add_argument("--traffic-command", default="", help="the ncu command recorded in profiles/traffic.json")
    p.add_argument("--profile-warmup", type=int, default=0,
                   help="with --profile-builds: builds run before the profiler range "
                        "(cudaProfilerStart/Stop; use ncu --profile-from-start off)")
    return p.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def workload(rank: int):
    # weak scaling: every rank parses its own batch of the same shape
    return li.bacterial_collection(seed=2 + 1000 * rank)


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


def cpu_baseline(coll, hf, target_s: float = 12.0):
    """The oracle as it stands, one host thread, on a bounded sample of the
    workload (its first strings, as many as fit about `target_s` seconds)."""
    from oracle import oracle as O
    probe = coll.subset([0])
    t = time.perf_counter()
    O.build(probe, hf)
    rate = probe.n / max(time.perf_counter() - t, 1e-6)
    take = max(1, min(coll.k, int(target_s * rate / max(1, probe.n))))
    sample = coll.subset(range(take))
    t = time.perf_counter()
    O.build(sample, hf)
    dt = time.perf_counter() - t
    return {"value": sample.n / dt / 1e9, "unit": "GB/s", "cores": 1, "kind": "oracle",
            "sample": f"first {take} of {coll.k} strings ({sample.n / 1e6:.1f} MB), one lcg oracle build, 1 thread",
            "seconds": dt}


def cpu_baseline_threaded(coll, hf, rate_1t: float, target_s: float = 10.0):
    """The oracle on every host core, as the paper's implementation runs in
    parallel: contiguous parts of a bounded sample, one oracle build per
    thread, merged in a tree by the oracle's MergeGrams (the result is the
    build of the whole sample).  ``rate_1t`` (bytes/s of one thread) sizes the
    sample to about ``target_s`` seconds."""
    from oracle import oracle as O
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else (os.cpu_count() or 1)
    per = coll.n / coll.k
    take = max(min(coll.k, cores), min(coll.k, int(target_s * rate_1t * cores / per)))
    sample = coll.subset(range(take))
    subs = O.split(sample, cores)
    t = time.perf_counter()
    g = O.build_parts(subs, hf)
    dt = time.perf_counter() - t
    if g.k != take:
        raise RuntimeError("threaded oracle lost strings")
    return {"value": sample.n / dt / 1e9, "unit": "GB/s", "cores": len(subs), "kind": "oracle",
            "sample": f"first {take} of {coll.k} strings ({sample.n / 1e6:.1f} MB) in {len(subs)} contiguous parts, "
                      f"one oracle build per thread, merged by the oracle MergeGrams in a tree",
            "seconds": dt}


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    hf = li.hash_family()
    coll = workload(0)
    from oracle import oracle as O
    O.build_library()
    sample = coll.subset(range(4))  # each step: a bounded 4-string sample (~20 MB)
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
        "config": {"workload": WORKLOAD, "sample": f"first 4 of {coll.k} strings ({sample.n / 1e6:.1f} MB) per step",
                   "parallelism": "single host thread"},
        "cpu_baseline": {"value": value, "unit": "GB/s", "cores": 1, "kind": "oracle",
                         "sample": f"first 4 of {coll.k} strings per step"},
        "e2e": {"value": value, "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


SERVING_WORKLOAD = ("serving stream: Poisson arrivals of strings with lognormal lengths (median 1 Mbp, sigma 1.5) "
                    "clipped to [10 kbp, 20 Mbp]; 80% windows of 8 seeded 20 Mbp genomes with 0.1-1% SNPs, "
                    "20% Zipf(1.1) byte text with copied blocks; 2 lanes, merged into a device-resident grammar")


def run_serving(hf, device: int, capacity_gbs: float, count: int = 300, loads=(0.1, 0.25, 0.5),
                mode: str = "merge") -> dict:
    """The serving loop on seeded streams, arrivals paced so that the offered
    input rate is ``load`` times ``capacity_gbs``: p50 / p99 latency and the
    input GB/s from first arrival to last completion, per load.  One server
    (two lanes) is warmed up on a stream of its own first, as a long-running
    server would be; each load then gets a stream with new content."""
    from paper_2411_12439_gb300 import serving

    import torch

    def make(seed):
        stream = li.serving_stream(seed=seed, count=count, rate_hz=1.0, n_bases=8, base_len=20_000_000,
                                   len_max=20_000_000)
        for item in stream:  # requests arrive in page-locked receive buffers
            item.data = torch.from_numpy(np.ascontiguousarray(item.data, dtype=np.uint8)).pin_memory().numpy()
        return stream

    backend = serving.CudaBackend(hf, device=device, lanes=2)
    srv = serving.Server(backend, lanes=2, max_batch_bytes=192 << 20, mode=mode)
    srv.start()
    warm = serving.replay(srv, make(50), time_scale=1e-4)
    srv.drain(warm, timeout=600)
    runs = []
    for i, load in enumerate(loads):
        stream = make(51 + i)
        mean_len = float(np.mean([r.data.shape[0] for r in stream]))
        rate = load * capacity_gbs * 1e9 / mean_len  # requests per second
        b0, e0 = len(srv.phases), len(srv.errors)
        reqs = serving.replay(srv, stream, time_scale=1.0 / rate)  # arrival_s was drawn at 1 request/s
        ok = srv.drain(reqs, timeout=600)
        st = serving.latency_stats(reqs)
        ph = srv.phases[b0:]
        runs.append({"requests": st.get("requests"), "load": load, "offered_gbs": load * capacity_gbs,
                     "gbs": st.get("gbs"), "p50_ms": 1e3 * st["p50_s"] if "p50_s" in st else None,
                     "p99_ms": 1e3 * st["p99_s"] if "p99_s" in st else None, "batches": len(ph),
                     "errors": len(srv.errors) - e0 + (0 if ok else 1),
                     "batch_ms": {k: 1e3 * float(np.mean([p.get(k, 0.0) for p in ph]))
                                  for k in ("gather", "build", "roots", "merge", "wait")}
                     if ph else None,
                     "builds_redone": sum(p.get("redone", 0) for p in ph),
                     "table_regrowths": sum(p.get("retries", 0) for p in ph)})
    srv.stop()
    return {"workload": SERVING_WORKLOAD, "max_batch_mb": 192, "lanes": 2, "mode": mode,
            "warmup": f"{count} requests of another seed", "resident_strings": backend.size(srv.resident),
            "runs": runs}


def run_ours(args):
    import torch
    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    from paper_2411_12439_gb300 import Context

    hf = li.hash_family()
    coll = workload(rank)
    d = torch.from_numpy(coll.data).to(f"cuda:{local}")
    # a stream of our own: the context launches on it and the timing events
    # are recorded on it (torch's default stream has handle 0, which would
    # make the context create a stream of its own)
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

    if args.profile_vbyte:
        offs = coll.offsets
        if args.profile_strings:
            offs = offs[:min(args.profile_strings, coll.k) + 1]
        g = ctx.build(d, offs)
        buf = torch.empty(g.vbyte_size(), dtype=torch.uint8, device=f"cuda:{local}")
        for _ in range(args.profile_warmup):
            g.export_vbyte(out=buf)
            ctx.import_vbyte(buf).free()
        torch.cuda.synchronize()
        torch.cuda.profiler.start()
        for _ in range(args.profile_vbyte):
            g.export_vbyte(out=buf)
            ctx.import_vbyte(buf).free()
        torch.cuda.synchronize()
        torch.cuda.profiler.stop()
        g.free()
        return 0

    if args.profile_builds:
        offs = coll.offsets
        if args.profile_strings:
            offs = offs[:min(args.profile_strings, coll.k) + 1]
        for _ in range(args.profile_warmup):
            ctx.build(d, offs).free()
        torch.cuda.synchronize()
        torch.cuda.profiler.start()
        for _ in range(args.profile_builds):
            ctx.build(d, offs).free()
        torch.cuda.synchronize()
        torch.cuda.profiler.stop()
        return 0

    for _ in range(args.warmup):
        ctx.build(d, coll.offsets).free()
    tuned = None
    if not args.no_autotune:
        # launch and sizing parameters picked by the project's autotuner on this workload
        from paper_2411_12439_gb300 import autotune
        rep = autotune.autotune(ctx, d, coll.offsets, reps=5, sweeps=1)
        tuned = {"tuning": rep["tuning"], "ms": rep["ms"], "trials": len(rep["trials"])}

    # ---- timed region: inputs resident in HBM (320 MB > L2, no flush needed).
    #      Only the parse launches (the kernel with most device time) carry
    #      CUDA events here; the per-kernel breakdown is taken afterwards.
    #      Each build is one launch of the CUDA graph of its planned rounds
    #      (captured by the first build of the shape, outside the timed region).
    ctx.set_kernel_timing(2)
    ctx.set_graph(not args.no_graph)
    for _ in range(2):
        ctx.build(d, coll.offsets).free()
    graph_modes = []
    kt = {}
    launches = 0
    sampler = ClockSampler(local)
    barrier()
    torch.cuda.synchronize()
    sampler.start()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        g = ctx.build(d, coll.offsets)
        for name, v in ctx.last_kernel_times().items():
            acc = kt.setdefault(name, {"launches": 0, "ms": 0.0, "bytes": 0.0})
            for key in acc:
                acc[key] += v[key]
        launches += ctx.last_build_stats()["kernel_launches"]
        graph_modes.append(ctx.last_build_stats()["graph"])
        g.free()  # a serving loop releases each grammar; the memory returns to the pool in stream order
    e1.record(stream)
    torch.cuda.synchronize()
    barrier()
    clocks = sampler.stop()
    ms = max_over_ranks(e0.elapsed_time(e1)) / args.steps
    stats = ctx.last_build_stats()
    # per-kernel breakdown (every launch timed) over separate builds, as launches
    ctx.set_graph(False)
    ctx.set_kernel_timing(1)
    breakdown = {}
    per_round = None
    for _ in range(max(1, min(args.steps, 5))):
        ctx.build(d, coll.offsets).free()
        rs = ctx.last_build_stats()["per_round"]
        if per_round is None or len(per_round) != len(rs):
            per_round = [{"symbols": r["n"], "bytes_per_symbol": 1 if i == 0 else 4, "phrases": r["phrases"],
                          "g": r["g"], "G": r["G"], "ms": [], "parse_ms": []}
                         for i, r in enumerate(rs)]
        for pr, r in zip(per_round, rs):
            pr["ms"].append(r["round_ms"])
            pr["parse_ms"].append(r["parse_ms"])
        for name, v in ctx.last_kernel_times().items():
            acc = breakdown.setdefault(name, {"launches": 0, "ms": 0.0, "builds": 0})
            acc["launches"] += v["launches"]
            acc["ms"] += v["ms"]
        for acc in breakdown.values():
            acc["builds"] += 1
    ctx.set_kernel_timing(0)
    value = world * coll.n / (ms / 1e3) / 1e9
    rounds_line = []
    peak_gbs, _ = measured_peak()
    for i, pr in enumerate(per_round or []):
        rms = float(np.median(pr["ms"]))
        # algorithmic bytes of the round: its sequence read (bytes in round 1;
        # ranks and their fingerprints later), the next sequence and its
        # fingerprints written, and the new rules (rhs, offsets, F)
        alg = (pr["symbols"] * (1 if i == 0 else 8) + 8 * pr["phrases"] + 4 * pr["G"] + 12 * pr["g"])
        rounds_line.append({"round": i + 1, "symbols": int(pr["symbols"]), "ms": rms,
                            "parse_ms": float(np.median(pr["parse_ms"])),
                            "gbs": pr["symbols"] * pr["bytes_per_symbol"] / (rms / 1e3) / 1e9 if rms > 0 else None,
                            "alg_bytes": int(alg),
                            "hbm_frac": alg / (rms / 1e3) / 1e9 / peak_gbs if rms > 0 else None})

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

    # ---- the VByte form of the batch's grammar (rules and rule lengths in
    #      VByte, Sec. 4 resource usage): sizes, export / import times, and the
    #      encode / decode kernels against the HBM peak; the import of the
    #      export must give back the same grammar
    vbyte_line = None
    if not args.no_vbyte:
        g = ctx.build(d, coll.offsets)
        packed = g.packed_size()
        nbytes = g.vbyte_size()
        buf = torch.empty(nbytes, dtype=torch.uint8, device=f"cuda:{local}")
        ex_t, im_t = [], []
        roundtrip = None
        for _ in range(3):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            g.export_vbyte(out=buf)
            ex_t.append(time.perf_counter() - t0)
            t0 = time.perf_counter()
            h = ctx.import_vbyte(buf)
            im_t.append(time.perf_counter() - t0)
            if roundtrip is None:
                a, b = g.export(), h.export()
                roundtrip = all(np.array_equal(x[key], y[key]) for x, y in zip(a["levels"], b["levels"])
                                for key in ("rhs_off", "rhs", "F")) and len(a["levels"]) == len(b["levels"]) \
                    and np.array_equal(a["c_rank"], b["c_rank"]) and np.array_equal(a["c_level"], b["c_level"])
            h.free()
        # one more pass with every launch timed, for the kernel breakdown
        ctx.set_kernel_timing(1)
        enc, dec = [], []
        for _ in range(2):
            g.export_vbyte(out=buf)
            enc.append(ctx.last_kernel_times())
            ctx.import_vbyte(buf).free()
            dec.append(ctx.last_kernel_times())
        ctx.set_kernel_timing(0)
        head = buf[:24].cpu().numpy().view(np.uint64)
        nl = int(head[2])
        lv = buf[24:24 + 32 * nl].cpu().numpy().view(np.uint64).reshape(nl, 4)
        rules_u32 = int(sum(4 * int(G_) + 8 * (int(g_) + 1) for g_, G_, _, _ in lv))
        rules_vb = int(sum(int(a_) + int(b_) for _, _, a_, b_ in lv))
        g.free()

        def kern(recs):
            out = {}
            for name in recs[0]:
                ms = float(np.median([r[name]["ms"] for r in recs]))
                byt = recs[0][name]["bytes"]
                gbs = byt / (ms / 1e3) / 1e9 if ms > 0 else None
                out[name] = {"ms": ms, "launches": recs[0][name]["launches"], "alg_bytes": int(byt), "gbs": gbs,
                             "frac": gbs / peak_gbs if gbs else None}
            return out

        vbyte_line = {"packed_bytes": packed, "vbyte_bytes": nbytes, "ratio": nbytes / packed,
                      "rules_u32_bytes": rules_u32, "rules_vbyte_bytes": rules_vb, "rules_ratio": rules_vb / rules_u32,
                      "export_ms": float(np.median(ex_t)) * 1e3, "import_ms": float(np.median(im_t)) * 1e3,
                      "export_kernels": kern(enc), "import_kernels": kern(dec), "roundtrip_equal": bool(roundtrip),
                      "timing": "host clock around lcg_export_vbyte / lcg_import_vbyte (device buffer; both "
                                "synchronise; kernel timing off); kernels in separate calls, CUDA events per "
                                "launch; algorithmic bytes: k_vb_write "
                                "values read + stream written, k_vb_dwrite stream read + values written, the "
                                "counting kernels their input read"}

    # ---- end to end through the public API: pinned host input, the whole
    #      grammar to a pinned host buffer in its packed form every step.
    #      Steps run on `--e2e-streams` contexts (each with its own stream and
    #      host thread, as a serving process would), so that one step's copies
    #      overlap another step's kernels.
    hd = torch.from_numpy(coll.data).pin_memory()
    lanes = max(1, args.e2e_streams)
    streams = [stream] + [torch.cuda.Stream(device=local) for _ in range(lanes - 1)]
    ectx = [ctx] + [Context(hf, device=local, stream=s.cuda_stream) for s in streams[1:]]
    outs = []
    for c in ectx:
        c.set_tuning(**ctx.tuning())
        c.set_graph(not args.no_graph)  # host input goes through the context's upload buffer
        for _ in range(2):  # a plan, then the graph's capture
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

    e2e_pass([2] * lanes)  # untimed: the lanes' steps running together once, as they will when timed
    barrier()
    t0 = time.perf_counter()
    e2e_pass(per_lane)
    if errors:
        raise RuntimeError("end-to-end step failed: " + errors[0])
    e2e_s = max_over_ranks((time.perf_counter() - t0) / e2e_steps)
    e2e = {"value": world * coll.n / e2e_s / 1e9, "unit": "GB/s", "h2d_bytes_per_step": int(coll.n),
           "d2h_bytes_per_step": max(d2h_seen), "ms_per_step": e2e_s * 1e3, "steps": e2e_steps, "streams": lanes,
           "result": "grammar in its packed form (lcg_export_packed) in page-locked host memory",
           "timing": "host clock from the first step's start to the last step's grammar in host memory"}
    for c in ectx[1:]:
        c.close()
    ctx.set_graph(False)

    # ---- plain form: one string per launch sequence, against the resident grammar
    plain = None
    if not args.no_plain:
        offs = coll.offsets.astype(np.int64)
        torch.cuda.synchronize()
        p0 = torch.cuda.Event(enable_timing=True)
        p1 = torch.cuda.Event(enable_timing=True)
        p0.record(stream)
        R = ctx.build(d[offs[0]:offs[1]], np.array([0, offs[1] - offs[0]], dtype=np.uint64))
        for j in range(1, coll.k):
            ctx.build_into(R, d[offs[j]:offs[j + 1]], np.array([0, offs[j + 1] - offs[j]], dtype=np.uint64))
        p1.record(stream)
        torch.cuda.synchronize()
        pms = max_over_ranks(p0.elapsed_time(p1))
        R.free()
        pv = world * coll.n / (pms / 1e3) / 1e9
        plain = {"value": pv, "unit": "GB/s", "ms_per_step": pms, "batched_over_plain": value / pv,
                 "form": "one string per launch sequence, each parsed against the resident grammar"}

    # ---- roofline of the kernel with the largest device time
    peak, peak_kind = measured_peak()
    dom = max(kt.items(), key=lambda kv: kv[1]["ms"]) if kt else None
    roofline = None
    if dom:
        name, v = dom
        per_launch_bytes = v["bytes"] / v["launches"]
        per_launch_s = v["ms"] / v["launches"] / 1e3
        achieved = per_launch_bytes / per_launch_s / 1e9
        ratio = profiled_traffic(name)
        roofline = {"bound": "hbm", "kernel": name, "achieved": achieved, "peak": peak, "unit": "GB/s",
                    "frac": achieved / peak, "peak_source": peak_kind,
                    "traffic": (ratio * per_launch_bytes) if ratio is not None else None,
                    "alg_bytes_per_launch": per_launch_bytes, "launches": v["launches"],
                    "timing": "CUDA events around every parse launch of the timed builds",
                    "share_of_kernel_time": (breakdown[name]["ms"] / sum(x["ms"] for x in breakdown.values()))
                    if name in breakdown else None}

    if rank != 0:
        return 0
    cpu = cpu_threaded = None
    if world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(coll, hf)
        cpu_threaded = cpu_baseline_threaded(coll, hf, cpu["value"] * 1e9)
    serving_line = None
    if world == 1 and not args.no_serving:
        serving_line = run_serving(hf, local, value)
    line = {
        "metric": METRIC, "value": value, "unit": "GB/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u8/u32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "strings": coll.k, "input_bytes": int(coll.n),
                   "rounds": stats["rounds"], "l2": "inputs larger than L2 (320 MB > 129 MB), no flush",
                   "autotuned": tuned,
                   "cuda_graph": ("every timed build a graph launch" if graph_modes and min(graph_modes) == 2
                                  else f"graph modes of the timed builds: {graph_modes}"),
                   "parallelism": f"dp{world}" if world > 1 else "single GPU"},
        "e2e": e2e, "gpu_launches": int(launches), "clocks": clocks, "roofline": roofline,
        "cpu_baseline": cpu, "cpu_baseline_threaded": cpu_threaded, "plain": plain, "serving": serving_line,
        "rounds": rounds_line, "postprocess": post, "vbyte": vbyte_line,
        "path_roofline": ({"alg_bytes_per_step": sum(r["alg_bytes"] for r in rounds_line),
                           "gbs": sum(r["alg_bytes"] for r in rounds_line) / (ms / 1e3) / 1e9,
                           "frac": sum(r["alg_bytes"] for r in rounds_line) / (ms / 1e3) / 1e9 / measured_peak()[0],
                           "note": "all rounds' algorithmic bytes over the timed step (HBM peak as in roofline)"}
                          if rounds_line else None),
        "kernels": {k: {"launches": v["launches"] // v["builds"], "ms_per_step": v["ms"] / v["builds"]}
                    for k, v in sorted(breakdown.items(), key=lambda kv: -kv[1]["ms"])},
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
    """profiles/traffic.json from an ncu capture of one profiled build: the
    algorithmic bytes of the same build come from the library's kernel timing."""
    import torch
    from paper_2411_12439_gb300 import Context
    dram = _ncu_dram_bytes(args.write_traffic)
    hf = li.hash_family()
    coll = workload(0)
    offs = coll.offsets[:min(args.profile_strings, coll.k) + 1] if args.profile_strings else coll.offsets
    d = torch.from_numpy(coll.data).cuda()
    torch.cuda.synchronize()
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    ctx = Context(hf, device=0, stream=stream.cuda_stream)
    for _ in range(args.profile_warmup):
        ctx.build(d, offs).free()
    ctx.set_kernel_timing(True)
    ctx.build(d, offs).free()
    kt = ctx.last_kernel_times()
    kernels = {}
    for kind, v in dram.items():
        if kind in kt and kt[kind]["bytes"] > 0:
            kernels[kind] = {"launches": v["launches"], "dram_bytes": v["dram_bytes"], "alg_bytes": kt[kind]["bytes"],
                             "dram_bytes_per_alg_byte": v["dram_bytes"] / kt[kind]["bytes"]}
    out = {"source_hash": kernel_source_hash(), "command": args.traffic_command,
           "workload": WORKLOAD + (f" (first {args.profile_strings} strings)" if args.profile_strings else ""),
           "input_bytes": int(offs[-1] - offs[0]), "kernels": kernels}
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
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
