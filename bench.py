"""Benchmark: GWCP race analysis throughput (trace events/s) on one GB300 per rank.

Headline workload: 256 blocks x 1024 threads analysed at warp granularity (8192 agents,
clocks of 8192 entries held as 256-entry tiles), 200M events, 64M addresses drawn
Zipf(1.05), 1% scoped synchronisation (70% block / 30% device scope), ~0.1% planted
races; seeded synthetic. One step = one full analysis (gwcp_compute_order: decode and
validate, epochs, critical sections, clock propagation, access grouping, per-location
check, race sort) over the resident trace. Beside it: the 8-block, 64-warp, 10M-event
workload (with the ranker and the compressed-clock mode), the tiny 64-thread trace,
the 512-trace batch and the Poisson-served stream.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Multi-GPU: the analysis of one trace does not shard; N ranks run N independent
replicas (weak scaling, no collective on the data path).
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

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)
sys.path.insert(1, os.path.join(ROOT, "tests"))  # race digests and ranker metrics (measurement helpers)

WORKLOAD = "256blk_8192warp_200M"
C2 = "8blk_64warp_10M"
TINY = "tiny_1blk_64thr_10k"
METRIC = "trace events/sec, race set bit-exact; batched/served vs plain; p50/p99 lat"
SEED = 1
DIGESTS = os.path.join(ROOT, "tests", "golden", "oracle_digests.json")


T0 = time.perf_counter()


CLOCK_MODES = {"auto": 0, "dense": 1, "tiles": 2, "compressed": 3}  # gwcp.CLOCKS_*


def log(msg):
    print(f"[bench] {msg}", file=sys.stderr, flush=True)


def read_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons, sampled every 200 ms; summary() keeps the
    samples taken between mark_start() and mark_end() (the timed region)."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    t_start = None
    t_end = None

    def mark_start(self):
        self.t_start = time.perf_counter()

    def mark_end(self):
        self.t_end = time.perf_counter()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append((time.perf_counter(), line.strip()))

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for t, ln in self.lines:
            if self.t_start is not None and (t < self.t_start or (self.t_end is not None and t > self.t_end + 0.2)):
                continue
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx = float(parts[2])
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def source_hash(names):
    h = hashlib.sha256()
    for n in names:
        with open(os.path.join(ROOT, "paper_2111_12478_gb300", "csrc", n), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


KERNEL_SOURCES = {"k_prop_wide": ["gwcp_wide.cu"], "k_propagate": ["gwcp_propagate.cu"], "k_wc_check": ["gwcp_wide.cu"]}


def traffic_for(kernel, workload):
    """DRAM bytes per launch of a kernel on a workload from the committed ncu summary
    (profiles/traffic.json), if the kernel's source has not changed since the counters
    were taken; else None."""
    try:
        with open(os.path.join(ROOT, "profiles", "traffic.json")) as f:
            t = json.load(f)
        e = t.get(f"{kernel}@{workload}")
        if e and e.get("source_sha") == source_hash(KERNEL_SOURCES.get(kernel, [])):
            return float(e["dram_bytes_per_launch"])
    except Exception:
        pass
    return None


def load_digests():
    try:
        with open(DIGESTS) as f:
            return json.load(f)
    except Exception:
        return None


def digest_check(ev, races, workload, seed):
    """The race set against the oracle's, through the stored oracle digests of this
    workload and seed (tests/golden/oracle_digests.json): the races whose later access
    lies in the oracle's prefix, bucket by bucket, after checking that the trace is the
    one the oracle ran on."""
    from race_digest import bucket_digests, trace_sha256

    d = load_digests()
    for e in (d or {}).get("c3", []):
        if e["workload"] == workload and e["seed"] == seed and len(ev) >= e["events"]:
            same_trace = trace_sha256(ev, e["events"]) == e["trace_sha256"]
            same = bucket_digests(races, e["bucket"], e["events"] // e["bucket"]) == e["buckets"]
            return {"events_checked": e["events"], "identical": bool(same_trace and same), "trace_matches": same_trace,
                    "how": f"stored oracle digests per {e['bucket']}-event bucket of the later access"}
    return None


def prop_roofline(kernel, workload, ms, cnt, W, tiles, peak, peak_kind):
    """Roofline of the clock propagation with the method's algorithmic bytes:
    a vector-clock join of width W reads two clocks and writes one (12 W bytes), each
    release-loop record visit compares one epoch (8 bytes). With clocks held as 256-entry
    tiles the walkers join only the tiles that differ, so the bytes they must move are the
    1 KB tiles read and written plus the epoch compares; that tile-sparse figure is the
    roofline's `achieved` and `frac`, and the dense figure (which can exceed the peak, since
    shared and unchanged tiles are never moved) is reported beside it."""
    joins, visits = cnt["joins"], cnt["loop_visits"]
    dense = 12.0 * W * joins + 8.0 * visits
    dense_out = {"algorithmic_bytes": dense, "achieved": dense / (ms / 1e3) / 1e9,
                 "frac": dense / (ms / 1e3) / 1e9 / peak,
                 "bytes_per_unit": "12*W per join (W = %d) + 8 per release-loop visit" % W}
    if tiles:
        b = 1024.0 * (cnt["tiles_read"] + cnt["tiles_written"]) + 8.0 * visits
        unit = "1 KB per tile read or written + 8 per release-loop visit"
    else:
        b, unit = dense, dense_out["bytes_per_unit"]
    ach = b / (ms / 1e3) / 1e9
    out = {"bound": "hbm", "kernel": kernel, "achieved": ach, "peak": peak, "unit": "GB/s", "frac": ach / peak,
           "peak_kind": f"{peak_kind} hbm_gbs", "traffic": traffic_for(kernel, workload), "algorithmic_bytes": b,
           "avg_ms": ms, "bytes_per_unit": unit, "joins": joins, "loop_visits": visits}
    if tiles:
        out["tiles_read"], out["tiles_written"] = cnt["tiles_read"], cnt["tiles_written"]
        out["dense_equivalent"] = dense_out
    return out


def check_roofline(ms, prof_bytes, cnt, n_races, workload, peak, peak_kind):
    """Roofline of the per-location check: the bytes it reads per access (sorted index,
    record fields, run flags), 8 bytes per partner test and 16 per race written."""
    b = prof_bytes + 8.0 * cnt["partner_tests"] + 16.0 * n_races
    ach = b / (ms / 1e3) / 1e9
    tr = traffic_for("k_wc_check", workload)
    return {"bound": "hbm", "kernel": "k_wc_check", "achieved": ach, "peak": peak, "unit": "GB/s", "frac": ach / peak,
            "peak_kind": f"{peak_kind} hbm_gbs", "traffic": tr, "algorithmic_bytes": b, "avg_ms": ms,
            "dram_frac": (tr / (ms / 1e3) / 1e9 / peak) if tr else None}


def replica_reduce(t_local: float, events_local: int, dist=None, device="cpu"):
    """Replicas (one independent trace per rank, no collective on the data path): the job's
    time is the slowest rank's, its work the events of all ranks. Returns (t_max, events)."""
    if dist is None:
        return t_local, events_local
    import torch

    t = torch.tensor([t_local], dtype=torch.float64, device=device)
    e = torch.tensor([float(events_local)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(e, op=dist.ReduceOp.SUM)
    return float(t.item()), int(e.item())


def bench_batched(args, local, torch, gwcp, tracegen, np):
    """The batched workload (512 independent traces, 10k-5M events, 64-4096 warps; inputs
    resident on the device): the plain path (one context, one trace after another) against
    the pool (lanes autotuned on every 8th trace). Wall-clock seconds with the device
    synchronised on both sides; the pool's race sets must equal the plain path's."""
    specs = tracegen.many_specs(SEED, **tracegen.BATCH_WORKLOAD)
    traces = tracegen.generate_many(specs, threads=os.cpu_count() or 8)
    n_total = int(sum(len(ev) for ev, _ in traces))
    dev = [torch.from_numpy(ev.view(np.uint8)).to(f"cuda:{local}") for ev, _ in traces]
    geos = [geo.astuple() for _, geo in traces]
    ctx = gwcp.Context(local)

    def plain(outs=None):
        out = []
        for i, (d, g) in enumerate(zip(dev, geos)):
            ctx.load_trace(d, *g)
            ctx.compute_order()
            out.append(ctx.report_races(out=outs[i]) if outs else ctx.report_races())
        return out

    first = plain()  # sizes the context's buffers and the result arrays
    # result arrays are allocated once and reused by every timed pass (plain and pool), as a
    # caller analysing batch after batch would
    outs = [np.zeros((max(len(r), 1), 2), dtype=np.uint64) for r in first]
    plain(outs)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    ref = plain(outs)
    torch.cuda.synchronize()
    t_plain = time.perf_counter() - t0
    ref = [r.copy() for r in ref]  # the pool writes into the same arrays next
    ctx.close()
    pool = gwcp.Pool(local, lanes=args.lanes)
    items = list(zip(dev, geos))
    best, tune = pool.autotune(items[::8])
    pack = pool.settings()[1]
    caps = [len(r) for r in ref]
    pool.run_batch(items, caps, outs)  # warm-up: lanes size their buffers
    times, got = [], None
    for _ in range(args.batch_steps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        got = pool.run_batch(items, caps, outs)
        torch.cuda.synchronize()
        times.append(time.perf_counter() - t0)
    identical = all(rc == 0 and np.array_equal(r, w) for (r, rc, _), w in zip(got, ref))
    pool.close()
    # the oracle on the short, narrow traces of the batch
    exact = None
    if not args.no_cpu_baseline:
        from oracle import oracle

        idx = [i for i, (ev, g) in enumerate(traces) if len(ev) <= 60_000 and g.num_agents <= 1024][:12]
        exact = all(np.array_equal(oracle.run(traces[i][0], *geos[i]).races, ref[i]) for i in idx)
        exact = {"traces_checked": len(idx), "identical": bool(exact)}
    t_b = statistics.median(times)
    return {"workload": "512 traces, 10k-5M events (log-uniform), 64-4096 warps, 64-warp 10M-event op mix",
            "traces": len(traces), "events": n_total, "lanes": best, "autotune_s": tune, "pack_walkers": pack,
            "value": n_total / t_b, "unit": "events/s", "s_per_batch": t_b, "batches_timed": len(times),
            "plain": {"value": n_total / t_plain, "s": t_plain, "path": "one context, traces in sequence"},
            "speedup_vs_plain": t_plain / t_b, "race_sets_identical_to_plain": identical,
            "oracle_sample": exact, "n_races": int(sum(len(r) for r in ref)),
            "inputs": "device-resident", "timing": "wall clock, device synchronised on both sides"}


def bench_served(args, local, torch, gwcp, tracegen, np, lanes, pack=True):
    """The served workload: requests arriving as a Poisson process at 200/s, 10k-20M
    events each (prefixes of one 20M-event trace per width class, in pinned host memory,
    copied to the device by the pool), races copied back to host memory. The same arrival
    schedule runs on the pool's lanes and on a single lane (the plain path, one trace at a
    time); latency = completion - arrival on the pool's clock."""
    cfg = tracegen.SERVE_WORKLOAD
    base = tracegen.generate_many(tracegen.serve_base_specs(SEED, cfg["n_max"]), threads=os.cpu_count() or 8)
    pinned = [torch.from_numpy(ev.view(np.uint8)).pin_memory() for ev, _ in base]
    geos = [g.astuple() for _, g in base]
    arr, wid, lens = tracegen.serve_requests(SEED, args.serve_requests, cfg["rate"], cfg["n_min"], cfg["n_max"],
                                            len(base))
    pool = gwcp.Pool(local, lanes=32, pack_walkers=pack)
    # lanes and walker packing tuned on a sample of this workload's own requests
    sample = [(pinned[wid[i]][: int(lens[i]) * 16], geos[wid[i]]) for i in range(0, len(arr), max(1, len(arr) // 32))]
    lanes, _ = pool.autotune(sample)
    pack = pool.settings()[1]
    # result arrays are recycled, as a server would: a free list per power-of-two size
    free, free_lock = {}, threading.Lock()

    def take(rows):
        k = 1 << max(10, int(rows - 1).bit_length())
        with free_lock:
            lst = free.get(k)
            if lst:
                return lst.pop()
        return np.empty((k, 2), dtype=np.uint64)

    def give(a):
        with free_lock:
            free.setdefault(a.shape[0], []).append(a)

    def schedule(active):
        pool.set_active_lanes(active)
        # warm the lanes on a few of the longest requests, then serve the schedule
        big = np.argsort(-lens)[: active]
        for i in big:
            pool.wait(pool.submit(pinned[wid[i]][: int(lens[i]) * 16], geos[wid[i]], 0))
        tickets = [None] * len(arr)
        bufs = [None] * len(arr)
        start = pool.now() + 0.02

        def submit_all():
            for i in range(len(arr)):
                dt = start + arr[i] - pool.now()
                if dt > 0:
                    time.sleep(dt)
                n = int(lens[i])
                buf = take(3 * n + 1024)
                bufs[i] = buf
                tickets[i] = pool.submit(pinned[wid[i]][: n * 16], geos[wid[i]], 3 * n + 1024, out=buf)

        th = threading.Thread(target=submit_all)
        th.start()
        infos = []
        for i in range(len(arr)):
            while tickets[i] is None:
                time.sleep(0.0005)
            races, info = pool.wait(tickets[i])
            infos.append((info.rc, info.n_races, info.t_submit, info.t_done, info.t_first_race))
            give(bufs[i])
            bufs[i] = None
        codes = {}
        for rc, *_ in infos:
            codes[rc] = codes.get(rc, 0) + 1
        th.join()
        lat = np.array([d - s for _, _, s, d, _ in infos])
        # time to first race: the check's stamp of the request's first race (GPU global timer on
        # the pool's clock), before the rest of the check, the race sort and the copy-out
        ttfr = np.array([f - s for _, n, s, _, f in infos if n > 0 and f > 0])
        span = max(d for _, _, _, d, _ in infos) - min(s for _, _, s, _, _ in infos)
        ok = sum(1 for rc, *_ in infos if rc == 0)
        return {"lanes": active, "value": float(lens.sum()) / span, "unit": "events/s",
                "p50_latency_s": float(np.percentile(lat, 50)), "p99_latency_s": float(np.percentile(lat, 99)),
                "mean_latency_s": float(lat.mean()), "span_s": span, "requests_ok": ok,
                "p50_time_to_first_race_s": float(np.percentile(ttfr, 50)) if len(ttfr) else None,
                "p99_time_to_first_race_s": float(np.percentile(ttfr, 99)) if len(ttfr) else None,
                "result_codes": {str(k): v for k, v in codes.items()},
                "n_races": int(sum(n for _, n, *_ in infos))}

    served = schedule(max(lanes, 1))
    plain = schedule(1)
    # the same requests at 60% of the served capacity just measured: the serving loop's own
    # latency, without the queue an over-capacity arrival rate builds up
    n2 = min(len(arr), 400)
    rate2 = 0.6 * served["value"] / float(lens.mean())
    arr_full, wid_full, lens_full = arr, wid, lens
    rng = np.random.default_rng(SEED + 1)
    arr = np.cumsum(rng.exponential(1.0 / rate2, size=n2))
    wid, lens = wid_full[:n2], lens_full[:n2]
    sustainable = schedule(max(lanes, 1))
    sustainable["rate_per_s"] = rate2
    sustainable["requests"] = n2
    arr, wid, lens = arr_full, wid_full, lens_full
    pool.close()
    return {"workload": f"Poisson {cfg['rate']:.0f} req/s, 10k-20M events (log-uniform), 64-4096 warps",
            "pack_walkers": pack,
            "requests": len(arr), "offered_events_per_s": float(lens.sum()) / float(arr[-1]),
            **served, "plain": plain, "speedup_vs_plain": served["value"] / plain["value"],
            "at_60pct_capacity": sustainable,
            "inputs": "pinned host memory; H2D copy and race D2H inside each request"}


def bench_ranker(args, local, torch, gwcp, np, ev, geo, dev):
    """The trained address ranker on the main workload: the check's timeline (time from its
    start to the first race and to 50% / 90% / all races) and the share of racy locations
    among the first 10% of locations checked, in location order and in ranked order. The
    ranker's features, scores and re-sort run beside the propagation; the race sets of the
    two orders must be identical."""
    import ranker_metrics
    from paper_2111_12478_gb300 import ranker

    theta = ranker.load_weights()
    if theta is None:
        return {"unavailable": "no trained weights (tests/train_ranker.py writes them)"}
    out, sets = {}, {}
    for name, t in (("location_order", None), ("ranked", theta)):
        ctx = gwcp.Context(local, timeline=True, profile=True)
        ctx.set_ranker(t)
        ctx.load_trace(dev, *geo.astuple())
        summ, steps = [], []
        for rep in range(args.warmup + 5):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            ctx.compute_order()
            n = ctx.race_count()
            dt = time.perf_counter() - t0
            if rep >= args.warmup:
                steps.append(dt)
                summ.append(ranker.timeline_summary(*ctx.check_timeline()))
        races = ctx.report_races()
        _, keys = ctx.location_features()
        sets[name] = races
        prof = {k: round(ms, 4) for k, ms, _ in ctx.profile()}
        ctx.close()
        med = {k: float(np.median([s_[k] for s_ in summ])) for k in summ[0] if k.endswith("_us")}
        out[name] = {**med, "races_in_first_10pct_chunks": summ[-1]["races_in_first_10pct_chunks"],
                     "racy_location_recall_first_10pct": ranker_metrics.racy_location_recall(
                         ev, geo.agents_per_block, races, keys.cpu().numpy().view(np.uint64), 0.1),
                     "ms_per_step": 1e3 * float(np.median(steps)), "h_rank_ms": prof.get("h_rank"),
                     "i_check_ms": prof.get("i_check"), "n_races": int(n)}
    out["race_sets_identical"] = bool(np.array_equal(sets["location_order"], sets["ranked"]))
    out["note"] = "times in microseconds from the check's start (globaltimer); ranker: BF16 MLP 16-64-64-1"
    return out


def bench_compressed(args, local, torch, gwcp, np, geo, dev, races):
    """The paper's memory mode on the main workload: forced compression at barriers and the
    clock versions the check reads stored in block/warp compressed form. Reports the bytes
    of the versions (dense, as stored, as reserved), the time per step and whether the race
    set equals the dense run's."""
    stream = torch.cuda.Stream(device=local)
    n_ev = dev.numel() // 16

    def measure(ctx):
        ctx.load_trace(dev, *geo.astuple(), stream=stream)
        for _ in range(max(2, args.warmup)):  # the first run sizes the version pool
            ctx.compute_order(stream=stream)
            ctx.race_count(stream=stream)
        steps, prof = [], {}
        for _ in range(5):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            ctx.compute_order(stream=stream)
            e1.record(stream)
            ctx.race_count(stream=stream)
            steps.append(e0.elapsed_time(e1))
            for name, ms_, _ in ctx.profile():
                prof.setdefault(name, []).append(ms_)
        ms = float(np.median(steps))
        out = {"ms_per_step": ms, "events_per_s": n_ev / (ms / 1e3),
               "phases_ms": {k: round(float(np.median(v)), 4) for k, v in prof.items()
                             if k in ("c_forced", "g_propagate", "i_check")},
               "race_set_identical_to_dense": bool(np.array_equal(ctx.report_races(stream=stream), races)),
               "counters": {k: v for k, v in ctx.counters().items() if k in ("loop_visits", "joins", "clock_versions")}}
        return out

    plain = gwcp.Context(local, profile=True)
    plain.set_clock_mode(gwcp.CLOCKS_DENSE)
    out_plain = measure(plain)
    plain.close()
    forced = gwcp.Context(local, profile=True, forced_barrier=True)
    forced.set_clock_mode(gwcp.CLOCKS_DENSE)
    out_forced = measure(forced)
    forced.close()
    ctx = gwcp.Context(local, profile=True)
    ctx.set_clock_mode(gwcp.CLOCKS_COMPRESSED)
    out = measure(ctx)
    cb = ctx.clock_bytes()
    ctx.close()
    out.update({"version_bytes": cb, "stored_over_dense": cb["stored"] / cb["dense"],
                "reserved_over_dense": cb["reserved"] / cb["dense"], "forced_barrier_dense": out_forced, "dense": out_plain,
                "note": "clock versions only; release snapshots stay dense"})
    return out


def run_steps(ctx, stream, steps, torch, gwcp, on_step=None):
    """K analyses of the resident trace, each bracketed by CUDA events on its stream, and
    the step's result read (the race count, which synchronises). Returns (per-step ms,
    per-phase [ms, bytes, count], races, launches)."""
    torch.cuda.synchronize()
    launches0 = gwcp.launch_count()
    prof, per_step, n_races = {}, [], 0
    for _ in range(steps):
        s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s0.record(stream)
        ctx.compute_order(stream=stream)
        s1.record(stream)
        n_races = ctx.race_count(stream=stream)
        per_step.append((s0, s1))
        for name, ms, by in ctx.profile():
            a = prof.setdefault(name, [0.0, 0.0, 0])
            a[0] += ms
            a[1] += by
            a[2] += 1
    torch.cuda.synchronize()
    return [a.elapsed_time(b) for a, b in per_step], prof, n_races, gwcp.launch_count() - launches0


def bench_c2(args, local, torch, gwcp, tracegen, np, peak, peak_kind):
    """The 8-block x 256-thread workload at warp granularity (64 agents, 10M events, 1M
    addresses Zipf(1.1), 3% synchronisation): events/s over the device-resident trace,
    phases, the propagation's and the check's rooflines, the whole race set against the
    oracle (which is also its CPU baseline), then the ranker and the compressed-clock mode
    on the same trace."""
    ev, geo, _ = tracegen.generate(SEED, workload=C2)
    dev = torch.from_numpy(ev.view(np.uint8).copy()).to(f"cuda:{local}")
    stream = torch.cuda.Stream(device=local)
    ctx = gwcp.Context(local, profile=True)
    ctx.load_trace(dev, *geo.astuple(), stream=stream)
    for _ in range(args.warmup):
        ctx.compute_order(stream=stream)
    ms, prof, n_races, launches = run_steps(ctx, stream, args.c2_steps, torch, gwcp)
    races = ctx.report_races(stream=stream)
    cnt = ctx.counters()
    ctx.close()
    phases = {k: (v[0] / v[2], v[1] / v[2]) for k, v in prof.items()}
    med = statistics.median(ms)
    out = {"workload": C2, "events": int(len(ev)), "agents": geo.num_agents, "value": len(ev) / (med / 1e3),
           "unit": "events/s", "ms_per_step": med, "steps": args.c2_steps, "warmup": args.warmup,
           "n_races": int(n_races), "gpu_launches_per_step": launches / max(1, args.c2_steps),
           "phases_ms": {k: round(v[0], 4) for k, v in sorted(phases.items(), key=lambda kv: -kv[1][0])},
           "roofline": prop_roofline("k_propagate", C2, phases["g_propagate"][0], cnt, geo.num_agents, False, peak,
                                     peak_kind),
           "roofline_check": check_roofline(phases["i_check"][0], phases["i_check"][1], cnt, len(races), C2, peak,
                                            peak_kind) if "i_check" in phases else None}
    if not args.no_cpu_baseline:
        from oracle import oracle

        t0 = time.perf_counter()
        want = oracle.run(ev, *geo.astuple()).races
        dt = time.perf_counter() - t0
        out["race_set_vs_oracle"] = {"events_checked": int(len(ev)), "identical": bool(np.array_equal(want, races))}
        out["cpu_oracle"] = {"value": len(ev) / dt, "unit": "events/s", "cores": 1, "sample": "whole trace"}
    log(f"c2 main done ({time.perf_counter() - T0:.1f} s)")
    if not args.no_ranker:
        out["ranker"] = bench_ranker(args, local, torch, gwcp, np, ev, geo, dev)
        log(f"ranker section done ({time.perf_counter() - T0:.1f} s)")
    if not args.no_compressed:
        out["compressed"] = bench_compressed(args, local, torch, gwcp, np, geo, dev, races.copy())
        log(f"compressed section done ({time.perf_counter() - T0:.1f} s)")
    del dev
    return out


def bench_tiny(args, local, torch, gwcp, tracegen, np):
    """The tiny 64-thread trace (thread granularity, 10k events): events/s and the race
    set against the oracle."""
    ev, geo, _ = tracegen.generate(SEED, workload=TINY)
    dev = torch.from_numpy(ev.view(np.uint8).copy()).to(f"cuda:{local}")
    s = torch.cuda.Stream(device=local)
    ctx = gwcp.Context(local)
    ctx.load_trace(dev, *geo.astuple(), stream=s)
    for _ in range(3):
        ctx.compute_order(stream=s)
    ms, _, n_races, _ = run_steps(ctx, s, 20, torch, gwcp)
    races = ctx.report_races(stream=s)
    ctx.close()
    out = {"events": int(len(ev)), "agents": geo.num_agents, "value": len(ev) / (statistics.median(ms) / 1e3),
           "unit": "events/s", "ms_per_step": statistics.median(ms), "steps": 20, "warmup": 3,
           "n_races": int(n_races)}
    if not args.no_cpu_baseline:
        from oracle import oracle

        t0 = time.perf_counter()
        want = oracle.run(ev, *geo.astuple()).races
        dt = time.perf_counter() - t0
        out["race_set_vs_oracle"] = {"events_checked": int(len(ev)), "identical": bool(np.array_equal(want, races))}
        out["cpu_oracle"] = {"value": len(ev) / dt, "unit": "events/s", "cores": 1, "sample": "whole trace"}
    return out


def host_cpu() -> dict:
    """The host's logical core count and CPU model (first model line of /proc/cpuinfo, or
    the platform's processor string)."""
    import platform

    model = None
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.lower().startswith(("model name", "cpu model")):
                    model = line.split(":", 1)[1].strip()
                    break
    except OSError:
        pass
    return {"nproc": os.cpu_count(), "cpu_model": model or platform.processor() or platform.machine()}


def run_reference(args, rank, world):
    """Reference arm: the CPU oracle as it stands, on the host cores, on a bounded
    prefix of the same workload per step (rank 0 only)."""
    if rank != 0:
        return
    from oracle import oracle
    from paper_2111_12478_gb300 import tracegen

    n_sample = args.ref_events
    # the workload's first n_sample events (the generator's stream does not depend on the
    # requested length, and a prefix of a well-formed trace is well-formed)
    ev, geo, _ = tracegen.generate(SEED, workload=WORKLOAD, n_events=n_sample)
    for _ in range(args.warmup):
        oracle.run(ev, *geo.astuple())
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        oracle.run(ev, *geo.astuple())
        times.append(time.perf_counter() - t0)
    t = statistics.mean(times)
    v = n_sample / t
    out = {"impl": "reference", "metric": METRIC, "value": v, "unit": "events/s", "n_gpus": args.gpus,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": t * 1e3, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
           "config": {"workload": WORKLOAD, "events_per_step": n_sample, "seed": SEED},
           "cpu_baseline": {"value": v, "unit": "events/s", "cores": 1, "kind": "oracle",
                            "sample": f"first {n_sample} events of the {WORKLOAD} trace (seed {SEED}), per step",
                            **host_cpu()},
           "e2e": {"value": v, "unit": "events/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gwcp", choices=["gwcp", "reference"])
    ap.add_argument("--ref-events", type=int, default=500_000,
                    help="events of the headline workload the reference arm's oracle analyses per step")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--e2e-steps", type=int, default=5)
    ap.add_argument("--events", type=int, default=0, help="analyse only this many events of the workload "
                    "(profiling runs); 0 = the full workload")
    ap.add_argument("--workload", default=WORKLOAD, help="a trace shape of tracegen.WORKLOADS")
    ap.add_argument("--c2-steps", type=int, default=20, help="timed steps of the 64-warp workload")
    ap.add_argument("--no-c2", action="store_true", help="skip the 64-warp workload (and its ranker and "
                    "compressed-clock measurements)")
    ap.add_argument("--no-ranker", action="store_true", help="skip the ranked-check measurement")
    ap.add_argument("--no-compressed", action="store_true", help="skip the compressed-versions measurement")
    ap.add_argument("--clock-mode", default="auto", choices=list(CLOCK_MODES),
                    help="clock representation of the headline section")
    ap.add_argument("--no-configs", action="store_true", help="skip the tiny workload")
    ap.add_argument("--no-batched", action="store_true", help="skip the batched (512-trace) measurement")
    ap.add_argument("--no-served", action="store_true", help="skip the served (Poisson arrivals) measurement")
    ap.add_argument("--batch-steps", type=int, default=3)
    ap.add_argument("--serve-requests", type=int, default=1000)
    ap.add_argument("--lanes", type=int, default=32, help="lanes of the batched/served pool")
    ap.add_argument("--cpu-events", type=int, default=0, help="events of the headline trace the oracle runs on "
                    "for the CPU baseline and the live exactness check (a prefix); 0 = the whole trace up to 1024 "
                    "agents, 3M events beyond")
    args = ap.parse_args()

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        return run_reference(args, rank, world)

    import numpy as np
    import torch

    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")

    import __graft_entry__

    if rank == 0:
        __graft_entry__.build()
    if dist:
        dist.barrier()
    from paper_2111_12478_gb300 import gwcp, tracegen

    # --events: a shorter trace of the same workload shape (profiling runs)
    ev, geo, planted = tracegen.generate(SEED + rank, workload=args.workload, n_events=args.events or None)
    n_ev = len(ev)
    stream = torch.cuda.Stream(device=local)
    dev = torch.from_numpy(ev.view(np.uint8)).to(f"cuda:{local}")
    ctx = gwcp.Context(local, profile=True)
    ctx.set_clock_mode(CLOCK_MODES[args.clock_mode])
    ctx.load_trace(dev, *geo.astuple(), stream=stream)

    clocks = ClockSampler(local).__enter__()  # started early: nvidia-smi takes a moment to start
    for _ in range(args.warmup):
        ctx.compute_order(stream=stream)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clocks.mark_start()
    step_ms, prof_acc, n_races, launches = run_steps(ctx, stream, args.steps, torch, gwcp)
    clocks.mark_end()
    clocks.__exit__(None, None, None)
    t_local = sum(step_ms) / 1e3
    t_max, ev_total = replica_reduce(t_local, n_ev * args.steps, dist, device=f"cuda:{local}")
    value = ev_total / t_max
    ms_per_step = t_max * 1e3 / args.steps
    races = ctx.report_races(stream=stream)
    cnt = ctx.counters()
    ctx.close()
    del dev
    log(f"headline timed ({time.perf_counter() - T0:.1f} s)")

    # end to end through the C ABI: pinned host trace -> device, compute, races -> host
    pinned = torch.from_numpy(ev.view(np.uint8)).pin_memory()
    ctx_e2e = gwcp.Context(local)
    ctx_e2e.set_clock_mode(CLOCK_MODES[args.clock_mode])
    e2e_times, d2h = [], 0
    # the step's result lands in a reused pinned buffer (one DMA, no page faults)
    out_pinned = torch.empty((max(len(races), 1) + 1024) * 2, dtype=torch.int64).pin_memory()
    out_np = out_pinned.numpy().view(np.uint64).reshape(-1, 2)
    parts = []  # per step: device ms of the H2D copy, the analysis, the race read-back
    for it in range(args.e2e_steps + max(1, args.warmup) if args.e2e_steps else 0):
        torch.cuda.synchronize()
        ev4 = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
        ev4[0].record(stream)
        t0 = time.perf_counter()
        rc = ctx_e2e._L.gwcp_load_trace(ctx_e2e._h, pinned.data_ptr(), n_ev, gwcp.Geometry(*geo.astuple(), 0), 0,
                                        stream.cuda_stream)
        assert rc == 0, rc
        ev4[1].record(stream)
        ctx_e2e.compute_order(stream=stream)
        ev4[2].record(stream)
        got = ctx_e2e.report_races(stream=stream, out=out_np)
        ev4[3].record(stream)
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
        if it >= max(1, args.warmup):  # untimed rounds size the context's buffers and warm the path
            e2e_times.append(max(wall, ev4[0].elapsed_time(ev4[3]) / 1e3))
            parts.append([ev4[j].elapsed_time(ev4[j + 1]) for j in range(3)])
        d2h = got.nbytes + 8
    e2e_value = n_ev * world / statistics.mean(e2e_times) if e2e_times else None
    ctx_e2e.close()
    del pinned, out_pinned
    log(f"e2e done ({time.perf_counter() - T0:.1f} s)")

    result = None
    if rank == 0:
        cpu, exact = None, None
        if not args.no_cpu_baseline:
            from oracle import oracle

            # a race (a, b) depends only on the events up to b, so the races of a prefix are
            # the full trace's races whose later access lies in it
            k = args.cpu_events or (n_ev if geo.num_agents <= 1024 else 3_000_000)
            k = min(k, n_ev)
            t0 = time.perf_counter()
            ref = oracle.run(ev[:k], *geo.astuple())
            dt = time.perf_counter() - t0
            exact = {"events_checked": k, "identical": bool(np.array_equal(ref.races, races[races[:, 1] < k])),
                     "how": "the oracle run of the CPU baseline"}
            what = f"the full {n_ev}-event trace" if k == n_ev else f"the first {k} events of the {n_ev}-event trace"
            cpu = {"value": k / dt, "unit": "events/s", "cores": 1, "kind": "oracle",
                   "sample": f"{what} of this run (seed {SEED}), single-threaded C++ -O2", "seconds": dt,
                   **host_cpu()}
        stored = digest_check(ev, races, args.workload, SEED + rank) if not args.events else None
        peak, peak_kind = read_peaks()
        wp = tracegen.WORKLOADS[args.workload]
        phases = {k: (v[0] / v[2], v[1] / v[2]) for k, v in prof_acc.items()}
        tiles = cnt["tiles_read"] + cnt["tiles_written"] > 0
        clk = clocks.summary()
        result = {
            "metric": METRIC, "value": value, "unit": "events/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "u32", "data": "synthetic",
            "config": {"workload": args.workload, "events": n_ev, "agents": geo.num_agents,
                       "clock_mode": args.clock_mode, "agents_per_block": geo.agents_per_block,
                       "granularity": "warp" if geo.granularity else "thread", "blocks": wp["num_blocks"],
                       "addresses": wp["n_ranks"], "zipf_s": wp["zipf_s"],
                       "sync_frac": round(wp["p_acqrel"] + wp["p_fence"] + wp["p_barrier"] + wp["p_atomic"], 6),
                       "plant_frac": wp["plant_frac"], "seed": SEED, "parallelism": f"replicas{world}",
                       "l2": f"inputs larger than L2 ({ev.nbytes / 1e6:.0f} MB trace; larger working set per step)"},
            "e2e": {"value": e2e_value, "unit": "events/s", "h2d_bytes_per_step": int(ev.nbytes),
                    "d2h_bytes_per_step": int(d2h), "steps": len(e2e_times),
                    "step_ms": [round(t * 1e3, 2) for t in e2e_times],
                    "device_ms_h2d_analysis_d2h": [round(float(np.mean([p[j] for p in parts])), 2) for j in range(3)],
                    "device_ms_per_step": [[round(x, 2) for x in p] for p in parts]}
            if e2e_value else None,
            "roofline": prop_roofline("k_prop_wide" if tiles else "k_propagate", args.workload,
                                      phases["g_propagate"][0], cnt, geo.num_agents, tiles, peak, peak_kind),
            "roofline_check": (check_roofline(phases["i_check"][0], phases["i_check"][1], cnt, len(races),
                                              args.workload, peak, peak_kind) if "i_check" in phases else None),
            "phases_ms": {k: round(v[0], 4) for k, v in sorted(phases.items(), key=lambda kv: -kv[1][0])},
            "counters": cnt,
            "cpu_baseline": cpu,
            "race_set_vs_oracle": {"live": exact, "stored_digests": stored},
            "race_set_bit_exact": (bool(exact["identical"]) if exact else None) if not stored else
                                  bool(stored["identical"] and (exact is None or exact["identical"])),
            "n_races": int(n_races), "gpu_launches": int(launches), "clocks": clk,
        }
    del ev
    log(f"headline section done ({time.perf_counter() - T0:.1f} s)")
    if rank == 0 and not args.no_c2:
        result["c2"] = bench_c2(args, local, torch, gwcp, tracegen, np, *read_peaks())
    if rank == 0 and not args.no_configs:
        result["tiny"] = bench_tiny(args, local, torch, gwcp, tracegen, np)
        log(f"tiny done ({time.perf_counter() - T0:.1f} s)")
    b = None
    if not args.no_batched:
        b = bench_batched(args, local, torch, gwcp, tracegen, np)
        if result is not None:
            result["batched"] = b
        log(f"batched section done ({time.perf_counter() - T0:.1f} s)")
    if not args.no_served:
        v = bench_served(args, local, torch, gwcp, tracegen, np, b["lanes"] if b else 16,
                         b["pack_walkers"] if b else True)
        if result is not None:
            result["served"] = v
        log(f"served section done ({time.perf_counter() - T0:.1f} s)")
    if dist:
        dist.barrier()
        dist.destroy_process_group()
    if result is not None:
        print(json.dumps(result), flush=True)


if __name__ == "__main__":
    main()
