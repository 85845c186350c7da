"""Writes tests/golden/oracle_digests.json: digests of the oracle's race sets on the large
workloads, which the GPU tests and bench.py compare the CUDA path's races with.

Calls only the oracle (oracle/) and the seeded input generator; nothing here runs the
CUDA path. Each entry also stores the SHA-256 of the trace it was computed on, so a
test can tell a different trace from a different race set.

  python tests/golden/make_oracle_digests.py --part c3|batch|serve [--workers N]

Parts (a part rewrites only its own key of the JSON file):
  c3     the 256-block, 8192-warp, 200M-event workload: the oracle on its first 50M
         events (seed 1) and 20M events (seed 2); digests per 1M-event bucket of the
         later access. The oracle's memory (dense L^r / L^w clocks per lock, scope and
         location) grows by ~0.7 GB per million events of this workload, which bounds
         the prefix.
  batch  every trace of the 512-trace batched workload (seed 1): one digest per trace.
  serve  the served workload's base traces (one 20M-event trace per width class, seed 1):
         digests per 250k-event bucket; a request of n events is the first n events of
         its class's trace, so its races are checked on every bucket below n.
"""
from __future__ import annotations

import argparse
import json
import multiprocessing as mp
import os
import resource
import sys
import time
from concurrent.futures import ProcessPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
for p in (ROOT, os.path.join(ROOT, "tests")):
    if p not in sys.path:
        sys.path.insert(0, p)

OUT = os.path.join(HERE, "oracle_digests.json")
SEED = 1
C3 = "256blk_8192warp_200M"
C3_PREFIXES = ((1, 50_000_000), (2, 20_000_000))
C3_BUCKET = 1_000_000
SERVE_PREFIX = 20_000_000
SERVE_BUCKET = 250_000


def _rss_gb():
    return resource.getrusage(resource.RUSAGE_SELF).ru_maxrss / 1e6


def _c3_one(seed, n):
    from oracle import oracle
    from paper_2111_12478_gb300 import tracegen
    from race_digest import bucket_digests, trace_sha256

    ev, geo, _ = tracegen.generate(seed, workload=C3, n_events=n)  # the workload's first n events
    t0 = time.perf_counter()
    r = oracle.run(ev, *geo.astuple())
    dt = time.perf_counter() - t0
    return {"workload": C3, "seed": seed, "events": n, "agents": geo.num_agents, "bucket": C3_BUCKET,
            "trace_sha256": trace_sha256(ev), "n_races": int(len(r.races)),
            "buckets": bucket_digests(r.races, C3_BUCKET, n // C3_BUCKET),
            "oracle_s": round(dt, 1), "oracle_max_rss_gb": round(_rss_gb(), 1), "counters": r.counters}


def _batch_one(i):
    from oracle import oracle
    from paper_2111_12478_gb300 import tracegen
    from race_digest import trace_sha256, whole_digest

    spec = tracegen.many_specs(SEED, **tracegen.BATCH_WORKLOAD)[i]
    ev, geo = tracegen.generate_many([spec], threads=1)[0]
    t0 = time.perf_counter()
    r = oracle.run(ev, *geo.astuple())
    return {"i": i, "events": int(len(ev)), "agents": geo.num_agents, "trace_sha256": trace_sha256(ev),
            "digest": whole_digest(r.races), "oracle_s": round(time.perf_counter() - t0, 2)}


def _serve_one(j):
    from oracle import oracle
    from paper_2111_12478_gb300 import tracegen
    from race_digest import bucket_digests, trace_sha256

    cfg = tracegen.SERVE_WORKLOAD
    spec = dict(tracegen.serve_base_specs(SEED, cfg["n_max"])[j])
    spec["n_events"] = SERVE_PREFIX  # the base trace's first SERVE_PREFIX events
    ev, geo = tracegen.generate_many([spec], threads=1)[0]
    t0 = time.perf_counter()
    r = oracle.run(ev, *geo.astuple())
    return {"j": j, "events": SERVE_PREFIX, "agents": geo.num_agents, "bucket": SERVE_BUCKET,
            "trace_sha256": trace_sha256(ev), "n_races": int(len(r.races)),
            "buckets": bucket_digests(r.races, SERVE_BUCKET, SERVE_PREFIX // SERVE_BUCKET),
            "oracle_s": round(time.perf_counter() - t0, 1), "oracle_max_rss_gb": round(_rss_gb(), 1)}


def _store(key, value):
    data = {}
    if os.path.exists(OUT):
        with open(OUT) as f:
            data = json.load(f)
    data[key] = value
    data["note"] = ("oracle race-set digests: per bucket [count, sum mod 2^64, xor] of splitmix64(later << 32 | "
                    "earlier); written by tests/golden/make_oracle_digests.py")
    with open(OUT + ".tmp", "w") as f:
        json.dump(data, f, separators=(",", ":"))
    os.replace(OUT + ".tmp", OUT)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--part", required=True, choices=["c3", "batch", "serve"])
    ap.add_argument("--workers", type=int, default=4)
    args = ap.parse_args()
    from paper_2111_12478_gb300 import tracegen

    ctx = mp.get_context("spawn")
    t0 = time.perf_counter()
    if args.part == "c3":
        out = []
        for seed, n in C3_PREFIXES:  # one at a time: each takes tens of GB
            with ProcessPoolExecutor(1, mp_context=ctx) as ex:
                out.append(ex.submit(_c3_one, seed, n).result())
            print(f"c3 seed {seed}: {n} events, {out[-1]['n_races']} races, {out[-1]['oracle_s']} s", flush=True)
        _store("c3", out)
    elif args.part == "batch":
        specs = tracegen.many_specs(SEED, **tracegen.BATCH_WORKLOAD)
        order = sorted(range(len(specs)), key=lambda i: -specs[i]["n_events"] * specs[i]["num_blocks"])
        with ProcessPoolExecutor(args.workers, mp_context=ctx) as ex:
            res = list(ex.map(_batch_one, order))
        res.sort(key=lambda e: e["i"])
        _store("batch", {"seed": SEED, "workload": tracegen.BATCH_WORKLOAD, "traces": res})
        print(f"batch: {len(res)} traces, {sum(e['events'] for e in res)} events", flush=True)
    else:
        n_base = len(tracegen.serve_base_specs(SEED, tracegen.SERVE_WORKLOAD["n_max"]))
        with ProcessPoolExecutor(args.workers, mp_context=ctx) as ex:
            res = list(ex.map(_serve_one, range(n_base)))
        _store("serve", {"seed": SEED, "prefix": SERVE_PREFIX, "bucket": SERVE_BUCKET, "traces": res})
        print(f"serve: {len(res)} base traces, first {SERVE_PREFIX} events each", flush=True)
    print(f"done in {time.perf_counter() - t0:.0f} s", flush=True)


if __name__ == "__main__":
    main()
