"""CUDA path vs the oracle on the large workloads, through the stored oracle digests
(tests/golden/oracle_digests.json, written by tests/golden/make_oracle_digests.py, which
runs only the oracle). Needs a GB300.

A race (a, b) depends only on the events up to b, so the races of a prefix are the whole
trace's races with b in the prefix; digests are compared per bucket of b. Each entry
first checks that the regenerated trace is the one the oracle ran on (SHA-256).

  * 256 blocks x 32 warps, 200M events: the GPU analyses the whole trace; its races with
    b in the first 50M (seed 1) and 20M (seed 2) events equal the oracle's, bucket by
    bucket, and every race involves a planted access.
  * the 512-trace batch, through the pool in one batch: every trace's whole race set.
  * served requests (prefixes of the seven 20M-event base traces, lengths multiples of
    the 250k-event bucket up to the whole trace), submitted to the pool while others
    run: every bucket of every request.
"""
import json
import os

import numpy as np
import pytest

from paper_2111_12478_gb300 import tracegen as TG
from race_digest import bucket_digests, trace_sha256, whole_digest

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "oracle_digests.json")


@pytest.fixture(scope="module")
def gw():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__

    __graft_entry__.build()
    from paper_2111_12478_gb300 import gwcp

    return gwcp


@pytest.fixture(scope="module")
def digests():
    with open(GOLDEN) as f:
        return json.load(f)


def _c3_entry(digests, seed):
    return next(e for e in digests["c3"] if e["seed"] == seed)


@pytest.mark.parametrize("seed", [1, 2])
def test_8192warp_200M_vs_oracle(gw, digests, seed):
    e = _c3_entry(digests, seed)
    ev, geo, planted = TG.generate(seed, workload=e["workload"])
    assert len(ev) == 200_000_000 and geo.num_agents == e["agents"]
    assert trace_sha256(ev, e["events"]) == e["trace_sha256"], "not the trace the oracle ran on"
    with gw.Context(0) as c:
        c.load_trace(ev, *geo.astuple())
        c.compute_order()
        got = c.report_races()
    nb = e["events"] // e["bucket"]
    assert bucket_digests(got, e["bucket"], nb) == e["buckets"]
    assert int((got[:, 1] < e["events"]).sum()) == e["n_races"]
    pl = np.zeros(len(ev), dtype=bool)
    pl[planted] = True
    assert len(got) > e["n_races"] and (pl[got[:, 0]] | pl[got[:, 1]]).all()


def test_batch_512_traces_vs_oracle(gw, digests):
    d = digests["batch"]
    specs = TG.many_specs(d["seed"], **d["workload"])
    traces = TG.generate_many(specs, threads=os.cpu_count() or 8)
    assert len(traces) == len(d["traces"]) == 512
    for (ev, geo), e in zip(traces, d["traces"]):
        assert trace_sha256(ev) == e["trace_sha256"] and geo.num_agents == e["agents"]
    caps = [e["digest"][0] + 1 for e in d["traces"]]
    with gw.Pool(0, lanes=12) as P:
        got = P.run_batch([(ev, geo.astuple()) for ev, geo in traces], caps)
    bad = [i for i, ((races, rc, n), e) in enumerate(zip(got, d["traces"]))
           if rc != 0 or n != e["digest"][0] or whole_digest(races) != e["digest"]]
    assert not bad, f"{len(bad)} traces differ from the oracle, first {bad[:5]}"


def test_served_requests_vs_oracle(gw, digests):
    import threading
    import time

    d = digests["serve"]
    bucket = d["bucket"]
    specs = TG.serve_base_specs(d["seed"], TG.SERVE_WORKLOAD["n_max"])
    base = TG.generate_many(specs, threads=os.cpu_count() or 8)
    for (ev, geo), e in zip(base, d["traces"]):
        assert trace_sha256(ev, e["events"]) == e["trace_sha256"] and geo.num_agents == e["agents"]
    rng = np.random.default_rng(7)
    reqs = [(j, k * bucket) for j in range(len(base)) for k in (1, 3, 8, 20, 40, d["prefix"] // bucket)]
    reqs = [reqs[i] for i in rng.permutation(len(reqs))]
    tickets = [None] * len(reqs)
    with gw.Pool(0, lanes=16) as P:
        def submit_all():  # requests arrive while earlier ones run
            for i, (j, n) in enumerate(reqs):
                cap = sum(b[0] for b in d["traces"][j]["buckets"][: n // bucket]) + 1
                tickets[i] = P.submit(base[j][0][:n], base[j][1].astuple(), cap)
                time.sleep(float(rng.uniform(0, 0.01)))

        th = threading.Thread(target=submit_all)
        th.start()
        for i, (j, n) in enumerate(reqs):
            while tickets[i] is None:
                time.sleep(0.001)
            races, info = P.wait(tickets[i])
            want = d["traces"][j]["buckets"][: n // bucket]
            assert info.rc == 0 and info.n_races == sum(b[0] for b in want), (j, n)
            assert bucket_digests(races, bucket, n // bucket) == want, (j, n)
        th.join()
