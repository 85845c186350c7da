"""Batched and served analysis (gwcp_pool) on the GPU, through the C ABI.

Every trace's race set from the pool must be identical to the single-context result for
the same trace (and to the oracle where the oracle is quick): alone and in a batch, in a
served mix whose requests arrive while others run, and under a memory budget that forces
the pool to release cached buffers and run requests one after another.
"""
import threading
import time

import numpy as np
import pytest

from oracle import oracle as O
from paper_2111_12478_gb300 import tracegen as TG

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gw():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__

    __graft_entry__.build()
    from paper_2111_12478_gb300 import gwcp

    return gwcp


def alone(gwcp, ev, geo):
    with gwcp.Context(0) as c:
        c.load_trace(ev, *geo.astuple())
        c.compute_order()
        return c.report_races()


@pytest.fixture(scope="module")
def mix(gw):
    """Traces of every width class (64-4096 warps), 1k-150k events, plus small thread-
    granularity traces, a one-event trace and an empty one; with their single-context races."""
    specs = TG.many_specs(11, 21, 1_000, 150_000)
    traces = [(ev, geo) for ev, geo in TG.generate_many(specs)]
    for seed, fam in enumerate(("mixed", "barriers", "dev_locks")):
        traces.append(TG.random_small(seed, fam, n_events=300, num_agents=64, agents_per_block=32,
                                      n_locks=3, n_keys=6))
    b = TG.TraceBuilder()
    b.wr(0, 0x10)
    traces.append((b.build(), TG.Geometry(4, 2, TG.THREAD)))
    traces.append((np.zeros(0, dtype=TG.EVENT_DTYPE), TG.Geometry(4, 2, TG.THREAD)))
    want = [alone(gw, ev, geo) for ev, geo in traces]
    assert sum(len(w) for w in want) > 0
    return traces, want


def test_mix_covers_widths_and_oracle(mix):
    traces, want = mix
    assert {geo.num_agents for _, geo in traces} >= set(TG.BATCH_WIDTHS)
    for (ev, geo), w in zip(traces, want):  # the single-context results are the oracle's
        if len(ev) <= 40_000 and geo.num_agents <= 1024:
            assert np.array_equal(w, O.run(ev, *geo.astuple()).races)


def test_batch_equals_alone(gw, mix):
    traces, want = mix
    with gw.Pool(0, lanes=8) as P:
        got = P.run_batch([(ev, geo.astuple()) for ev, geo in traces], [len(w) + 4 for w in want])
    for (races, rc, n), w in zip(got, want):
        assert rc == 0 and n == len(w)
        assert np.array_equal(races, w)


def test_batch_twice_and_device_inputs(gw, mix):
    import torch

    traces, want = mix
    dev = [(torch.from_numpy(ev.view(np.uint8).copy()).cuda() if len(ev) else ev, geo.astuple())
           for ev, geo in traces]
    with gw.Pool(0, lanes=4) as P:
        for _ in range(2):  # lanes reuse their cached buffers on the second batch
            got = P.run_batch(dev, [len(w) for w in want])
            for (races, rc, n), w in zip(got, want):
                assert rc == 0 and n == len(w) and np.array_equal(races, w)


def test_served_mix_equals_alone(gw, mix):
    traces, want = mix
    rng = np.random.default_rng(5)
    order = rng.permutation(len(traces))
    tickets = {}
    with gw.Pool(0, lanes=6) as P:
        def submitter():
            for i in order:
                tickets[int(i)] = P.submit(traces[i][0], traces[i][1].astuple(), len(want[i]) + 1)
                time.sleep(float(rng.uniform(0, 0.004)))

        th = threading.Thread(target=submitter)
        th.start()
        th.join()
        done = set()
        while len(done) < len(traces):  # poll in submission-independent order
            for i in rng.permutation(len(traces)):
                i = int(i)
                if i in done:
                    continue
                r = P.wait(tickets[i], block=False)
                if r is None:
                    continue
                races, info = r
                assert info.rc == 0 and info.n_races == len(want[i])
                assert np.array_equal(races, want[i])
                assert info.t_submit <= info.t_admit <= info.t_done
                done.add(i)
            time.sleep(0.001)


def test_memory_admission(gw, mix):
    traces, want = mix
    budget = 96 << 20  # smaller than what most of these traces need alone
    with gw.Pool(0, lanes=8, mem_budget=budget) as P:
        got = P.run_batch([(ev, geo.astuple()) for ev, geo in traces], [len(w) for w in want])
        for (races, rc, n), w in zip(got, want):
            assert rc == 0 and n == len(w) and np.array_equal(races, w)
        assert P.device_bytes() <= max(budget, 512 << 20)


def test_invalid_trace_in_batch(gw, mix):
    traces, want = mix
    bad = np.zeros(3, dtype=TG.EVENT_DTYPE)
    bad[1] = (9, TG.READ, 0, 0, 0, 1)  # agent out of range
    rc0, idx0 = O.validate(bad, 4, 2, TG.THREAD)
    batch = [(traces[0][0], traces[0][1].astuple()), (bad, (4, 2, TG.THREAD)), (traces[1][0], traces[1][1].astuple())]
    with gw.Pool(0, lanes=2) as P:
        got = P.run_batch(batch, [len(want[0]), 1, len(want[1])])
        assert got[1][1] == gw.ERR_INVALID_TRACE == rc0
        assert got[0][1] == 0 and np.array_equal(got[0][0], want[0])
        assert got[2][1] == 0 and np.array_equal(got[2][0], want[1])
        t = P.submit(bad, (4, 2, TG.THREAD), 1)
        _, info = P.wait(t)
        assert info.rc == gw.ERR_INVALID_TRACE and info.first_bad_index == idx0


def test_autotune(gw, mix):
    traces, want = mix
    with gw.Pool(0, lanes=8) as P:
        best, secs = P.autotune([(ev, geo.astuple()) for ev, geo in traces])
        assert best in secs and set(secs) == {1, 2, 4, 8}
        # the most lanes whose batch time is within 5% of the fastest
        fastest = min(secs.values())
        assert secs[best] <= 1.05 * fastest
        assert all(k <= best for k, v in secs.items() if v <= 1.05 * fastest)
        assert P.settings()[0] == best  # (active lanes, packed walkers)
        # width classes 7..10 (128..1024 warps) hold only traces that take both clock
        # representations; class 6 also holds thread-granularity traces
        modes = P.clock_modes()
        assert {7, 8, 9, 10} <= set(modes) <= {6, 7, 8, 9, 10} and set(modes.values()) <= {1, 2}
        got = P.run_batch([(ev, geo.astuple()) for ev, geo in traces], [len(w) for w in want])
        for (races, rc, n), w in zip(got, want):
            assert rc == 0 and np.array_equal(races, w)


def test_memory_mode_pool(gw, mix):
    """Lanes in the paper's memory mode (compressed clock versions, forced barrier
    compression): every trace's race set is the plain single-context one, in a batch, under
    a tight memory budget, and after the autotuner (which leaves the clock modes alone)."""
    traces, want = mix
    batch = [(ev, geo.astuple()) for ev, geo in traces]
    with gw.Pool(0, lanes=8, compress_versions=True) as P:
        for _ in range(2):  # the second batch runs on the lanes' grown version pools
            got = P.run_batch(batch, [len(w) for w in want])
            for (races, rc, n), w in zip(got, want):
                assert rc == 0 and n == len(w) and np.array_equal(races, w)
        P.autotune(batch)
        assert P.clock_modes() == {}
        got = P.run_batch(batch, [len(w) for w in want])
        for (races, rc, n), w in zip(got, want):
            assert rc == 0 and np.array_equal(races, w)
    with gw.Pool(0, lanes=8, mem_budget=96 << 20, compress_versions=True) as P:
        got = P.run_batch(batch, [len(w) for w in want])
        for (races, rc, n), w in zip(got, want):
            assert rc == 0 and np.array_equal(races, w)
