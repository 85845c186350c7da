"""Pins of the oracle's vector-clock compression (section "Vector Clock Compression"):
forced compression at barriers and the size of a clock in the block/warp compressed form.

The paper states that setting the participants' entries to the highest of them at a
barrier keeps the ordering, because every participant restarts only after all of them
arrived: the race set must not change. The pins below check that against the unforced
oracle and the brute-force closure, check hand-computed clocks and sizes, and check the
number of clock versions against a direct count of the steps that create one.
"""
import numpy as np
import pytest

import gwcp_closure as GC
from oracle import oracle as O
from paper_2111_12478_gb300 import tracegen as TG
from paper_2111_12478_gb300.tracegen import ACQ, ATOMIC, BARRIER, CTA, READ, REL, THREAD, WRITE

WARP_GRAN = 1
GEOMS = [(4, 2, THREAD), (6, 3, THREAD), (8, 8, WARP_GRAN), (48, 24, THREAD), (64, 64, THREAD), (40, 8, WARP_GRAN)]


@pytest.mark.parametrize("fam", TG.FAMILIES)
def test_forced_barrier_keeps_the_race_set(fam):
    for seed in range(12):
        for W, apb, gran in GEOMS:
            ev, geo = TG.random_small(seed, fam, n_events=120, num_agents=W, agents_per_block=apb,
                                      granularity=gran, n_locks=3, n_keys=5)
            plain = O.run(ev, *geo.astuple())
            forced = O.run(ev, *geo.astuple(), forced_barrier=True)
            assert O.race_set(forced) == O.race_set(plain), (fam, seed, W)
            assert forced.counters["epoch_test_disagree"] == 0
            both = O.run(ev, *geo.astuple(), forced_barrier=True, all_pairs=True)
            assert O.race_set(both) == O.race_set(O.run(ev, *geo.astuple(), all_pairs=True))
            hb = O.run(ev, *geo.astuple(), forced_barrier=True, hb_only=True)
            assert O.race_set(hb) == O.race_set(O.run(ev, *geo.astuple(), hb_only=True))


@pytest.mark.parametrize("fam", ("barriers", "uniform_bar", "mixed"))
def test_forced_barrier_against_the_closure(fam):
    """On tiny traces the forced oracle's full pair set holds the algorithm-mode closure's
    (which orders events from the trace alone: no clocks, no local times), as the unforced
    oracle's does, and the exact families give equality."""
    for seed in range(25):
        for W, apb in [(4, 2), (6, 2)]:
            ev, geo = TG.random_small(seed * 5 + W, fam, n_events=36, num_agents=W, agents_per_block=apb)
            alg, _, _ = GC.analyze(ev, *geo.astuple(), mode="algorithm")
            forced = O.race_set(O.run(ev, *geo.astuple(), forced_barrier=True, all_pairs=True))
            assert alg <= forced
            if fam == "barriers":
                assert forced == alg


def _worked_trace():
    """Warp 0 takes lock L twice (N_0 = 3), warp 1 does nothing; a barrier of their block;
    then both write x (a race), and warp 0 writes y that warp 1 wrote before the barrier
    (ordered)."""
    b = TG.TraceBuilder()
    b.wr(1, 0x20)          # 0
    b.acq(0, 7)            # 1
    b.rel(0, 7)            # 2
    b.acq(0, 7)            # 3
    b.rel(0, 7)            # 4
    b.barrier(0)           # 5: CTA barrier of block 0
    b.wr(1, 0x10)          # 6
    b.wr(0, 0x10)          # 7
    b.wr(0, 0x20)          # 8
    return b.build(), TG.Geometry(2, 2, WARP_GRAN)


def test_forced_barrier_worked_example():
    ev, geo = _worked_trace()
    plain = O.run(ev, *geo.astuple(), clock_events=[6, 7])
    forced = O.run(ev, *geo.astuple(), forced_barrier=True, clock_events=[6, 7])
    # plain: the join gives each warp the other's local time (3 and 1); N_1 becomes 2
    assert plain.clocks_c[6].tolist() == [3, 2] and plain.clocks_c[7].tolist() == [4, 1]
    # forced: both leave at max(3, 1) = 3; the join holds 3 for both entries, N_t = 4
    assert forced.clocks_c[6].tolist() == [3, 4] and forced.clocks_c[7].tolist() == [4, 3]
    assert forced.clocks_h[6].tolist() == [3, 4]
    assert O.race_set(forced) == O.race_set(plain) == {(6, 7)}


def test_block_entries_equal_after_a_barrier():
    """Under forced compression, an agent's clock right after a CTA barrier of its block
    (before its next synchronisation) holds one value M for every other member and M + 1
    for itself."""
    for seed in range(20):
        for W, apb, gran in [(8, 4, WARP_GRAN), (16, 8, THREAD)]:
            ev, geo = TG.random_small(seed, "mixed", n_events=150, num_agents=W, agents_per_block=apb,
                                      granularity=gran, n_locks=2, n_keys=4)
            acc = [i for i in range(len(ev)) if ev["op"][i] in (READ, WRITE, ATOMIC)]
            r = O.run(ev, *geo.astuple(), forced_barrier=True, clock_events=acc)
            last_sync = {}
            checked = 0
            for i in range(len(ev)):
                op, t = int(ev["op"][i]), int(ev["agent"][i])
                if op == BARRIER and int(ev["scope"][i]) == CTA:
                    blk = int(ev["addr"][i])
                    for m in range(blk * apb, blk * apb + apb):
                        last_sync[m] = ("bar", blk)
                elif op == BARRIER:  # a warp barrier: its members synchronised otherwise
                    if gran == WARP_GRAN:
                        last_sync[t] = ("other", None)
                    else:
                        base = t // apb * apb + (t % apb) // 32 * 32
                        for lane in range(32):
                            if (int(ev["addr"][i]) >> lane) & 1:
                                last_sync[base + lane] = ("other", None)
                elif op in (ACQ, REL):
                    last_sync[t] = ("other", None)
                elif op in (READ, WRITE, ATOMIC) and last_sync.get(t, ("", None))[0] == "bar":
                    blk = last_sync[t][1]
                    c = r.clocks_c[i]
                    others = [int(c[m]) for m in range(blk * apb, blk * apb + apb) if m != t]
                    assert len(set(others)) == 1 and int(c[t]) == others[0] + 1, (seed, i)
                    checked += 1
            assert checked > 0 or not (ev["op"] == BARRIER).any()


def test_version_words_worked_examples():
    # the trace above: 2 initial versions, 4 lock steps of warp 0, 2 barrier participations;
    # one block of two agents (warp granularity: one word per agent when expanded)
    ev, geo = _worked_trace()
    forced = O.run(ev, *geo.astuple(), forced_barrier=True, version_words=True).counters
    plain = O.run(ev, *geo.astuple(), version_words=True).counters
    assert forced["versions"] == plain["versions"] == 8
    assert forced["version_words"] == 8     # every version is uniform: [0, 0] or [3, 3]
    assert plain["version_words"] == 12     # the barrier's versions [3, 1] take 1 + 2 words
    # thread granularity, one block of 64 threads (two warps): thread 1's in-section write
    # joins L^w(x) = H_0 = [1, 0, ...], so its versions there and at its release hold
    # [1, 0, ...]: header, two warp words and the 32 values of warp 0
    b = TG.TraceBuilder()
    b.acq(0, 3)
    b.wr(0, 0x40)
    b.rel(0, 3)
    b.acq(1, 3)
    b.wr(1, 0x40)
    b.rel(1, 3)
    c = O.run(b.build(), 64, 64, THREAD, version_words=True).counters
    assert c["versions"] == 64 + 6
    assert c["version_words"] == 64 + 4 * 1 + 2 * (1 + 2 + 32)


def test_version_words_without_synchronisation():
    ev, geo = TG.random_small(2, "nosync", n_events=100, num_agents=12, agents_per_block=4)
    c = O.run(ev, *geo.astuple(), version_words=True).counters
    assert c["versions"] == 12 and c["version_words"] == 12 * 3  # one zero word per block


def test_versions_count_the_clock_changing_steps():
    """One version per agent at the start, per acquire and release, per barrier member,
    and per access made while holding a lock (counted here from the trace alone)."""
    for seed in range(10):
        for W, apb, gran in [(8, 4, THREAD), (64, 64, THREAD), (40, 8, WARP_GRAN)]:
            ev, geo = TG.random_small(seed, "mixed", n_events=150, num_agents=W, agents_per_block=apb,
                                      granularity=gran, n_locks=3, n_keys=4)
            depth = [0] * W
            n = W
            for e in ev:
                op, t = int(e["op"]), int(e["agent"])
                if op == ACQ:
                    depth[t] += 1
                    n += 1
                elif op == REL:
                    depth[t] -= 1
                    n += 1
                elif op == BARRIER:
                    if int(e["scope"]) == CTA:
                        n += apb
                    elif gran == WARP_GRAN:
                        n += 1
                    else:
                        n += bin(int(e["addr"])).count("1")
                elif op in (READ, WRITE, ATOMIC) and depth[t] > 0:
                    n += 1
            for forced in (False, True):
                c = O.run(ev, *geo.astuple(), forced_barrier=forced, version_words=True).counters
                assert c["versions"] == n, (seed, W, forced)
                assert c["version_words"] >= c["versions"] * (W // apb)  # at least a header per block


def test_forced_barrier_shrinks_the_workload_versions():
    """On a sample of the 8-block, 64-warp workload the forced barriers leave most blocks of
    every version uniform: the compressed versions take well under half the dense words."""
    ev, geo, _ = TG.generate(1, workload="8blk_64warp_10M", n_events=100_000)
    W = geo.num_agents
    plain = O.run(ev, *geo.astuple(), version_words=True).counters
    forced = O.run(ev, *geo.astuple(), forced_barrier=True, version_words=True).counters
    assert forced["versions"] == plain["versions"]
    assert forced["version_words"] < 0.5 * forced["versions"] * W
    assert forced["version_words"] < 0.7 * plain["version_words"]
