"""Pins of the CPU oracle against things other than itself.

* the paper's worked examples (figure traces under tests/golden/, expected race sets
  derived by hand from the Definition of GWCP);
* an independent fixpoint closure of the Definition (tests/gwcp_closure.py) on tiny
  random traces: exact equality where the Algorithm and the Definition coincide,
  containment elsewhere;
* closed forms (no synchronisation, all accesses under one device lock, barrier
  phases, blocks without device synchronisation);
* invariants (H_t[t] = N_t, the one-entry epoch test equals the component-wise test,
  HB-only races are a subset of GWCP races);
* FastTrack's detector, written independently, finds the first race on each location at
  the same access as the oracle's race set.
"""
import itertools

import numpy as np
import pytest

import gwcp_closure as GC
from conftest import GOLDEN_FILES, load_golden
from oracle import oracle as O
from paper_2111_12478_gb300 import tracegen as TG
from paper_2111_12478_gb300.tracegen import ACQ, ATOMIC, BARRIER, CTA, DEVICE, READ, REL, THREAD, WRITE


def races(ev, geo, **kw):
    return O.race_set(O.run(ev, *geo.astuple(), **kw))


@pytest.mark.parametrize("name", GOLDEN_FILES)
def test_figure_traces(name):
    ev, geo, expect = load_golden(name)
    r = O.run(ev, *geo.astuple())
    assert O.race_set(r) == expect
    assert r.counters["epoch_test_disagree"] == 0
    assert r.counters["invariant_violations"] == 0


@pytest.mark.parametrize("name", GOLDEN_FILES)
def test_figure_traces_match_definition_closure(name):
    ev, geo, expect = load_golden(name)
    dfn, _, _ = GC.analyze(ev, *geo.astuple(), mode="definition")
    assert GC.project(ev, *geo.astuple(), dfn) == expect


EXACT_FAMILIES = ("nosync", "barriers", "dev_locks", "uniform")
GEOMS = [(4, 2), (3, 3), (6, 2)]


def _family_cases(families, n_seeds):
    for fam in families:
        for seed in range(n_seeds):
            yield fam, seed


@pytest.mark.parametrize("fam,seed", list(_family_cases(EXACT_FAMILIES, 40)))
def test_closure_exact(fam, seed):
    for W, apb in GEOMS:
        ev, geo = TG.random_small(seed * 7 + W, fam, n_events=36, num_agents=W, agents_per_block=apb)
        r = O.run(ev, *geo.astuple(), all_pairs=True)
        ora = O.race_set(r)
        alg, _, _ = GC.analyze(ev, *geo.astuple(), mode="algorithm")
        dfn, _, _ = GC.analyze(ev, *geo.astuple(), mode="definition")
        assert ora == alg, (fam, seed, W)
        assert ora == dfn, (fam, seed, W)
        assert races(ev, geo) == GC.project(ev, *geo.astuple(), ora)
        assert r.counters["epoch_test_disagree"] == 0
        assert r.counters["invariant_violations"] == 0


@pytest.mark.parametrize("fam,seed", list(_family_cases(("uniform_bar", "mixed"), 40)))
def test_closure_containment(fam, seed):
    """Where Algorithm 1 orders less than the Definition (barriers pass on C_t, the
    release loop stops at the first unordered record), the oracle reports a superset of
    the Definition's races, and of the algorithm-mode closure's."""
    for W, apb in GEOMS:
        ev, geo = TG.random_small(seed * 7 + W, fam, n_events=36, num_agents=W, agents_per_block=apb)
        r = O.run(ev, *geo.astuple(), all_pairs=True)
        ora = O.race_set(r)
        alg, _, _ = GC.analyze(ev, *geo.astuple(), mode="algorithm")
        dfn, _, _ = GC.analyze(ev, *geo.astuple(), mode="definition")
        assert dfn <= alg <= ora
        assert r.counters["epoch_test_disagree"] == 0
        assert races(ev, geo) == GC.project(ev, *geo.astuple(), ora)


def test_definition_gap_barrier_fifo():
    """A trace where the Algorithm and the Definition disagree: thread 2 learns thread 3's
    acquire through a barrier (which passes on C_t), never learns thread 0's earlier
    acquire, and the release loop stops at thread 0's record. The Definition orders the
    read at 5 before the write at 33; Algorithm 1 does not."""
    ev, geo = TG.random_small(85, "uniform_bar", n_events=40)
    ora = races(ev, geo, all_pairs=True)
    dfn, _, _ = GC.analyze(ev, *geo.astuple(), mode="definition")
    alg, _, _ = GC.analyze(ev, *geo.astuple(), mode="algorithm")
    assert ora - alg == {(5, 33)}
    assert dfn <= ora


@pytest.mark.parametrize("seed", range(12))
def test_hb_races_subset(seed):
    for fam in ("uniform_bar", "mixed", "dev_locks"):
        ev, geo = TG.random_small(seed, fam, n_events=40)
        gw = races(ev, geo, all_pairs=True)
        hb = races(ev, geo, all_pairs=True, hb_only=True)
        assert hb <= gw
        assert hb == GC.hb_races(ev, *geo.astuple())


# ---- closed forms ----------------------------------------------------------------

@pytest.mark.parametrize("seed", range(10))
def test_no_sync_all_conflicting_pairs_race(seed):
    ev, geo = TG.random_small(seed, "nosync", n_events=50, num_agents=4, agents_per_block=2)
    assert races(ev, geo, all_pairs=True) == GC.all_conflicting(ev, *geo.astuple())


@pytest.mark.parametrize("seed", range(10))
def test_all_accesses_under_one_device_lock_no_race(seed):
    rng = np.random.default_rng(seed)
    b = TG.TraceBuilder()
    for _ in range(12):
        t = int(rng.integers(4))
        b.acq(t, 5, DEVICE)
        for _ in range(int(rng.integers(1, 4))):
            x = 0x1000 + 4 * int(rng.integers(3))
            (b.wr if rng.random() < 0.5 else b.rd)(t, x)
        b.rel(t, 5, DEVICE)
    ev = b.build()
    assert races(ev, TG.Geometry(4, 2, THREAD), all_pairs=True) == set()


@pytest.mark.parametrize("seed", range(10))
def test_one_block_barrier_phases(seed):
    """One block, barriers only: conflicting accesses race iff no barrier separates them."""
    rng = np.random.default_rng(100 + seed)
    b = TG.TraceBuilder()
    phase = []
    ph = 0
    for _ in range(40):
        if rng.random() < 0.15:
            b.barrier(0, agent=0)
            phase.append(None)
            ph += 1
            continue
        t = int(rng.integers(4))
        x = 0x1000 + 4 * int(rng.integers(3))
        (b.wr if rng.random() < 0.4 else b.rd)(t, x)
        phase.append(ph)
    ev = b.build()
    geo = TG.Geometry(4, 4, THREAD)
    want = {(a, c) for a, c in GC.all_conflicting(ev, *geo.astuple()) if phase[a] == phase[c]}
    assert races(ev, geo, all_pairs=True) == want


@pytest.mark.parametrize("seed", range(10))
def test_blocks_without_device_sync_race_across_blocks(seed):
    """Block barriers and block-scoped locks only: every conflicting cross-block pair races."""
    ev, geo = TG.random_small(seed, "mixed", n_events=48, num_agents=4, agents_per_block=2)
    keep = ~((ev["op"] == ACQ) | (ev["op"] == REL)) | (ev["scope"] == CTA)
    ev = ev[keep]
    ev = ev[~((ev["op"] == ATOMIC) & (ev["scope"] == DEVICE))]
    got = races(ev, geo, all_pairs=True)
    blk = ev["agent"] // 2
    cross = {(a, c) for a, c in GC.all_conflicting(ev, *geo.astuple()) if blk[a] != blk[c]}
    assert cross <= got


def test_single_device_lock_is_textbook_wcp():
    """One device-scoped lock, no barriers: GWCP is WCP. The canonical WCP example (a
    predictable race hidden from HB by an unrelated critical section) plus a conflicting
    pair ordered by rule (i)."""
    b = TG.TraceBuilder()
    b.wr(0, 0x10)                 # 0
    b.acq(0, 1); b.rd(0, 0x20); b.rel(0, 1)  # 1..3  (reads z)
    b.acq(1, 1); b.rd(1, 0x20); b.rel(1, 1)  # 4..6  (reads z: no conflict, no rule (i))
    b.wr(1, 0x10)                 # 7: races with 0 under WCP, HB orders it
    b.acq(2, 1); b.wr(2, 0x20); b.rel(2, 1)  # 8..10 (writes z: rule (i) from 3 and 6)
    b.rd(2, 0x10)                 # 11: ordered after 0 via 3 <(i) 9
    ev = b.build()
    geo = TG.Geometry(3, 3, THREAD)
    assert races(ev, geo, all_pairs=True) == {(0, 7), (7, 11)}
    # HB orders 0 before 7 through the unrelated sections; 7 follows thread 1's last
    # release, so HB leaves (7, 11) unordered as well.
    assert races(ev, geo, all_pairs=True, hb_only=True) == {(7, 11)}


# ---- readings with switchable alternatives -----------------------------------------

def test_atomic_scope_reading():
    """A6: a block-scoped atomic and a device-scoped atomic from different blocks.
    Overlap reading: exempt. 'Lesser scope covers both' reading: race."""
    b = TG.TraceBuilder()
    b.atomic(0, 0x40, scope=CTA)
    b.atomic(2, 0x40, scope=DEVICE)
    ev = b.build()
    geo = TG.Geometry(4, 2, THREAD)
    assert races(ev, geo) == set()
    assert races(ev, geo, atomic_scope_lesser=True) == {(0, 1)}


def test_release_scope_reading():
    """A2: at a device-scoped release, a popped record of another block's block-scoped
    section is joined under the overlap reading and not under the literal IEEE test.
    Thread 2 learns thread 3's write through lock q inside its block-scoped section on
    l; thread 0 learns thread 2's acquire of l through rule (i) on lock m, then releases
    l at device scope. Only the joined record carries thread 3's write to thread 0."""
    b = TG.TraceBuilder()
    b.wr(3, 0x50)                                   # 0
    b.acq(3, 9, DEVICE); b.rel(3, 9, DEVICE)        # 1, 2   (lock q)
    b.acq(2, 3, CTA)                                # 3      (lock l, block 1)
    b.acq(2, 4, DEVICE); b.wr(2, 0x60); b.rel(2, 4, DEVICE)   # 4..6  (lock m)
    b.acq(2, 9, DEVICE); b.rel(2, 9, DEVICE)        # 7, 8
    b.rel(2, 3, CTA)                                # 9
    b.acq(0, 4, DEVICE); b.rd(0, 0x60); b.rel(0, 4, DEVICE)   # 10..12
    b.acq(0, 3, DEVICE); b.rel(0, 3, DEVICE)        # 13, 14
    b.rd(0, 0x50)                                   # 15
    ev = b.build()
    geo = TG.Geometry(4, 2, THREAD)
    assert races(ev, geo) == set()
    assert races(ev, geo, release_scope_ieee=True) == {(0, 15)}


# ---- validation (well-formedness W1-W4) --------------------------------------------

def _bad(rows, geo=(4, 2, 0)):
    ev = np.zeros(len(rows), dtype=TG.EVENT_DTYPE)
    for i, r in enumerate(rows):
        ev[i] = r
    return O.validate(ev, *geo)


def test_validation_rejects():
    ok = [(0, ACQ, DEVICE, 0, 0, 1), (0, REL, DEVICE, 0, 0, 1)]
    assert _bad(ok) == (0, 2**64 - 1)
    assert _bad([(9, READ, 0, 0, 0, 1)]) == (O.ERR_INVALID_TRACE, 0)            # W1 agent
    assert _bad([(0, 7, 0, 0, 0, 1)]) == (O.ERR_INVALID_TRACE, 0)               # W1 op
    assert _bad([(0, REL, DEVICE, 0, 0, 1)]) == (O.ERR_INVALID_TRACE, 0)        # W2 unmatched
    assert _bad([(0, ACQ, DEVICE, 0, 0, 1), (0, ACQ, DEVICE, 0, 0, 2), (0, REL, DEVICE, 0, 0, 1)]) == (
        O.ERR_INVALID_TRACE, 2)                                                 # W2 not LIFO
    assert _bad([(0, ACQ, DEVICE, 0, 0, 1), (0, REL, CTA, 0, 0, 1)]) == (O.ERR_INVALID_TRACE, 1)  # scope
    assert _bad([(0, ACQ, DEVICE, 0, 0, 1), (2, ACQ, CTA, 0, 0, 1)]) == (O.ERR_INVALID_TRACE, 1)  # W3
    assert _bad([(0, ACQ, CTA, 0, 0, 1), (1, ACQ, CTA, 0, 0, 1)]) == (O.ERR_INVALID_TRACE, 1)    # W3 blk
    assert _bad([(0, ACQ, CTA, 0, 0, 1), (2, ACQ, CTA, 0, 0, 1)])[0] == 0       # other block: fine
    assert _bad([(0, BARRIER, CTA, 0, 0, 2)]) == (O.ERR_INVALID_TRACE, 0)       # no block 2
    assert _bad([(0, READ, 2, 0, 0, 1)]) == (O.ERR_INVALID_TRACE, 0)            # WARP scope on access
    assert _bad([(0, READ, 0, 1, 0, 1 << 41)]) == (O.ERR_INVALID_TRACE, 0)      # shared addr too wide
    deep = [(0, ACQ, DEVICE, 0, 0, k) for k in range(5)]
    assert _bad(deep) == (O.ERR_INVALID_TRACE, 4)                               # nesting > 4


def test_warp_barrier_members_thread_granularity():
    """A warp-scope barrier at thread granularity orders only the lanes in its mask."""
    b = TG.TraceBuilder()
    b.wr(0, 0x10); b.wr(1, 0x14); b.wr(2, 0x18)
    b.syncwarp(0, mask=0b011)
    b.rd(1, 0x10); b.rd(0, 0x14); b.rd(1, 0x18)
    ev = b.build()
    assert races(ev, TG.Geometry(4, 4, THREAD)) == {(2, 6)}


def test_shared_memory_keyed_per_block():
    b = TG.TraceBuilder()
    b.wr(0, 0x10, shared=True)
    b.wr(2, 0x10, shared=True)   # another block: a different location
    b.wr(1, 0x10, shared=True)   # same block as 0: races
    ev = b.build()
    assert races(ev, TG.Geometry(4, 2, THREAD)) == {(0, 2)}


# ---- generated workload traces ----------------------------------------------------

@pytest.mark.parametrize("seed", [1, 2, 3])
def test_tiny_workload_planted(seed):
    """The tiny workload (1 block x 64 threads, 10k events) has no race except those that
    involve a planted event, and each planted event appears in a race."""
    ev, geo, planted = TG.generate(seed, workload="tiny_1blk_64thr_10k")
    assert len(planted) == 4
    r = O.run(ev, *geo.astuple())
    pl = set(planted.tolist())
    got = O.race_set(r)
    assert got, "planted races must show"
    assert all(a in pl or b in pl for a, b in got)
    assert pl <= {x for p in got for x in p}
    assert r.counters["epoch_test_disagree"] == 0
    assert r.counters["invariant_violations"] == 0


def test_clock_capture_invariants():
    ev, geo = TG.random_small(3, "mixed", n_events=60)
    idx = list(range(len(ev)))
    r = O.run(ev, *geo.astuple(), clock_events=idx)
    for i in idx:
        if ev["op"][i] in (READ, WRITE, ATOMIC, ACQ, REL):
            t = int(ev["agent"][i])
            assert r.clocks_h[i][t] == r.clocks_c[i][t]      # H_t[t] = N_t
            assert (r.clocks_c[i] <= r.clocks_h[i]).all()    # GWCP knowledge within HB knowledge
    # clocks of one thread never go down along its events
    for t in range(geo.num_agents):
        mine = [i for i in idx if ev["agent"][i] == t and ev["op"][i] in (READ, WRITE, ATOMIC, ACQ, REL)]
        for a, c in itertools.pairwise(mine):
            assert (r.clocks_c[a] <= r.clocks_c[c]).all()


def _location(ev, i, apb):
    shared = int(ev["space"][i]) == 1
    return (shared, int(ev["agent"][i]) // apb if shared else -1, int(ev["addr"][i]))


@pytest.mark.parametrize("seed", range(24))
def test_fasttrack_first_race_per_location(seed):
    # FastTrack's detector (last write as an epoch, last reads per agent), written here from
    # its published description and fed the oracle's clocks C_b, reports its first race on
    # a location at the same access b as the earliest race (a*, b) of the oracle's reading
    # of the race set on that location: before the first race every earlier conflicting
    # access is ordered, so the last write (or reads) is unordered iff some earlier one is.
    # Atomics are made plain writes so that no exemption is involved.
    fam = TG.FAMILIES[seed % len(TG.FAMILIES)]
    ev, geo = TG.random_small(seed, fam, n_events=160, num_agents=6, agents_per_block=3, n_locks=2, n_keys=4)
    ev = ev.copy()
    ev["op"][ev["op"] == ATOMIC] = WRITE
    acc = [i for i in range(len(ev)) if ev["op"][i] in (READ, WRITE)]
    r = O.run(ev, *geo.astuple(), clock_events=acc)
    apb = geo.agents_per_block
    W, R, first_ft = {}, {}, {}
    for b in acc:
        x, u, C = _location(ev, b, apb), int(ev["agent"][b]), r.clocks_c[b]
        racy = x in W and W[x][1] != u and W[x][0] > C[W[x][1]]
        if ev["op"][b] == WRITE:
            racy |= any(v != u and e > C[v] for v, e in R.get(x, {}).items())
            W[x] = (int(C[u]), u)
            R[x] = {}
        else:
            R.setdefault(x, {})[u] = int(C[u])
        if racy and x not in first_ft:
            first_ft[x] = b
    first_or = {}
    for a, b in r.races.tolist():
        x = _location(ev, b, apb)
        first_or[x] = min(first_or.get(x, b), b)
    assert first_ft == first_or
