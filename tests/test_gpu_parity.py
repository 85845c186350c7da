"""CUDA path vs the CPU oracle, through the C ABI (needs a GB300).

Race sets must be identical (integer work: bit-exact). Clock rows are compared at
sampled events through gwcp_debug_clock. Invalid traces must fail with the oracle's
first bad index.
"""
import numpy as np
import pytest

from conftest import GOLDEN_FILES, load_golden
from oracle import oracle as O
from paper_2111_12478_gb300 import tracegen as TG
from paper_2111_12478_gb300.tracegen import ACQ, ATOMIC, BARRIER, CTA, DEVICE, READ, REL, THREAD, WARP_GRAN, WRITE

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__

    __graft_entry__.build()
    from paper_2111_12478_gb300 import gwcp

    c = gwcp.Context(0)
    yield c
    c.close()


def gpu_races(ctx, ev, geo):
    ctx.load_trace(ev, *geo.astuple())
    ctx.compute_order()
    return ctx.report_races()


def same(ctx, ev, geo):
    got = gpu_races(ctx, ev, geo)
    want = O.run(ev, *geo.astuple()).races
    assert got.shape == want.shape, (len(got), len(want))
    assert np.array_equal(got, want)
    return got


@pytest.mark.parametrize("name", GOLDEN_FILES)
def test_figures(ctx, name):
    ev, geo, expect = load_golden(name)
    got = gpu_races(ctx, ev, geo)
    assert {(int(a), int(b)) for a, b in got} == expect


@pytest.mark.parametrize("fam", TG.FAMILIES)
def test_random_families(ctx, fam):
    for seed in range(30):
        for W, apb, gran in [(4, 2, THREAD), (6, 3, THREAD), (8, 8, WARP_GRAN), (64, 64, THREAD), (40, 8, WARP_GRAN)]:
            ev, geo = TG.random_small(seed, fam, n_events=120, num_agents=W, agents_per_block=apb,
                                      granularity=gran, n_locks=3, n_keys=5)
            same(ctx, ev, geo)


def test_clock_rows_match_oracle(ctx):
    for seed in range(6):
        ev, geo = TG.random_small(seed, "mixed", n_events=200, num_agents=8, agents_per_block=4, n_locks=3,
                                  n_keys=4)
        idx = [i for i in range(len(ev)) if ev["op"][i] in (READ, WRITE, ATOMIC, ACQ, REL)]
        r = O.run(ev, *geo.astuple(), clock_events=idx)
        gpu_races(ctx, ev, geo)
        for i in idx:
            c = ctx.debug_clock(i, 0, geo.num_agents)
            assert np.array_equal(c, r.clocks_c[i]), (seed, i)
            if ev["op"][i] == REL:
                h = ctx.debug_clock(i, 1, geo.num_agents)
                assert np.array_equal(h, r.clocks_h[i]), (seed, i)


def test_edge_cases(ctx):
    geo = TG.Geometry(4, 2, THREAD)
    assert len(gpu_races(ctx, np.zeros(0, dtype=TG.EVENT_DTYPE), geo)) == 0
    b = TG.TraceBuilder()
    b.wr(0, 0x10)
    same(ctx, b.build(), geo)                                   # one access
    b = TG.TraceBuilder()
    b.acq(0, 1); b.rel(0, 1); b.barrier(0, agent=0); b.fence(1)
    same(ctx, b.build(), geo)                                   # no accesses
    b = TG.TraceBuilder()
    for k in range(4):
        b.acq(0, k)
    b.wr(0, 0x20); b.wr(1, 0x20)
    for k in reversed(range(4)):
        b.rel(0, k)
    b.acq(1, 2); b.rd(1, 0x20)                                  # depth 4, open section at the end
    same(ctx, b.build(), geo)
    ev, geo1 = TG.random_small(1, "mixed", n_events=80, num_agents=1, agents_per_block=1)
    same(ctx, ev, geo1)                                         # one agent
    ev, geo2 = TG.random_small(2, "mixed", n_events=200, num_agents=16, agents_per_block=1, granularity=WARP_GRAN)
    same(ctx, ev, geo2)                                         # one agent per block


@pytest.mark.parametrize("W,apb,gran", [(1024, 32, WARP_GRAN), (512, 16, WARP_GRAN), (256, 16, WARP_GRAN),
                                        (96, 96, THREAD), (128, 64, THREAD)])
def test_wide_clocks(ctx, W, apb, gran):
    # register-resident (dense) clocks at every width they take
    from paper_2111_12478_gb300 import gwcp

    ev, geo = TG.random_small(7, "mixed", n_events=3000, num_agents=W, agents_per_block=apb, granularity=gran,
                              n_locks=6, n_keys=12)
    with gwcp.Context(0) as c:
        c.set_clock_mode(gwcp.CLOCKS_DENSE)
        same(c, ev, geo)


# ---- clocks wider than 1024 agents: tables of copy-on-write tiles -------------------------

@pytest.mark.parametrize("W,apb", [(1088, 32), (1280, 16), (2048, 32)])
def test_tiled_random(ctx, W, apb):
    # 1088 agents: a ragged last tile; 1280/16: five tiles, a block of 16 per CTA
    for fam in ("mixed", "uniform_bar", "dev_locks", "barriers", "nosync"):
        for seed in range(2):
            ev, geo = TG.random_small(seed, fam, n_events=5000, num_agents=W, agents_per_block=apb,
                                      granularity=WARP_GRAN, n_locks=4, n_keys=8)
            same(ctx, ev, geo)


@pytest.mark.parametrize("W,apb", [(2080, 32), (4096, 16)])
def test_agent_sorted_stream(ctx, W, apb):
    # more than 2048 agents: phase A builds the agent-sorted stream by a sort on the agent
    # (2080 agents: a ragged last tile), and the check runs on the grouped order with the
    # written-location filter
    from paper_2111_12478_gb300 import gwcp

    for fam in TG.FAMILIES:
        ev, geo = TG.random_small(3, fam, n_events=6000, num_agents=W, agents_per_block=apb,
                                  granularity=WARP_GRAN, n_locks=4, n_keys=8)
        same(ctx, ev, geo)
    b = TG.TraceBuilder()  # synchronisation only
    b.acq(0, 1)
    b.rel(0, 1)
    b.barrier(W // apb - 1, apb=apb)
    b.acq(W - 1, 1)
    b.rel(W - 1, 1)
    assert len(same(ctx, b.build(), TG.Geometry(W, apb, WARP_GRAN))) == 0
    b = TG.TraceBuilder()  # reads only: the filter leaves nothing to check
    for k in range(64):
        b.rd(k * 37 % W, 0x100 + 4 * (k % 5))
    assert len(same(ctx, b.build(), TG.Geometry(W, apb, WARP_GRAN))) == 0
    b = TG.TraceBuilder()  # one write among reads of the same location: races with each later read
    b.wr(5, 0x40)
    for k in range(1, 40):
        b.rd(k * 53 % W, 0x40)
    same(ctx, b.build(), TG.Geometry(W, apb, WARP_GRAN))
    # an event that breaks W1 (agent out of range) after some valid ones
    ev, geo = TG.random_small(4, "mixed", n_events=3000, num_agents=W, agents_per_block=apb,
                              granularity=WARP_GRAN, n_locks=4, n_keys=8)
    ev = ev.copy()
    ev["agent"][1777] = W + 5
    rc, bad = O.validate(ev, *geo.astuple())
    assert rc == O.ERR_INVALID_TRACE and bad == 1777
    ctx.load_trace(ev, *geo.astuple())
    with pytest.raises(gwcp.GwcpError) as ei:
        ctx.compute_order()
    assert ei.value.code == gwcp.ERR_INVALID_TRACE and ei.value.bad_index == bad


@pytest.mark.parametrize("W,apb", [(64, 8), (256, 32), (512, 16), (1024, 32)])
def test_tiles_at_dense_widths(W, apb):
    # the tile-table clocks at widths the register clocks also take: same races as the oracle
    pytest.importorskip("torch")
    from paper_2111_12478_gb300 import gwcp

    with gwcp.Context(0) as c:
        c.set_clock_mode(gwcp.CLOCKS_TILES)
        cases = [TG.random_small(seed, fam, n_events=3000, num_agents=W, agents_per_block=apb, granularity=WARP_GRAN,
                                 n_locks=4, n_keys=8)
                 for fam in ("mixed", "uniform_bar", "dev_locks", "barriers", "nosync") for seed in range(2)]
        nb = W // apb
        cases.append(TG.generate(5, n_events=100_000, workload="8blk_64warp_10M", num_blocks=nb,
                                 agents_per_block=apb)[:2])
        for ev, geo in cases:
            c.load_trace(ev, *geo.astuple())
            c.compute_order()
            assert np.array_equal(c.report_races(), O.run(ev, *geo.astuple()).races)
        # thread granularity cannot use tiles
        ev, geo = TG.random_small(0, "mixed", n_events=100, num_agents=8, agents_per_block=4)
        with pytest.raises(gwcp.GwcpError) as ei:
            c.load_trace(ev, *geo.astuple())
        assert ei.value.code == gwcp.ERR_UNSUPPORTED


def test_tiled_clock_rows(ctx):
    ev, geo = TG.random_small(3, "mixed", n_events=4000, num_agents=1280, agents_per_block=16,
                              granularity=WARP_GRAN, n_locks=4, n_keys=6)
    rng = np.random.default_rng(0)
    cand = [i for i in range(len(ev)) if ev["op"][i] in (READ, WRITE, ATOMIC, ACQ, REL)]
    idx = sorted(rng.choice(cand, size=300, replace=False).tolist())
    r = O.run(ev, *geo.astuple(), clock_events=idx)
    gpu_races(ctx, ev, geo)
    for i in idx:
        assert np.array_equal(ctx.debug_clock(i, 0, geo.num_agents), r.clocks_c[i]), i
        if ev["op"][i] == REL:
            assert np.array_equal(ctx.debug_clock(i, 1, geo.num_agents), r.clocks_h[i]), i


@pytest.mark.parametrize("blocks,n,seed", [(64, 300_000, 1), (256, 150_000, 2), (256, 1_000_000, 3)])
def test_tiled_workload(ctx, blocks, n, seed):
    # the 8192-warp workload's shape (scoped sync 1%, Zipf(1.05)) on few addresses
    ev, geo, _ = TG.generate(seed, n_events=n, workload="256blk_8192warp_200M", num_blocks=blocks, n_ranks=2000,
                             plant_min_rank=64)
    got = same(ctx, ev, geo)
    assert len(got) > 0


def test_invalid_traces_first_bad_index(ctx):
    from paper_2111_12478_gb300 import gwcp

    cases = [
        [(0, ACQ, DEVICE, 0, 0, 1), (9, READ, 0, 0, 0, 1)],                         # W1
        [(0, REL, DEVICE, 0, 0, 1)],                                                 # W2
        [(0, ACQ, DEVICE, 0, 0, 1), (0, ACQ, DEVICE, 0, 0, 2), (0, REL, DEVICE, 0, 0, 1)],
        [(0, ACQ, DEVICE, 0, 0, 1), (2, ACQ, CTA, 0, 0, 1), (0, 7, 0, 0, 0, 0)],     # W3 before W1
        [(0, ACQ, CTA, 0, 0, 1), (1, ACQ, CTA, 0, 0, 1), (1, REL, DEVICE, 0, 0, 5)],  # W3 before W2
        [(0, ACQ, DEVICE, 0, 0, k) for k in range(5)],                               # nesting > 4
        [(0, BARRIER, CTA, 0, 0, 7)],
    ]
    for rows in cases:
        ev = np.zeros(len(rows), dtype=TG.EVENT_DTYPE)
        for i, r in enumerate(rows):
            ev[i] = r
        rc, bad = O.validate(ev, 4, 2, THREAD)
        assert rc == O.ERR_INVALID_TRACE
        ctx.load_trace(ev, 4, 2, THREAD)
        with pytest.raises(gwcp.GwcpError) as ei:
            ctx.compute_order()
        assert ei.value.code == gwcp.ERR_INVALID_TRACE
        assert ei.value.bad_index == bad, rows


def test_tiny_workload(ctx):
    for seed in (1, 2, 3):
        ev, geo, planted = TG.generate(seed, workload="tiny_1blk_64thr_10k")
        got = same(ctx, ev, geo)
        assert set(planted.tolist()) <= set(got.ravel().tolist())


@pytest.mark.parametrize("n,seed", [(200_000, 1), (200_000, 2), (1_000_000, 3)])
def test_warp_workload_scaled(ctx, n, seed):
    ev, geo, _ = TG.generate(seed, n_events=n, workload="8blk_64warp_10M")
    same(ctx, ev, geo)


def test_warp_workload_full_10M(ctx):
    """The 8-block, 64-warp, 10M-event workload at full size: the whole race set."""
    ev, geo, planted = TG.generate(1, workload="8blk_64warp_10M")
    got = same(ctx, ev, geo)
    pl = set(planted.tolist())
    assert all(int(a) in pl or int(b) in pl for a, b in got)


def test_capacity_and_determinism(ctx):
    from paper_2111_12478_gb300 import gwcp

    ev, geo, _ = TG.generate(4, n_events=100_000, workload="8blk_64warp_10M")
    a = gpu_races(ctx, ev, geo)
    b = gpu_races(ctx, ev, geo)
    assert np.array_equal(a, b)
    with gwcp.Context(0, race_capacity=max(1, len(a) // 2)) as small:
        small.load_trace(ev, *geo.astuple())
        small.compute_order()
        with pytest.raises(gwcp.GwcpError) as ei:
            small.report_races(cap=len(a))
        assert ei.value.code == gwcp.ERR_CAPACITY
        assert small.race_count() == len(a)


def test_more_races_than_events(ctx):
    # no synchronisation: 1024 agents each read a location, then agents 0 and 1 write it.
    # The first write races with the 1023 other readers, the second with the 1022 readers
    # other than agents 0 and 1 and with the first write: 2046 races per 1026 events,
    # more than the automatic race buffer's first size (max(2^20, n))
    W, n_loc = 1024, 600
    per = W + 2
    ev = np.zeros(n_loc * per, dtype=TG.EVENT_DTYPE)
    for x in range(n_loc):
        o = x * per
        ev["agent"][o:o + W] = np.arange(W)
        ev["op"][o:o + W] = READ
        ev["agent"][o + W], ev["agent"][o + W + 1] = 0, 1
        ev["op"][o + W:o + W + 2] = WRITE
        ev["addr"][o:o + per] = 64 * (x + 1)
    geo = TG.Geometry(W, 32, WARP_GRAN)
    got = gpu_races(ctx, ev, geo)
    assert len(got) == n_loc * 2046 > max(1 << 20, len(ev))
    w1 = np.arange(n_loc) * per + W
    first = got[np.isin(got[:, 1], w1)]
    assert len(first) == n_loc * 1023 and set(np.unique(first[:, 1]).tolist()) == set(w1.tolist())
    assert np.array_equal(got, O.run(ev, *geo.astuple()).races)


@pytest.mark.parametrize("mode", [1, 2])
def test_check_modes_dense_clocks(mode):
    # the chunked check and the partner-group check over dense register clocks
    pytest.importorskip("torch")
    from paper_2111_12478_gb300 import gwcp, ranker

    with gwcp.Context(0, timeline=True) as c:
        c.set_clock_mode(gwcp.CLOCKS_DENSE)
        c.set_check_mode(mode)
        for W, apb, gran in [(4, 2, THREAD), (64, 64, THREAD), (40, 8, WARP_GRAN), (256, 16, WARP_GRAN)]:
            for fam in TG.FAMILIES:
                for seed in range(4):
                    ev, geo = TG.random_small(seed, fam, n_events=300, num_agents=W, agents_per_block=apb,
                                              granularity=gran, n_locks=3, n_keys=5)
                    same(c, ev, geo)
        for ev, geo in (TG.generate(2, workload="tiny_1blk_64thr_10k")[:2],
                        TG.generate(8, n_events=200_000, workload="8blk_64warp_10M")[:2]):
            want = same(c, ev, geo)
            c.set_ranker(ranker.init_theta(3))  # a ranked order: same races, full timeline
            got = gpu_races(c, ev, geo)
            _, _, per = c.check_timeline()
            c.set_ranker(None)
            assert np.array_equal(got, want) and int(per.sum()) == len(want)


@pytest.mark.parametrize("mode", [1, 2])
def test_hb_only_variant(mode):
    # the paper's happens-before baseline (H clocks) on both clock representations: the
    # oracle's HB-only race set, contained in the GWCP race set (C_t <= H_t: GWCP orders
    # fewer pairs and predicts the races HB misses)
    pytest.importorskip("torch")
    from paper_2111_12478_gb300 import gwcp

    cases = [TG.random_small(seed, fam, n_events=600, num_agents=16, agents_per_block=8, granularity=WARP_GRAN,
                             n_locks=3, n_keys=6)
             for fam in TG.FAMILIES for seed in range(3)]
    cases.append(TG.generate(6, n_events=150_000, workload="8blk_64warp_10M")[:2])
    n_more = 0
    with gwcp.Context(0, hb_only=True) as h, gwcp.Context(0) as w:
        h.set_clock_mode(mode)
        for ev, geo in cases:
            h.load_trace(ev, *geo.astuple())
            h.compute_order()
            hb = h.report_races()
            assert np.array_equal(hb, O.run(ev, *geo.astuple(), hb_only=True).races)
            gw = gpu_races(w, ev, geo)
            assert {tuple(r) for r in hb.tolist()} <= {tuple(r) for r in gw.tolist()}
            n_more += len(gw) - len(hb)
    assert n_more > 0  # GWCP predicts races that HB misses


def test_bounded_wait_gives_up_and_device_stays_usable(ctx):
    # failure detection without a fault: the walkers' bounded wait on a clock row that
    # nothing completes gives up with a timeout status; the next analysis runs normally
    import time

    from paper_2111_12478_gb300 import gwcp

    t0 = time.perf_counter()
    assert gwcp.debug_wait_timeout(0, 20_000) == gwcp.ERR_TIMEOUT
    assert time.perf_counter() - t0 < 10
    ev, geo, _ = TG.generate(2, workload="tiny_1blk_64thr_10k")
    same(ctx, ev, geo)


def test_injected_oom_leaves_the_context_usable():
    # failure detection without a fault: a memory cap on the context makes the analysis
    # fail with OOM, as an exhausted device would; raised again, the next compute is exact
    from paper_2111_12478_gb300 import gwcp

    ev, geo, _ = TG.generate(6, n_events=200_000, workload="8blk_64warp_10M")
    want = O.run(ev, *geo.astuple()).races
    with gwcp.Context(0) as c:
        c.load_trace(ev, *geo.astuple())
        c.debug_alloc_limit(4 << 20)
        with pytest.raises(gwcp.GwcpError) as ei:
            c.compute_order()
        assert ei.value.code == gwcp.ERR_OOM
        with pytest.raises(gwcp.GwcpError) as ei:
            c.report_races()
        assert ei.value.code == gwcp.ERR_OOM
        c.debug_alloc_limit(0)
        c.compute_order()
        assert np.array_equal(c.report_races(), want)


def test_device_input_and_stream(ctx):
    import torch

    ev, geo, _ = TG.generate(5, n_events=50_000, workload="8blk_64warp_10M")
    dev = torch.from_numpy(ev.view(np.uint8).copy()).cuda()
    s = torch.cuda.Stream()
    ctx.load_trace(dev, *geo.astuple(), stream=s)
    ctx.compute_order(stream=s)
    got = ctx.report_races(stream=s)
    assert np.array_equal(got, O.run(ev, *geo.astuple()).races)
