"""Forced compression at barriers and compressed clock versions on the GPU (section "Vector
Clock Compression"), through the C ABI, against the oracle.

Forced compression renumbers local times: the clocks the library shows must equal the
forced oracle's, entry for entry, and the race set must equal the oracle's (which forced
compression does not change). Compressed versions store the clocks the check reads in the
block/warp form: the race set, the decoded clocks, the number of versions and the number
of words written must all equal the oracle's.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2111_12478_gb300 import tracegen as TG
from paper_2111_12478_gb300.tracegen import ACQ, ATOMIC, READ, REL, THREAD, WRITE

pytestmark = pytest.mark.gpu
WARP_GRAN = 1

GEOMS = [(4, 2, THREAD), (6, 3, THREAD), (8, 8, WARP_GRAN), (48, 24, THREAD), (64, 64, THREAD), (40, 8, WARP_GRAN),
         (96, 32, WARP_GRAN)]


@pytest.fixture(scope="module")
def gw():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__

    __graft_entry__.build()
    from paper_2111_12478_gb300 import gwcp

    return gwcp


def run(ctx, ev, geo):
    ctx.load_trace(ev, *geo.astuple())
    ctx.compute_order()
    return ctx.report_races()


def clocks_match(ctx, ev, geo, r, idx):
    for i in idx:
        assert np.array_equal(ctx.debug_clock(i, 0, geo.num_agents), r.clocks_c[i]), i
        if ev["op"][i] == REL:
            assert np.array_equal(ctx.debug_clock(i, 1, geo.num_agents), r.clocks_h[i]), i


def sample_events(ev, k, seed):
    idx = np.nonzero(np.isin(ev["op"], (READ, WRITE, ATOMIC, ACQ, REL)))[0]
    if len(idx) > k:
        idx = np.sort(np.random.default_rng(seed).choice(idx, k, replace=False))
    return [int(i) for i in idx]


@pytest.mark.parametrize("fam", TG.FAMILIES)
def test_forced_barrier_dense_and_compressed(gw, fam):
    forced = gw.Context(0, forced_barrier=True)
    comp = gw.Context(0)
    comp.set_clock_mode(gw.CLOCKS_COMPRESSED)
    try:
        for seed in range(8):
            for W, apb, gran in GEOMS:
                ev, geo = TG.random_small(seed, fam, n_events=160, num_agents=W, agents_per_block=apb,
                                          granularity=gran, n_locks=3, n_keys=5)
                idx = sample_events(ev, 40, seed)
                r = O.run(ev, *geo.astuple(), forced_barrier=True, version_words=True, clock_events=idx)
                assert np.array_equal(r.races, O.run(ev, *geo.astuple()).races)
                for ctx in (forced, comp):
                    got = run(ctx, ev, geo)
                    assert np.array_equal(got, r.races), (fam, seed, W)
                    clocks_match(ctx, ev, geo, r, idx)
                    assert ctx.counters()["clock_versions"] == r.counters["versions"]
                cb = comp.clock_bytes()
                assert cb["stored"] == 4 * r.counters["version_words"], (fam, seed, W)
                assert cb["reserved"] >= cb["stored"]
                assert cb["dense"] == 4 * r.counters["versions"] * max(32, 1 << (W - 1).bit_length())
    finally:
        forced.close()
        comp.close()


def test_compressed_hb_only(gw):
    ctx = gw.Context(0, hb_only=True)
    ctx.set_clock_mode(gw.CLOCKS_COMPRESSED)
    try:
        for seed in range(6):
            for W, apb, gran in GEOMS:
                ev, geo = TG.random_small(seed, "mixed", n_events=160, num_agents=W, agents_per_block=apb,
                                          granularity=gran, n_locks=3, n_keys=5)
                r = O.run(ev, *geo.astuple(), hb_only=True, forced_barrier=True, version_words=True)
                assert np.array_equal(run(ctx, ev, geo), r.races)
                assert ctx.clock_bytes()["stored"] == 4 * r.counters["version_words"]
    finally:
        ctx.close()


def test_forced_barrier_tiles(gw):
    """Forced compression with tile clocks (the wide walker) and with the chunked check."""
    tiles = gw.Context(0, forced_barrier=True)
    tiles.set_clock_mode(gw.CLOCKS_TILES)
    chunked = gw.Context(0, forced_barrier=True)
    chunked.set_clock_mode(gw.CLOCKS_DENSE)
    chunked.set_check_mode(gw.CHECK_CHUNKED)
    try:
        for seed in range(6):
            for W, apb in [(8, 8), (40, 8), (96, 32)]:
                ev, geo = TG.random_small(seed, "mixed", n_events=200, num_agents=W, agents_per_block=apb,
                                          granularity=WARP_GRAN, n_locks=3, n_keys=5)
                idx = sample_events(ev, 30, seed)
                r = O.run(ev, *geo.astuple(), forced_barrier=True, clock_events=idx)
                for ctx in (tiles, chunked):
                    assert np.array_equal(run(ctx, ev, geo), r.races), (seed, W)
                    clocks_match(ctx, ev, geo, r, idx)
    finally:
        tiles.close()
        chunked.close()


def test_workload_sample_compressed(gw):
    """A 300k-event sample of the 8-block, 64-warp workload (several tiles of every kernel,
    ragged tails): races, sizes and sampled clocks equal the oracle's; the compressed
    versions take under half the dense bytes."""
    ev, geo, _ = TG.generate(3, workload="8blk_64warp_10M", n_events=300_000)
    idx = sample_events(ev, 60, 3)
    r = O.run(ev, *geo.astuple(), forced_barrier=True, version_words=True, clock_events=idx)
    with gw.Context(0) as ctx:
        ctx.set_clock_mode(gw.CLOCKS_COMPRESSED)
        assert np.array_equal(run(ctx, ev, geo), r.races)
        clocks_match(ctx, ev, geo, r, idx)
        cb = ctx.clock_bytes()
        assert cb["stored"] == 4 * r.counters["version_words"]
        assert cb["stored"] < 0.5 * cb["dense"]


def test_compressed_pool_grows_and_reruns(gw):
    """The pool is sized from the previous run: a larger trace in the same context outgrows
    it, and the analysis runs again with a pool of the counted size."""
    small, geo, _ = TG.generate(4, workload="8blk_64warp_10M", n_events=3_000)
    big, _, _ = TG.generate(5, workload="8blk_64warp_10M", n_events=1_000_000)
    W, B = geo.num_agents, geo.num_agents // geo.agents_per_block
    with gw.Context(0) as ctx:
        ctx.set_clock_mode(gw.CLOCKS_COMPRESSED)
        run(ctx, small, geo)
        cb = ctx.clock_bytes()
        taken = (cb["reserved"] - 4 * B * ctx.counters()["clock_versions"]) // 4
        cap_after_small = taken + taken // 8 + W * 2048
        got = run(ctx, big, geo)
        pool_words = ctx.clock_bytes()["stored"] // 4 - B * ctx.counters()["clock_versions"]
        assert pool_words > cap_after_small  # the first pool could not hold it
        with gw.Context(0) as dense:
            dense.set_clock_mode(gw.CLOCKS_DENSE)
            assert np.array_equal(got, run(dense, big, geo))


def test_compressed_mode_limits(gw):
    ev, geo, _ = TG.generate(1, workload="256blk_8192warp_200M", n_events=20_000)
    with gw.Context(0) as ctx:
        ctx.set_clock_mode(gw.CLOCKS_COMPRESSED)
        with pytest.raises(gw.GwcpError) as ei:
            ctx.load_trace(ev, *geo.astuple())
        assert ei.value.code == gw.ERR_UNSUPPORTED
        empty = np.zeros(0, dtype=TG.EVENT_DTYPE)
        assert len(run(ctx, empty, TG.Geometry(4, 2, THREAD))) == 0
        assert ctx.clock_bytes() == dict(dense=0, stored=0, reserved=0)
