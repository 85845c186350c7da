"""Host-side logic that needs no GPU: the batched and served input recipes, the ranker's
host helpers, and that the product fails loudly without its library or without a GPU
(there is no CPU path)."""
import math

import numpy as np
import pytest

from oracle import ranker as R
from paper_2111_12478_gb300 import tracegen as TG


def test_batch_specs_follow_the_recipe():
    specs = TG.many_specs(1, **TG.BATCH_WORKLOAD)
    assert len(specs) == 512
    n = np.array([s["n_events"] for s in specs])
    assert n.min() >= 10_000 and n.max() <= 5_000_000
    # log-uniform: the median of log(n) sits near the middle of [log 1e4, log 5e6]
    mid = 0.5 * (math.log(1e4) + math.log(5e6))
    assert abs(np.median(np.log(n)) - mid) < 0.4
    widths = {s["num_blocks"] * s["agents_per_block"] for s in specs}
    assert widths == set(TG.BATCH_WIDTHS)
    for s in specs:
        W = s["num_blocks"] * s["agents_per_block"]
        assert s["agents_per_block"] <= 32 and s["num_blocks"] <= 128 and W % s["agents_per_block"] == 0
    assert len({s["seed"] for s in specs}) == 512
    assert specs == TG.many_specs(1, **TG.BATCH_WORKLOAD)  # deterministic


def test_serve_requests_are_poisson():
    arr, wid, lens = TG.serve_requests(3, 20_000, 200.0, 10_000, 20_000_000)
    gaps = np.diff(np.r_[0.0, arr])
    assert (gaps > 0).all()
    assert abs(gaps.mean() - 1 / 200) < 0.1 / 200      # rate 200/s
    assert abs(gaps.std() / gaps.mean() - 1) < 0.05    # exponential: cv = 1
    assert set(np.unique(wid).tolist()) == set(range(len(TG.BATCH_WIDTHS)))
    assert lens.min() >= 10_000 and lens.max() <= 20_000_000


def test_location_keys_match_the_oracles():
    import ranker_metrics as ranker

    ev, _ = TG.random_small(4, "mixed", n_events=300, num_agents=16, agents_per_block=4)
    acc = ev[ev["op"] <= TG.ATOMIC]
    assert np.array_equal(ranker.location_keys(acc, 4), R.location_keys(acc, 4))


def test_racy_location_recall_by_brute_force():
    import ranker_metrics as ranker

    ev, _ = TG.random_small(5, "nosync", n_events=200, num_agents=8, agents_per_block=4, n_keys=12)
    keys = np.unique(ranker.location_keys(ev[ev["op"] <= TG.ATOMIC], 4))
    rng = np.random.default_rng(0)
    order = keys[rng.permutation(len(keys))]
    idx = np.nonzero(ev["op"] <= TG.ATOMIC)[0]
    races = np.stack([idx[:-1], idx[1:]], axis=1)[::3].astype(np.uint64)
    racy = {int(k) for k in ranker.location_keys(ev[races[:, 1].astype(np.int64)], 4)}
    k = max(1, int(len(order) * 0.25))
    want = sum(int(x) in racy for x in order[:k]) / len(racy)
    assert ranker.racy_location_recall(ev, 4, races, order, 0.25) == pytest.approx(want)


def test_timeline_summary():
    from paper_2111_12478_gb300 import ranker

    ends = np.array([110, 120, 130, 140, 150, 160, 170, 180, 190, 200], dtype=np.uint64)
    per = np.array([0, 0, 3, 0, 1, 0, 0, 4, 0, 2], dtype=np.uint32)
    s = ranker.timeline_summary(100, ends, per)
    assert s["races"] == 10 and s["chunks"] == 10
    assert s["first_race_us"] == pytest.approx(0.030)    # chunk ending at 130 ns
    assert s["half_races_us"] == pytest.approx(0.080)    # 5 of 10 races by 180 ns
    assert s["all_races_us"] == pytest.approx(0.100)
    assert s["races_in_first_10pct_chunks"] == 0.0


def test_init_theta_shape_and_scale():
    from paper_2111_12478_gb300 import ranker

    t = ranker.init_theta(3)
    assert t.dtype == np.float32 and t.size == R.N_PARAMS
    W1, b1, W2, b2, w3, b3 = R.split(t)
    assert not b1.any() and not b2.any() and not b3.any()
    assert abs(W1.std() - math.sqrt(2 / 16)) < 0.05 and abs(W2.std() - math.sqrt(2 / 64)) < 0.02


def test_shipped_weights_load():
    from paper_2111_12478_gb300 import ranker

    t = ranker.load_weights()
    assert t is not None and t.size == R.N_PARAMS and np.isfinite(t).all()


def test_missing_library_fails_loudly(monkeypatch):
    from paper_2111_12478_gb300 import gwcp

    monkeypatch.setattr(gwcp, "_lib", None)
    monkeypatch.setattr(gwcp, "LIB_PATH", "/nonexistent/libgwcp.so")
    with pytest.raises(RuntimeError, match="not built"):
        gwcp.load_library()


def test_without_a_gpu_contexts_fail_loudly():
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_2111_12478_gb300 import build as B
    from paper_2111_12478_gb300 import gwcp

    B.build()
    with pytest.raises(gwcp.GwcpError) as ei:
        gwcp.Context(0)
    assert ei.value.code == gwcp.ERR_CUDA
    with pytest.raises(gwcp.GwcpError):
        gwcp.Pool(0, lanes=2)


def test_argument_checks_before_any_cuda_call():
    """Entry points reject bad arguments on the host, before any CUDA call (so also here,
    without a GPU): null contexts, an unknown pool option value, reserved fields."""
    import ctypes

    from paper_2111_12478_gb300 import build as B
    from paper_2111_12478_gb300 import gwcp

    B.build()
    L = gwcp.load_library()
    out = (ctypes.c_uint64 * 3)()
    assert L.gwcp_clock_bytes(None, out) == gwcp.ERR_ARGS
    assert L.gwcp_debug_alloc_limit(None, 0) == gwcp.ERR_ARGS
    h = ctypes.c_void_p()
    for opt in (gwcp.PoolOptions(4, 0, 0, 0, 2), gwcp.PoolOptions(4, 2, 0, 0, 0), gwcp.PoolOptions(300, 0, 0, 0, 0)):
        assert L.gwcp_pool_create(ctypes.byref(h), 0, ctypes.byref(opt)) == gwcp.ERR_ARGS
    bad = gwcp.PoolOptions(4, 0, 0, 0, 0)
    bad.reserved[1] = 1
    assert L.gwcp_pool_create(ctypes.byref(h), 0, ctypes.byref(bad)) == gwcp.ERR_ARGS
