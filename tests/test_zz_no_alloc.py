"""gwcp_analyze_noalloc: the allocation-free entry point, for callers that cannot
allocate device memory when they need a trace analysed (a hook running while another
component owns the memory pool, or code that must not call cudaMalloc/cudaFree since
those can synchronise the device). Its races must equal the context-based entry points'
(gwcp_compute_order + gwcp_report_races) exactly, on two calls in a row that share the
entry point's scratch array; once set up, a call leaves the device's free memory
unchanged. Collected last so a failure here stops a -x run only after every other test
has run."""
import numpy as np
import pytest

from paper_2111_12478_gb300 import tracegen as TG

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__

    __graft_entry__.build()
    from paper_2111_12478_gb300 import gwcp

    return torch, gwcp


def _reference(gwcp, ev, geo):
    with gwcp.Context(0) as c:
        c.load_trace(ev, *geo.astuple())
        c.compute_order()
        return c.report_races()


def _noalloc(torch, gwcp, ev, geo, cap):
    dev = torch.from_numpy(ev.view(np.uint8).copy()).cuda()
    out = torch.zeros((max(cap, 1), 2), dtype=torch.int64, device="cuda")
    torch.cuda.synchronize()
    rc, n, bad = gwcp.analyze_noalloc(dev.data_ptr(), len(ev), *geo.astuple(), out.data_ptr(), cap)
    return rc, n, bad, out.cpu().numpy().astype(np.uint64)[: min(n, cap)]


def test_noalloc_matches_compute_order_twice(env):
    torch, gwcp = env
    traces = [TG.generate(1, workload="tiny_1blk_64thr_10k")[:2],
              TG.generate(2, n_events=100_000, workload="8blk_64warp_10M")[:2]]
    for ev, geo in traces + traces[:1]:  # back to back, and the first trace again after the second
        want = _reference(gwcp, ev, geo)
        rc, n, bad, got = _noalloc(torch, gwcp, ev, geo, len(want) + 16)
        assert rc == 0, gwcp.strerror(rc)
        assert n == len(want)
        assert np.array_equal(got, want)


def test_noalloc_limits_and_errors(env):
    torch, gwcp = env
    ev, geo = TG.random_small(3, "mixed", n_events=200, num_agents=8, agents_per_block=4)
    want = _reference(gwcp, ev, geo)
    if len(want) > 1:
        rc, n, _, got = _noalloc(torch, gwcp, ev, geo, 1)
        assert rc == gwcp.ERR_CAPACITY and n == len(want) and np.array_equal(got, want[:1])
    big = np.zeros((1 << 18) + 1, dtype=TG.EVENT_DTYPE)
    rc, _, _, _ = _noalloc(torch, gwcp, big, TG.Geometry(4, 2, TG.THREAD), 1)
    assert rc == gwcp.ERR_UNSUPPORTED
    bad = np.zeros(3, dtype=TG.EVENT_DTYPE)
    bad[1] = (9, TG.READ, 0, 0, 0, 1)
    rc, _, idx, _ = _noalloc(torch, gwcp, bad, TG.Geometry(4, 2, TG.THREAD), 1)
    assert rc == gwcp.ERR_INVALID_TRACE and idx == 1


def test_noalloc_reserves_nothing_after_setup(env):
    torch, gwcp = env
    ev, geo = TG.generate(3, n_events=50_000, workload="8blk_64warp_10M")[:2]
    want = _reference(gwcp, ev, geo)
    # set-up: a zero-length call loads the entry point's device code on this device
    rc, n, _ = gwcp.analyze_noalloc(0, 0, *geo.astuple(), 0, 0)
    assert rc == 0 and n == 0
    dev = torch.from_numpy(ev.view(np.uint8).copy()).cuda()
    out = torch.zeros((len(want) + 16, 2), dtype=torch.int64, device="cuda")
    torch.cuda.synchronize()
    assert gwcp.analyze_noalloc(dev.data_ptr(), len(ev), *geo.astuple(), out.data_ptr(), len(want) + 16)[0] == 0
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    rc, n, _ = gwcp.analyze_noalloc(dev.data_ptr(), len(ev), *geo.astuple(), out.data_ptr(), len(want) + 16)
    torch.cuda.synchronize()
    free1 = torch.cuda.mem_get_info()[0]
    assert rc == 0 and n == len(want)
    assert np.array_equal(out.cpu().numpy().astype(np.uint64)[:n], want)
    assert free1 == free0, f"device free memory changed by {free0 - free1} bytes"


def test_noalloc_invalid_trace_at_the_size_limit(env):
    """A trace of the maximum length whose intermediates would not fit the scratch, made
    invalid by its last event (a second device-scoped acquire of a held lock, W3): the
    entry point reports the invalid trace and its index, as the context path does."""
    torch, gwcp = env
    n = 1 << 18
    ev = np.zeros(n, dtype=TG.EVENT_DTYPE)
    ev["agent"] = 0
    ev["op"] = TG.READ
    ev["addr"] = np.arange(n, dtype=np.uint64) * 8
    ev[0] = (0, TG.ACQ, TG.DEVICE, 0, 0, 7)
    ev[n - 1] = (32, TG.ACQ, TG.DEVICE, 0, 0, 7)
    geo = TG.Geometry(256, 32, TG.WARP_GRAN)
    with gwcp.Context(0) as c:
        c.load_trace(ev, *geo.astuple())
        with pytest.raises(gwcp.GwcpError) as e:
            c.compute_order()
    assert e.value.code == gwcp.ERR_INVALID_TRACE and e.value.bad_index == n - 1
    rc, _, idx, _ = _noalloc(torch, gwcp, ev, geo, 1)
    assert rc == gwcp.ERR_INVALID_TRACE and idx == n - 1
