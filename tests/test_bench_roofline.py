"""The bench line's roofline arithmetic (CPU only): the propagation's algorithmic bytes are
12·W per join plus 8 per release-loop record visit (the tile-sparse figure for tiled
clocks: 1 KB per tile read or written plus the visits), achieved = bytes / kernel time,
frac = achieved / peak; the committed DRAM traffic is used only while the kernel's source
is the one it was measured on.
"""
import importlib.util
import json
import os

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def bench():
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    m = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(m)
    return m


CNT = {"joins": 1_000, "loop_visits": 500, "tiles_read": 300, "tiles_written": 40, "partner_tests": 70}


def test_dense_propagation_roofline(bench):
    W, ms, peak = 64, 2.0, 6785.5
    r = bench.prop_roofline("k_propagate", "no_such_workload", ms, CNT, W, False, peak, "measured")
    want = 12.0 * W * CNT["joins"] + 8.0 * CNT["loop_visits"]
    assert r["algorithmic_bytes"] == want
    assert r["achieved"] == pytest.approx(want / (ms / 1e3) / 1e9)
    assert r["frac"] == pytest.approx(r["achieved"] / peak)
    assert r["traffic"] is None and "dense_equivalent" not in r


def test_tiled_propagation_roofline(bench):
    W, ms, peak = 8192, 5.0, 6785.5
    r = bench.prop_roofline("k_prop_wide", "no_such_workload", ms, CNT, W, True, peak, "measured")
    want = 1024.0 * (CNT["tiles_read"] + CNT["tiles_written"]) + 8.0 * CNT["loop_visits"]
    assert r["algorithmic_bytes"] == want
    assert r["frac"] == pytest.approx(want / (ms / 1e3) / 1e9 / peak)
    dense = r["dense_equivalent"]
    assert dense["algorithmic_bytes"] == 12.0 * W * CNT["joins"] + 8.0 * CNT["loop_visits"]
    assert dense["frac"] == pytest.approx(dense["algorithmic_bytes"] / (ms / 1e3) / 1e9 / peak)


def test_check_roofline(bench):
    ms, peak, races = 0.5, 6785.5, 9
    r = bench.check_roofline(ms, 1.0e6, CNT, races, "no_such_workload", peak, "measured")
    want = 1.0e6 + 8.0 * CNT["partner_tests"] + 16.0 * races
    assert r["algorithmic_bytes"] == want
    assert r["frac"] == pytest.approx(want / (ms / 1e3) / 1e9 / peak)
    assert r["traffic"] is None and r["dram_frac"] is None


def test_committed_traffic_only_for_the_measured_source(bench):
    with open(os.path.join(ROOT, "profiles", "traffic.json")) as f:
        t = json.load(f)
    for key, e in t.items():
        if key.startswith("_"):
            continue
        kernel, workload = key.split("@")
        got = bench.traffic_for(kernel, workload)
        if e["source_sha"] == bench.source_hash(bench.KERNEL_SOURCES[kernel]):
            assert got == float(e["dram_bytes_per_launch"])
        else:
            assert got is None
    assert bench.traffic_for("k_prop_wide", "no_such_workload") is None
    assert bench.traffic_for("no_such_kernel", "256blk_8192warp_200M") is None
