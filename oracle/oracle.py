"""ctypes wrapper of the GWCP reference oracle (gwcp_oracle.cpp).

TEST INFRASTRUCTURE ONLY. The oracle is the plain CPU statement of the paper's
analysis (Algorithms 1 and 2 of "Predictive Data Race Detection for GPUs") that the
CUDA path is checked against. Only tests/, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` leg of ``bench.py`` may import this module. It imports nothing from
the CUDA package; traces are passed as raw 16-byte records.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "gwcp_oracle.cpp")
LIB = os.path.join(HERE, "liboracle_gwcp.so")

ERR_INVALID_TRACE = -1
ERR_ARGS = -2


class _Geometry(ctypes.Structure):
    _fields_ = [("num_agents", ctypes.c_uint32), ("agents_per_block", ctypes.c_uint32),
                ("granularity", ctypes.c_uint32), ("reserved", ctypes.c_uint32)]


class _Options(ctypes.Structure):
    _fields_ = [("all_pairs", ctypes.c_int32), ("release_scope_ieee", ctypes.c_int32),
                ("atomic_scope_lesser", ctypes.c_int32), ("hb_only", ctypes.c_int32),
                ("forced_barrier", ctypes.c_int32), ("version_words", ctypes.c_int32)]


def build(force: bool = False) -> str:
    """Compiles the oracle into a shared library next to its source (plain -O2, no SIMD flags)."""
    if force or not os.path.exists(LIB) or os.path.getmtime(LIB) < os.path.getmtime(SRC):
        tmp = LIB + ".tmp"
        subprocess.check_call(["g++", "-O2", "-std=c++17", "-shared", "-fPIC", "-o", tmp, SRC])
        os.replace(tmp, LIB)
    return LIB


_lib = None


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(LIB)
        vp, u64, pu64 = ctypes.c_void_p, ctypes.c_uint64, ctypes.POINTER(ctypes.c_uint64)
        L.oracle_validate.argtypes = [vp, u64, ctypes.POINTER(_Geometry), pu64]
        L.oracle_validate.restype = ctypes.c_int
        L.oracle_run.argtypes = [vp, u64, ctypes.POINTER(_Geometry), ctypes.POINTER(_Options), pu64, u64,
                                 ctypes.POINTER(vp), pu64]
        L.oracle_run.restype = ctypes.c_int
        L.oracle_num_races.argtypes = [vp]
        L.oracle_num_races.restype = u64
        L.oracle_copy_races.argtypes = [vp, pu64]
        L.oracle_counters.argtypes = [vp, pu64]
        L.oracle_versions.argtypes = [vp, pu64]
        L.oracle_clock.argtypes = [vp, u64, ctypes.POINTER(ctypes.c_uint32), ctypes.POINTER(ctypes.c_uint32)]
        L.oracle_clock.restype = ctypes.c_int
        L.oracle_free.argtypes = [vp]
        _lib = L
    return _lib


@dataclass
class OracleRun:
    races: np.ndarray                      # (k, 2) uint64: (earlier, later), sorted by (later, earlier)
    counters: dict
    clocks_c: dict = field(default_factory=dict)  # event index -> C clock (uint32[W])
    clocks_h: dict = field(default_factory=dict)  # event index -> H clock (uint32[W])


class InvalidTrace(Exception):
    def __init__(self, bad_index: int):
        super().__init__(f"invalid trace at event {bad_index}")
        self.bad_index = bad_index


def _raw(events) -> np.ndarray:
    a = np.ascontiguousarray(events)
    if a.dtype.itemsize != 16:
        raise ValueError("events must be 16-byte records")
    return a


def validate(events, num_agents: int, agents_per_block: int, granularity: int) -> tuple[int, int]:
    a = _raw(events)
    g = _Geometry(num_agents, agents_per_block, granularity, 0)
    bad = ctypes.c_uint64(0)
    rc = lib().oracle_validate(a.ctypes.data_as(ctypes.c_void_p), len(a), ctypes.byref(g), ctypes.byref(bad))
    return rc, int(bad.value)


def run(events, num_agents: int, agents_per_block: int, granularity: int, *, all_pairs=False,
        release_scope_ieee=False, atomic_scope_lesser=False, hb_only=False, forced_barrier=False,
        version_words=False, clock_events=None) -> OracleRun:
    a = _raw(events)
    g = _Geometry(num_agents, agents_per_block, granularity, 0)
    o = _Options(int(all_pairs), int(release_scope_ieee), int(atomic_scope_lesser), int(hb_only),
                 int(forced_barrier), int(version_words))
    ce = np.ascontiguousarray(np.asarray([] if clock_events is None else clock_events, dtype=np.uint64))
    handle = ctypes.c_void_p()
    bad = ctypes.c_uint64(0)
    L = lib()
    rc = L.oracle_run(a.ctypes.data_as(ctypes.c_void_p), len(a), ctypes.byref(g), ctypes.byref(o),
                      ce.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)), len(ce), ctypes.byref(handle),
                      ctypes.byref(bad))
    if rc == ERR_INVALID_TRACE:
        raise InvalidTrace(int(bad.value))
    if rc != 0:
        raise ValueError(f"oracle_run failed with {rc}")
    try:
        k = L.oracle_num_races(handle)
        races = np.zeros((k, 2), dtype=np.uint64)
        if k:
            L.oracle_copy_races(handle, races.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)))
        cnt = np.zeros(5, dtype=np.uint64)
        L.oracle_counters(handle, cnt.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)))
        counters = dict(joins=int(cnt[0]), epoch_test_disagree=int(cnt[1]), loop_visits=int(cnt[2]),
                        partner_tests=int(cnt[3]), invariant_violations=int(cnt[4]))
        if version_words:
            vw = np.zeros(2, dtype=np.uint64)
            L.oracle_versions(handle, vw.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)))
            counters.update(versions=int(vw[0]), version_words=int(vw[1]))
        out = OracleRun(races, counters)
        c = np.zeros(num_agents, dtype=np.uint32)
        h = np.zeros(num_agents, dtype=np.uint32)
        for kk, ev in enumerate(ce.tolist()):
            if L.oracle_clock(handle, kk, c.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32)),
                              h.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32))) == 0:
                out.clocks_c[int(ev)] = c.copy()
                out.clocks_h[int(ev)] = h.copy()
        return out
    finally:
        L.oracle_free(handle)


def race_set(r: OracleRun) -> set:
    return {(int(a), int(b)) for a, b in r.races}
