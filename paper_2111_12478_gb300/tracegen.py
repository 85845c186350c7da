"""Seeded synthetic trace generators (inputs only).

This module builds traces; it holds none of the analysis. It serves both the CUDA
path and the oracle: hand-written traces (``TraceBuilder``), tiny random traces drawn
from named families (``random_small``) and the large workload traces produced by the
C++ generator in ``csrc/tracegen.cpp`` (``generate``).

Trace format: one 16-byte record per event, in trace order::

    agent u32 | op u8 | scope u8 | space u8 | flags u8 | addr u64

op: 0 READ, 1 WRITE, 2 ATOMIC, 3 ACQ, 4 REL, 5 BARRIER, 6 FENCE.
scope: 0 CTA (block), 1 DEVICE, 2 WARP (barriers only).
space: 0 GLOBAL, 1 SHARED (accesses only).
addr: byte address (accesses), lock id (ACQ/REL), block id (CTA barrier) or lane mask
(WARP barrier). flags bit 0 marks an event the generator planted to break its
address's synchronisation discipline.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

EVENT_DTYPE = np.dtype([("agent", "<u4"), ("op", "u1"), ("scope", "u1"), ("space", "u1"),
                        ("flags", "u1"), ("addr", "<u8")])
assert EVENT_DTYPE.itemsize == 16

READ, WRITE, ATOMIC, ACQ, REL, BARRIER, FENCE = range(7)
CTA, DEVICE, WARP = 0, 1, 2
GLOBAL, SHARED = 0, 1
THREAD, WARP_GRAN = 0, 1
FLAG_PLANTED = 1


@dataclass
class Geometry:
    num_agents: int
    agents_per_block: int
    granularity: int = THREAD

    def astuple(self):
        return (self.num_agents, self.agents_per_block, self.granularity)


class TraceBuilder:
    """Hand-built traces: one method per event kind, appended in trace order."""

    def __init__(self):
        self.rows = []

    def _add(self, agent, op, scope=0, space=0, addr=0, flags=0):
        self.rows.append((agent, op, scope, space, flags, addr))
        return len(self.rows) - 1

    def rd(self, agent, x, shared=False):
        return self._add(agent, READ, space=int(shared), addr=x)

    def wr(self, agent, x, shared=False, planted=False):
        return self._add(agent, WRITE, space=int(shared), addr=x, flags=int(planted))

    def atomic(self, agent, x, scope=DEVICE, shared=False):
        return self._add(agent, ATOMIC, scope=scope, space=int(shared), addr=x)

    def acq(self, agent, lock, scope=DEVICE):
        return self._add(agent, ACQ, scope=scope, addr=lock)

    def rel(self, agent, lock, scope=DEVICE):
        return self._add(agent, REL, scope=scope, addr=lock)

    def barrier(self, block, agent=None, apb=None):
        a = agent if agent is not None else (block * apb if apb else 0)
        return self._add(a, BARRIER, scope=CTA, addr=block)

    def syncwarp(self, agent, mask=0xFFFFFFFF):
        return self._add(agent, BARRIER, scope=WARP, addr=mask)

    def fence(self, agent, scope=DEVICE):
        return self._add(agent, FENCE, scope=scope)

    def build(self) -> np.ndarray:
        out = np.zeros(len(self.rows), dtype=EVENT_DTYPE)
        for i, (a, op, sc, sp, fl, ad) in enumerate(self.rows):
            out[i] = (a, op, sc, sp, fl, ad)
        return out


# ---------------------------------------------------------------------------------
# Tiny random traces for closure checks and parity cases.
#
# families:
#   "nosync"       accesses and fences only
#   "barriers"     accesses, atomics and barriers, no locks
#   "dev_locks"    device-scoped locks only, no barriers, no nesting
#   "uniform"      every lock is used either only at device scope or only at block
#                  scope by one home block, so any two critical sections on one lock
#                  overlap in scope; no barriers; nesting <= 2
#   "uniform_bar"  "uniform" plus barriers outside critical sections
#   "mixed"        any lock at any scope from any block, barriers, nesting <= 2
# ---------------------------------------------------------------------------------

FAMILIES = ("nosync", "barriers", "dev_locks", "uniform", "uniform_bar", "mixed")


def random_small(seed: int, family: str, n_events: int = 48, num_agents: int = 4, agents_per_block: int = 2,
                 granularity: int = THREAD, n_locks: int = 2, n_keys: int = 3, shared_frac: float = 0.15,
                 atomic_frac: float = 0.15, close_all: bool = False):
    """Returns (events, Geometry) for a random well-formed trace of the given family."""
    if family not in FAMILIES:
        raise ValueError(family)
    rng = np.random.default_rng(seed)
    W, apb = num_agents, agents_per_block
    B = W // apb
    b = TraceBuilder()
    held = [[] for _ in range(W)]           # per agent: list of (lock, scope)
    open_cs = {}                            # lock -> list of (agent, scope)
    lock_mode = {}
    for l in range(n_locks):
        if family == "dev_locks":
            lock_mode[l] = ("dev", None)
        elif family in ("uniform", "uniform_bar"):
            lock_mode[l] = ("dev", None) if rng.random() < 0.5 else ("blk", int(rng.integers(B)))
        else:
            lock_mode[l] = ("any", None)
    locks_on = family in ("dev_locks", "uniform", "uniform_bar", "mixed")
    barriers_on = family in ("barriers", "uniform_bar", "mixed")
    max_nest = 1 if family == "dev_locks" else 2

    def blk(t):
        return t // apb

    def sid(t, scope):
        return 0 if scope == DEVICE else blk(t) + 1

    def can_acquire(t, l, scope):
        s = sid(t, scope)
        for (a, sc) in open_cs.get(l, []):
            s2 = sid(a, sc)
            if s == 0 or s2 == 0 or s == s2:
                return False
        return True

    def access(t):
        r = rng.random()
        x = int(rng.integers(n_keys)) * 4 + 0x1000
        shared = rng.random() < shared_frac
        if r < atomic_frac:
            sc = DEVICE if rng.random() < 0.5 else CTA
            b.atomic(t, x, scope=sc, shared=shared)
        elif r < atomic_frac + (1 - atomic_frac) * 0.45:
            b.wr(t, x, shared=shared)
        else:
            b.rd(t, x, shared=shared)

    while len(b.rows) < n_events:
        t = int(rng.integers(W))
        r = rng.random()
        if held[t]:
            if r < 0.6:
                access(t)
            elif r < 0.92 or len(held[t]) >= max_nest or not locks_on:
                l, sc = held[t].pop()
                b.rel(t, l, sc)
                open_cs[l].remove((t, sc))
            else:
                _try_acquire(b, rng, t, held, open_cs, lock_mode, n_locks, blk, can_acquire, access)
            continue
        if r < 0.62:
            access(t)
        elif r < 0.80 and locks_on:
            _try_acquire(b, rng, t, held, open_cs, lock_mode, n_locks, blk, can_acquire, access)
        elif r < 0.90 and barriers_on:
            if granularity == THREAD and apb > 1 and rng.random() < 0.3:
                # warp-scope barrier over some lanes of t's hardware warp (thread granularity)
                base = blk(t) * apb + ((t - blk(t) * apb) // 32) * 32
                lanes = [a - base for a in range(base, min(base + 32, (blk(t) + 1) * apb))]
                pick = [ln for ln in lanes if rng.random() < 0.7] or [t - base]
                members = [base + ln for ln in pick]
                if any(held[a] for a in members):
                    access(t)
                    continue
                mask = 0
                for ln in pick:
                    mask |= 1 << ln
                b.syncwarp(t, mask)
            else:
                bb = blk(t)
                members = range(bb * apb, (bb + 1) * apb)
                if family != "mixed" and any(held[a] for a in members):
                    access(t)
                    continue
                b.barrier(bb, agent=t)
        else:
            b.fence(t, scope=DEVICE if rng.random() < 0.5 else CTA)
    if close_all:
        for t in range(W):
            while held[t]:
                l, sc = held[t].pop()
                b.rel(t, l, sc)
    return b.build(), Geometry(W, apb, granularity)


def _try_acquire(b, rng, t, held, open_cs, lock_mode, n_locks, blk, can_acquire, access):
    choices = []
    for l in range(n_locks):
        if any(h[0] == l for h in held[t]):
            continue
        mode, home = lock_mode[l]
        if mode == "dev":
            scs = [DEVICE]
        elif mode == "blk":
            scs = [CTA] if blk(t) == home else []
        else:
            scs = [DEVICE, CTA]
        for sc in scs:
            if can_acquire(t, l, sc):
                choices.append((l, sc))
    if not choices:
        access(t)
        return
    l, sc = choices[int(rng.integers(len(choices)))]
    b.acq(t, l, sc)
    held[t].append((l, sc))
    open_cs.setdefault(l, []).append((t, sc))


# ---------------------------------------------------------------------------------
# Large workload traces (C++ generator)
# ---------------------------------------------------------------------------------

_HERE = os.path.dirname(os.path.abspath(__file__))
_GEN_SRC = os.path.join(_HERE, "csrc", "tracegen.cpp")
_GEN_LIB = os.path.join(_HERE, "lib", "libgwcp_tracegen.so")


def build_generator(force: bool = False) -> str:
    os.makedirs(os.path.dirname(_GEN_LIB), exist_ok=True)
    if force or not os.path.exists(_GEN_LIB) or os.path.getmtime(_GEN_LIB) < os.path.getmtime(_GEN_SRC):
        tmp = _GEN_LIB + ".tmp"
        # no fused multiply-add contraction (gcc's default on aarch64): the same seed gives
        # the same trace on x86-64 and aarch64 hosts
        subprocess.check_call(["g++", "-O2", "-std=c++17", "-ffp-contract=off", "-shared", "-fPIC", "-o", tmp,
                               _GEN_SRC])
        os.replace(tmp, _GEN_LIB)
    return _GEN_LIB


class _GenParams(ctypes.Structure):
    _fields_ = [
        ("seed", ctypes.c_uint64),
        ("n_events", ctypes.c_uint64),
        ("num_blocks", ctypes.c_uint32),
        ("agents_per_block", ctypes.c_uint32),
        ("granularity", ctypes.c_uint32),
        ("n_ranks", ctypes.c_uint32),
        ("zipf_s", ctypes.c_double),
        ("n_locks", ctypes.c_uint32),
        ("dev_lock_frac", ctypes.c_double),
        ("p_read", ctypes.c_double),
        ("p_write", ctypes.c_double),
        ("p_atomic", ctypes.c_double),
        ("p_acqrel", ctypes.c_double),
        ("p_fence", ctypes.c_double),
        ("p_barrier", ctypes.c_double),
        ("atomic_dev_frac", ctypes.c_double),
        ("plant_frac", ctypes.c_double),
        ("n_plant_exact", ctypes.c_uint32),
        ("cs_len_mean", ctypes.c_double),
        ("nest_prob", ctypes.c_double),
        ("shared_frac", ctypes.c_double),
        ("p_syncwarp", ctypes.c_double),
        ("plant_min_rank", ctypes.c_uint32),
    ]


# The workloads the benchmark and the parity tests use, by name. In the 8192-warp trace
# the planted accesses avoid the 65536 hottest address ranks: a write planted on a read-
# mostly address read by all 8192 warps would race with every later unordered read. Sizes follow the
# trace shapes the analysis targets: a 64-thread single-block trace at thread
# granularity, a 64-warp 8-block trace, a 8192-warp 256-block trace.
WORKLOADS = {
    "tiny_1blk_64thr_10k": dict(n_events=10_000, num_blocks=1, agents_per_block=64, granularity=THREAD,
                                n_ranks=16, zipf_s=0.0, n_locks=2, dev_lock_frac=0.5, p_read=0.60,
                                p_write=0.30, p_atomic=0.05, p_acqrel=0.03, p_fence=0.0, p_barrier=0.002,
                                atomic_dev_frac=0.5, plant_frac=0.0, n_plant_exact=4, cs_len_mean=3.0,
                                nest_prob=0.1, shared_frac=0.2, p_syncwarp=0.3),
    "8blk_64warp_10M": dict(n_events=10_000_000, num_blocks=8, agents_per_block=8, granularity=WARP_GRAN,
                            n_ranks=1_000_000, zipf_s=1.1, n_locks=1024, dev_lock_frac=0.5, p_read=0.62,
                            p_write=0.35, p_atomic=0.01, p_acqrel=0.01, p_fence=0.005, p_barrier=0.005,
                            atomic_dev_frac=0.5, plant_frac=0.001, n_plant_exact=0, cs_len_mean=3.0,
                            nest_prob=0.1, shared_frac=0.1, p_syncwarp=0.0),
    "256blk_8192warp_200M": dict(n_events=200_000_000, num_blocks=256, agents_per_block=32,
                                 granularity=WARP_GRAN, n_ranks=64_000_000, zipf_s=1.05, n_locks=4096,
                                 dev_lock_frac=0.3, p_read=0.66, p_write=0.32, p_atomic=0.003,
                                 p_acqrel=0.004, p_fence=0.002, p_barrier=0.001, atomic_dev_frac=0.3,
                                 plant_frac=0.001, n_plant_exact=0, cs_len_mean=3.0, nest_prob=0.1,
                                 shared_frac=0.1, p_syncwarp=0.0, plant_min_rank=65536),
}


def generate(seed: int, n_events: int | None = None, workload: str | None = None, **overrides):
    """Runs the C++ generator. Returns (events, Geometry, planted_indices)."""
    params = dict(WORKLOADS[workload]) if workload else {}
    params.update(overrides)
    if n_events is not None:
        params["n_events"] = n_events
    L = ctypes.CDLL(build_generator())
    L.gwcp_tracegen_run.argtypes = [ctypes.POINTER(_GenParams), ctypes.c_void_p, ctypes.POINTER(ctypes.c_uint64)]
    L.gwcp_tracegen_run.restype = ctypes.c_int
    p = _GenParams()
    p.seed = seed
    for k, v in params.items():
        setattr(p, k, v)
    n = int(p.n_events)
    out = np.zeros(n, dtype=EVENT_DTYPE)
    written = ctypes.c_uint64(0)
    rc = L.gwcp_tracegen_run(ctypes.byref(p), out.ctypes.data_as(ctypes.c_void_p), ctypes.byref(written))
    if rc != 0:
        raise RuntimeError(f"trace generator failed ({rc})")
    out = out[: written.value]
    geo = Geometry(int(p.num_blocks) * int(p.agents_per_block), int(p.agents_per_block), int(p.granularity))
    planted = np.nonzero(out["flags"] & FLAG_PLANTED)[0]
    return out, geo, planted


# ---- many independent traces: the batched and the served workloads ----------------------

BATCH_WIDTHS = (64, 128, 256, 512, 1024, 2048, 4096)


def blocks_for_width(W: int) -> tuple[int, int]:
    """(num_blocks, agents_per_block) for a W-warp trace: 8 warps (256 threads) per block up to
    512 warps, then blocks of W/64 warps (at most 32, the widest block the tile-table clocks
    take), so that no trace has more than 128 blocks."""
    apb = min(32, max(8, W // 64))
    return W // apb, apb


def many_specs(seed: int, n_traces: int, n_min: int, n_max: int, widths=BATCH_WIDTHS) -> list[dict]:
    """Per-trace generator parameters: lengths log-uniform over [n_min, n_max], widths drawn
    uniformly from `widths` (warp granularity), the op/scope mix of the 64-warp 10M-event
    workload, address ranks Zipf(1.1) over max(1000, n/10) ranks, a distinct seed per trace."""
    rng = np.random.default_rng(seed)
    lens = np.exp(rng.uniform(np.log(n_min), np.log(n_max), size=n_traces)).astype(np.int64)
    ws = rng.choice(np.asarray(widths), size=n_traces)
    base = WORKLOADS["8blk_64warp_10M"]
    specs = []
    for i in range(n_traces):
        nb, apb = blocks_for_width(int(ws[i]))
        p = dict(base)
        p.update(n_events=int(lens[i]), num_blocks=nb, agents_per_block=apb, n_ranks=max(1000, int(lens[i]) // 10),
                 seed=int(seed) * 100_003 + i)
        specs.append(p)
    return specs


def generate_many(specs: list[dict], threads: int = 8) -> list[tuple[np.ndarray, Geometry]]:
    """Runs the C++ generator for every spec (threads in parallel); returns (events, Geometry)."""
    from concurrent.futures import ThreadPoolExecutor

    def one(p):
        q = dict(p)
        s = q.pop("seed")
        ev, geo, _ = generate(s, **q)
        return ev, geo

    with ThreadPoolExecutor(max(1, threads)) as ex:
        return list(ex.map(one, specs))


# The batched workload: 512 independent traces, 10k-5M events each, 64-4096 warps.
BATCH_WORKLOAD = dict(n_traces=512, n_min=10_000, n_max=5_000_000)
# The served workload: traces of 10k-20M events, 64-4096 warps, arriving as a Poisson
# process at 200 traces/s.
SERVE_WORKLOAD = dict(rate=200.0, n_min=10_000, n_max=20_000_000)


def serve_base_specs(seed: int, n_max: int, widths=BATCH_WIDTHS) -> list[dict]:
    """One n_max-event trace per width class; a served request of n events is the first n
    events of its class's trace (a prefix of a well-formed trace is well-formed)."""
    base = WORKLOADS["8blk_64warp_10M"]
    specs = []
    for j, W in enumerate(widths):
        nb, apb = blocks_for_width(int(W))
        p = dict(base)
        p.update(n_events=int(n_max), num_blocks=nb, agents_per_block=apb, n_ranks=max(1000, int(n_max) // 10),
                 seed=int(seed) * 7_919 + j)
        specs.append(p)
    return specs


def serve_requests(seed: int, n_requests: int, rate: float, n_min: int, n_max: int, n_widths: int = len(BATCH_WIDTHS)):
    """Arrival times of a Poisson process of `rate` requests/s (seconds from the start), each
    request's width class (uniform) and length (log-uniform over [n_min, n_max])."""
    rng = np.random.default_rng(seed)
    arrivals = np.cumsum(rng.exponential(1.0 / rate, size=n_requests))
    widths = rng.integers(0, n_widths, size=n_requests)
    lens = np.exp(rng.uniform(np.log(n_min), np.log(n_max), size=n_requests)).astype(np.int64)
    return arrivals, widths, lens
