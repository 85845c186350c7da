"""Thin ctypes binding of libgwcp (include/gwcp.h): argument marshalling only.

Every step of the analysis runs in the CUDA library; this module converts arguments
and return codes. It fails loudly when the library has not been built: there is no
CPU path. PyTorch is used only for device memory and CUDA streams (optional).
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "lib", "libgwcp.so")

GWCP_OK = 0
ERRORS = {-1: "INVALID_TRACE", -2: "OOM", -3: "CUDA", -4: "CAPACITY", -5: "TIMEOUT", -6: "STATE", -7: "ARGS",
          -8: "UNSUPPORTED"}
ERR_INVALID_TRACE, ERR_OOM, ERR_CUDA, ERR_CAPACITY, ERR_TIMEOUT, ERR_STATE, ERR_ARGS, ERR_UNSUPPORTED = range(-1, -9, -1)
EXPORTS = ("gwcp_create", "gwcp_load_trace", "gwcp_compute_order", "gwcp_report_races", "gwcp_debug_clock",
           "gwcp_first_bad_index", "gwcp_profile_get", "gwcp_counters", "gwcp_launch_count", "gwcp_destroy",
           "gwcp_strerror", "gwcp_analyze_noalloc")


class GwcpError(RuntimeError):
    def __init__(self, code: int, what: str, bad_index: int | None = None):
        super().__init__(f"{what}: {ERRORS.get(code, code)}" + (f" at event {bad_index}" if bad_index is not None else ""))
        self.code = code
        self.bad_index = bad_index


class Geometry(ctypes.Structure):
    _fields_ = [("num_agents", ctypes.c_uint32), ("agents_per_block", ctypes.c_uint32),
                ("granularity", ctypes.c_uint32), ("reserved", ctypes.c_uint32)]


class Options(ctypes.Structure):
    _fields_ = [("race_capacity", ctypes.c_uint64), ("profile", ctypes.c_uint32),
                ("reserved", ctypes.c_uint32 * 5)]


class Race(ctypes.Structure):
    _fields_ = [("earlier", ctypes.c_uint64), ("later", ctypes.c_uint64)]


_lib = None


def load_library():
    """Loads libgwcp.so; raises if it is missing (build it with __graft_entry__.build())."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"libgwcp.so is not built ({LIB_PATH}); run __graft_entry__.build()")
    L = ctypes.CDLL(LIB_PATH)
    vp, u64, i32 = ctypes.c_void_p, ctypes.c_uint64, ctypes.c_int
    L.gwcp_create.argtypes = [ctypes.POINTER(vp), i32, ctypes.POINTER(Options)]
    L.gwcp_load_trace.argtypes = [vp, vp, u64, ctypes.POINTER(Geometry), i32, vp]
    L.gwcp_compute_order.argtypes = [vp, vp]
    L.gwcp_report_races.argtypes = [vp, vp, u64, ctypes.POINTER(u64), vp]
    L.gwcp_debug_clock.argtypes = [vp, u64, i32, ctypes.POINTER(ctypes.c_uint32)]
    L.gwcp_first_bad_index.argtypes = [vp]
    L.gwcp_first_bad_index.restype = u64
    L.gwcp_profile_get.argtypes = [vp, i32, ctypes.POINTER(ctypes.c_char_p), ctypes.POINTER(ctypes.c_float),
                                   ctypes.POINTER(ctypes.c_double)]
    L.gwcp_counters.argtypes = [vp, ctypes.POINTER(u64)]
    L.gwcp_analyze_noalloc.argtypes = [vp, u64, ctypes.POINTER(Geometry), vp, u64, ctypes.POINTER(u64),
                                       ctypes.POINTER(u64), vp]
    L.gwcp_analyze_noalloc.restype = i32
    L.gwcp_launch_count.argtypes = []
    L.gwcp_launch_count.restype = u64
    L.gwcp_destroy.argtypes = [vp]
    L.gwcp_destroy.restype = None
    L.gwcp_strerror.argtypes = [i32]
    L.gwcp_strerror.restype = ctypes.c_char_p
    for name in ("gwcp_create", "gwcp_load_trace", "gwcp_compute_order", "gwcp_report_races", "gwcp_debug_clock",
                 "gwcp_profile_get", "gwcp_counters"):
        getattr(L, name).restype = i32
    _lib = L
    return L


def launch_count() -> int:
    """Kernels launched by libgwcp in this process so far."""
    return int(load_library().gwcp_launch_count())


def strerror(code: int) -> str:
    return load_library().gwcp_strerror(code).decode()


def _stream_ptr(stream) -> int | None:
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return int(stream.cuda_stream)  # torch.cuda.Stream


class Context:
    """One analysis context on one CUDA device (gwcp_ctx)."""

    def __init__(self, device: int = 0, race_capacity: int = 0, profile: bool = False):
        L = load_library()
        opt = Options(race_capacity, int(profile))
        h = ctypes.c_void_p()
        rc = L.gwcp_create(ctypes.byref(h), device, ctypes.byref(opt))
        if rc:
            raise GwcpError(rc, "gwcp_create")
        self._h = h
        self._L = L
        self._keep = None

    def close(self):
        if getattr(self, "_h", None):
            self._L.gwcp_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def load_trace(self, events, num_agents: int, agents_per_block: int, granularity: int, stream=None,
                   n: int | None = None):
        """events: numpy array of 16-byte records (host), or a torch CUDA tensor / raw device
        pointer (int, with n) holding them (device, read in place)."""
        geo = Geometry(num_agents, agents_per_block, granularity, 0)
        if isinstance(events, np.ndarray):
            a = np.ascontiguousarray(events)
            if a.dtype.itemsize != 16:
                raise ValueError("events must be 16-byte records")
            self._keep = a
            ptr, count, dev = a.ctypes.data, len(a), 0
        elif isinstance(events, int):
            ptr, count, dev = events, int(n), 1
        else:  # torch tensor on the GPU (uint8 of 16 * n bytes, or any dtype of that size)
            if not events.is_cuda:
                raise ValueError("tensor must be on the GPU")
            self._keep = events
            ptr, count, dev = events.data_ptr(), events.numel() * events.element_size() // 16, 1
        rc = self._L.gwcp_load_trace(self._h, ctypes.c_void_p(ptr), count, ctypes.byref(geo), dev,
                                     _stream_ptr(stream))
        if rc:
            raise GwcpError(rc, "gwcp_load_trace")

    def compute_order(self, stream=None):
        rc = self._L.gwcp_compute_order(self._h, _stream_ptr(stream))
        if rc == ERR_INVALID_TRACE:
            raise GwcpError(rc, "gwcp_compute_order", self.first_bad_index())
        if rc:
            raise GwcpError(rc, "gwcp_compute_order")

    def report_races(self, stream=None, cap: int | None = None) -> np.ndarray:
        """Returns races as a (k, 2) uint64 array of (earlier, later), sorted by (later, earlier)."""
        n = ctypes.c_uint64(0)
        if cap is None:
            rc = self._L.gwcp_report_races(self._h, None, 0, ctypes.byref(n), _stream_ptr(stream))
            if rc not in (GWCP_OK, ERR_CAPACITY) or (rc == ERR_CAPACITY and n.value == 0):
                raise GwcpError(rc, "gwcp_report_races")
            cap = n.value
        out = np.zeros((max(cap, 1), 2), dtype=np.uint64)
        rc = self._L.gwcp_report_races(self._h, out.ctypes.data_as(ctypes.c_void_p), cap, ctypes.byref(n),
                                       _stream_ptr(stream))
        if rc:
            raise GwcpError(rc, "gwcp_report_races")
        return out[: n.value]

    def race_count(self, stream=None) -> int:
        n = ctypes.c_uint64(0)
        rc = self._L.gwcp_report_races(self._h, None, 0, ctypes.byref(n), _stream_ptr(stream))
        if rc not in (GWCP_OK, ERR_CAPACITY):
            raise GwcpError(rc, "gwcp_report_races")
        return int(n.value)

    def debug_clock(self, event_idx: int, which: int, num_agents: int) -> np.ndarray:
        out = np.zeros(num_agents, dtype=np.uint32)
        rc = self._L.gwcp_debug_clock(self._h, event_idx, which, out.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32)))
        if rc:
            raise GwcpError(rc, "gwcp_debug_clock")
        return out

    def first_bad_index(self) -> int:
        return int(self._L.gwcp_first_bad_index(self._h))

    def profile(self) -> list[tuple[str, float, float]]:
        out, i = [], 0
        name, ms, by = ctypes.c_char_p(), ctypes.c_float(), ctypes.c_double()
        while self._L.gwcp_profile_get(self._h, i, ctypes.byref(name), ctypes.byref(ms), ctypes.byref(by)) == 0:
            out.append((name.value.decode(), float(ms.value), float(by.value)))
            i += 1
        return out

    def counters(self) -> dict:
        a = (ctypes.c_uint64 * 8)()
        self._L.gwcp_counters(self._h, a)
        keys = ("accesses", "sync_entries", "critical_sections", "in_section_accesses", "clock_versions",
                "partner_tests", "loop_visits", "joins")
        return dict(zip(keys, [int(v) for v in a]))


def analyze_noalloc(ev_dev_ptr: int, n: int, num_agents: int, agents_per_block: int, granularity: int,
                    races_dev_ptr: int, races_cap: int, stream=None) -> tuple[int, int, int]:
    """gwcp_analyze_noalloc on device pointers (e.g. torch tensors' data_ptr()); returns
    (return code, total races, first bad index). Allocates nothing on the device."""
    L = load_library()
    geo = Geometry(num_agents, agents_per_block, granularity, 0)
    nr = ctypes.c_uint64(0)
    bad = ctypes.c_uint64(0)
    rc = L.gwcp_analyze_noalloc(ctypes.c_void_p(ev_dev_ptr), n, ctypes.byref(geo), ctypes.c_void_p(races_dev_ptr),
                                races_cap, ctypes.byref(nr), ctypes.byref(bad), _stream_ptr(stream))
    return int(rc), int(nr.value), int(bad.value)


def analyze(events, num_agents, agents_per_block, granularity, device: int = 0, **kw) -> np.ndarray:
    """One-shot: load a host trace, compute, return the sorted race pairs."""
    with Context(device, **kw) as c:
        c.load_trace(events, num_agents, agents_per_block, granularity)
        c.compute_order()
        return c.report_races()
