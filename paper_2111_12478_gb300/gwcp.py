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
           "gwcp_first_bad_index", "gwcp_profile_get", "gwcp_profile_start", "gwcp_counters", "gwcp_launch_count", "gwcp_destroy",
           "gwcp_strerror", "gwcp_analyze_noalloc", "gwcp_pool_create", "gwcp_pool_submit", "gwcp_pool_wait",
           "gwcp_pool_run_batch", "gwcp_pool_set_active_lanes", "gwcp_pool_autotune", "gwcp_pool_now",
           "gwcp_pool_device_bytes", "gwcp_pool_destroy", "gwcp_set_ranker", "gwcp_location_features",
           "gwcp_rank_scores", "gwcp_rank_grad", "gwcp_rank_train", "gwcp_check_timeline", "gwcp_set_clock_mode",
           "gwcp_pool_clock_modes", "gwcp_set_check_mode", "gwcp_debug_wait_timeout", "gwcp_pool_settings",
           "gwcp_clock_bytes", "gwcp_debug_alloc_limit", "gwcp_counters_ex")
CLOCKS_AUTO, CLOCKS_DENSE, CLOCKS_TILES, CLOCKS_COMPRESSED = 0, 1, 2, 3
CHECK_AUTO, CHECK_CHUNKED, CHECK_SPARSE = 0, 1, 2


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
                ("blocking_sync", ctypes.c_uint32), ("timeline", ctypes.c_uint32), ("hb_only", ctypes.c_uint32),
                ("pack_walkers", ctypes.c_uint32), ("forced_barrier", ctypes.c_uint32)]


class TrainOptions(ctypes.Structure):
    _fields_ = [("epochs", ctypes.c_uint32), ("batch", ctypes.c_uint32), ("lr", ctypes.c_float),
                ("pos_weight", ctypes.c_float), ("reserved", ctypes.c_uint32 * 4)]


RANK_PARAMS, RANK_FEATURES = 5313, 16


class TraceDesc(ctypes.Structure):
    _fields_ = [("ev", ctypes.c_void_p), ("n", ctypes.c_uint64), ("geo", Geometry), ("ev_is_device", ctypes.c_int32),
                ("reserved", ctypes.c_uint32)]


class PoolOptions(ctypes.Structure):
    _fields_ = [("lanes", ctypes.c_uint32), ("pack_walkers", ctypes.c_uint32), ("mem_budget", ctypes.c_uint64),
                ("race_capacity", ctypes.c_uint64), ("compress_versions", ctypes.c_uint32),
                ("reserved", ctypes.c_uint32 * 3)]


class RequestInfo(ctypes.Structure):
    _fields_ = [("rc", ctypes.c_int32), ("lane", ctypes.c_uint32), ("n_races", ctypes.c_uint64),
                ("first_bad_index", ctypes.c_uint64), ("t_submit", ctypes.c_double), ("t_admit", ctypes.c_double),
                ("t_done", ctypes.c_double), ("t_first_race", ctypes.c_double)]


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
    L.gwcp_profile_start.argtypes = [vp, i32, ctypes.POINTER(ctypes.c_float)]
    L.gwcp_counters.argtypes = [vp, ctypes.POINTER(u64)]
    L.gwcp_counters_ex.argtypes = [vp, ctypes.POINTER(u64), ctypes.c_uint32]
    L.gwcp_clock_bytes.argtypes = [vp, ctypes.POINTER(u64)]
    L.gwcp_debug_alloc_limit.argtypes = [vp, u64]
    L.gwcp_debug_alloc_limit.restype = i32
    L.gwcp_clock_bytes.restype = i32
    L.gwcp_analyze_noalloc.argtypes = [vp, u64, ctypes.POINTER(Geometry), vp, u64, ctypes.POINTER(u64),
                                       ctypes.POINTER(u64), vp]
    L.gwcp_analyze_noalloc.restype = i32
    L.gwcp_pool_create.argtypes = [ctypes.POINTER(vp), i32, ctypes.POINTER(PoolOptions)]
    L.gwcp_pool_submit.argtypes = [vp, ctypes.POINTER(TraceDesc), vp, u64, ctypes.POINTER(u64)]
    L.gwcp_pool_wait.argtypes = [vp, u64, i32, ctypes.POINTER(RequestInfo)]
    L.gwcp_pool_run_batch.argtypes = [vp, ctypes.POINTER(TraceDesc), ctypes.c_uint32, ctypes.POINTER(vp),
                                      ctypes.POINTER(u64), ctypes.POINTER(u64), ctypes.POINTER(ctypes.c_int32)]
    L.gwcp_pool_set_active_lanes.argtypes = [vp, ctypes.c_uint32]
    L.gwcp_pool_autotune.argtypes = [vp, ctypes.POINTER(TraceDesc), ctypes.c_uint32, ctypes.POINTER(ctypes.c_uint32),
                                     ctypes.POINTER(ctypes.c_double)]
    L.gwcp_pool_now.argtypes = [vp]
    L.gwcp_pool_now.restype = ctypes.c_double
    L.gwcp_pool_device_bytes.argtypes = [vp]
    L.gwcp_pool_device_bytes.restype = u64
    L.gwcp_pool_destroy.argtypes = [vp]
    L.gwcp_pool_destroy.restype = None
    for name in ("gwcp_pool_create", "gwcp_pool_submit", "gwcp_pool_wait", "gwcp_pool_run_batch",
                 "gwcp_pool_set_active_lanes", "gwcp_pool_autotune"):
        getattr(L, name).restype = i32
    fp = ctypes.POINTER(ctypes.c_float)
    L.gwcp_set_ranker.argtypes = [vp, vp]
    L.gwcp_pool_settings.argtypes = [vp, ctypes.POINTER(ctypes.c_uint32), ctypes.POINTER(ctypes.c_uint32)]
    L.gwcp_pool_settings.restype = i32
    L.gwcp_pool_clock_modes.argtypes = [vp, ctypes.POINTER(ctypes.c_uint32)]
    L.gwcp_pool_clock_modes.restype = i32
    L.gwcp_debug_wait_timeout.argtypes = [i32, ctypes.c_uint32, ctypes.POINTER(ctypes.c_int)]
    L.gwcp_debug_wait_timeout.restype = i32
    L.gwcp_set_check_mode.argtypes = [vp, ctypes.c_uint32]
    L.gwcp_set_check_mode.restype = i32
    L.gwcp_set_clock_mode.argtypes = [vp, ctypes.c_uint32]
    L.gwcp_set_clock_mode.restype = i32
    L.gwcp_location_features.argtypes = [vp, vp, vp, u64, ctypes.POINTER(u64), vp]
    L.gwcp_rank_scores.argtypes = [vp, vp, u64, vp, vp]
    L.gwcp_rank_grad.argtypes = [vp, vp, vp, u64, ctypes.c_float, vp, vp, vp]
    L.gwcp_rank_train.argtypes = [vp, vp, vp, u64, ctypes.POINTER(TrainOptions), fp, vp]
    L.gwcp_check_timeline.argtypes = [vp, ctypes.POINTER(u64), vp, vp, u64, ctypes.POINTER(u64)]
    for name in ("gwcp_set_ranker", "gwcp_location_features", "gwcp_rank_scores", "gwcp_rank_grad",
                 "gwcp_rank_train", "gwcp_check_timeline"):
        getattr(L, name).restype = i32
    L.gwcp_launch_count.argtypes = []
    L.gwcp_launch_count.restype = u64
    L.gwcp_destroy.argtypes = [vp]
    L.gwcp_destroy.restype = None
    L.gwcp_strerror.argtypes = [i32]
    L.gwcp_strerror.restype = ctypes.c_char_p
    for name in ("gwcp_create", "gwcp_load_trace", "gwcp_compute_order", "gwcp_report_races", "gwcp_debug_clock",
                 "gwcp_profile_get", "gwcp_profile_start", "gwcp_counters", "gwcp_counters_ex"):
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

    def __init__(self, device: int = 0, race_capacity: int = 0, profile: bool = False, timeline: bool = False,
                 hb_only: bool = False, forced_barrier: bool = False, pack_walkers: bool = False):
        L = load_library()
        opt = Options(race_capacity, int(profile), 0, int(timeline), int(hb_only), int(pack_walkers),
                      int(forced_barrier))
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

    def report_races(self, stream=None, cap: int | None = None, out: np.ndarray | None = None) -> np.ndarray:
        """Returns races as a (k, 2) uint64 array of (earlier, later), sorted by (later, earlier).
        out: a reusable (cap, 2) uint64 host array to write into (e.g. a view of pinned memory,
        which makes the device-to-host copy a single DMA); the result is a view of it."""
        n = ctypes.c_uint64(0)
        if out is not None:
            if out.dtype != np.uint64 or out.ndim != 2 or out.shape[1] != 2 or not out.flags.c_contiguous:
                raise ValueError("out must be a C-contiguous (cap, 2) uint64 array")
            rc = self._L.gwcp_report_races(self._h, out.ctypes.data_as(ctypes.c_void_p), out.shape[0],
                                           ctypes.byref(n), _stream_ptr(stream))
            if rc:
                raise GwcpError(rc, "gwcp_report_races")
            return out[: n.value]
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

    def set_clock_mode(self, mode: int):
        """CLOCKS_AUTO, CLOCKS_DENSE, CLOCKS_TILES or CLOCKS_COMPRESSED from the next load_trace on."""
        rc = self._L.gwcp_set_clock_mode(self._h, mode)
        if rc:
            raise GwcpError(rc, "gwcp_set_clock_mode")

    def set_check_mode(self, mode: int):
        """CHECK_AUTO, CHECK_CHUNKED or CHECK_SPARSE from the next compute_order on."""
        rc = self._L.gwcp_set_check_mode(self._h, mode)
        if rc:
            raise GwcpError(rc, "gwcp_set_check_mode")

    def set_ranker(self, theta):
        """Checks locations in the ranker's order from the next compute_order on (theta: 5313
        float32 parameters, or None to turn the ranker off)."""
        if theta is None:
            rc = self._L.gwcp_set_ranker(self._h, None)
        else:
            t = np.ascontiguousarray(theta, dtype=np.float32)
            if t.size != RANK_PARAMS:
                raise ValueError("theta must hold 5313 values")
            self._theta = t
            rc = self._L.gwcp_set_ranker(self._h, t.ctypes.data)
        if rc:
            raise GwcpError(rc, "gwcp_set_ranker")

    def location_features(self, stream=None):
        """Features of every accessed location of the last compute, in check order: (features
        float32 CUDA tensor [n, 16], location keys int64 CUDA tensor [n] holding the u64 keys)."""
        import torch

        n = ctypes.c_uint64(0)
        rc = self._L.gwcp_location_features(self._h, None, None, 0, ctypes.byref(n), _stream_ptr(stream))
        if rc not in (GWCP_OK, ERR_CAPACITY):
            raise GwcpError(rc, "gwcp_location_features")
        feat = torch.zeros((max(n.value, 1), RANK_FEATURES), dtype=torch.float32, device="cuda")
        keys = torch.zeros(max(n.value, 1), dtype=torch.int64, device="cuda")
        rc = self._L.gwcp_location_features(self._h, feat.data_ptr(), keys.data_ptr(), n.value, ctypes.byref(n),
                                            _stream_ptr(stream))
        if rc:
            raise GwcpError(rc, "gwcp_location_features")
        return feat[: n.value], keys[: n.value]

    def check_timeline(self):
        """(start ns, per-chunk end ns uint64 array, per-chunk race counts uint32 array), chunks
        in check order (needs timeline=True)."""
        start, n = ctypes.c_uint64(0), ctypes.c_uint64(0)
        rc = self._L.gwcp_check_timeline(self._h, ctypes.byref(start), None, None, 0, ctypes.byref(n))
        if rc not in (GWCP_OK, ERR_CAPACITY):
            raise GwcpError(rc, "gwcp_check_timeline")
        ends = np.zeros(max(n.value, 1), dtype=np.uint64)
        races = np.zeros(max(n.value, 1), dtype=np.uint32)
        rc = self._L.gwcp_check_timeline(self._h, ctypes.byref(start), ends.ctypes.data, races.ctypes.data, n.value,
                                         ctypes.byref(n))
        if rc:
            raise GwcpError(rc, "gwcp_check_timeline")
        return int(start.value), ends[: n.value], races[: n.value]

    def first_bad_index(self) -> int:
        return int(self._L.gwcp_first_bad_index(self._h))

    def profile(self) -> list[tuple[str, float, float]]:
        out, i = [], 0
        name, ms, by = ctypes.c_char_p(), ctypes.c_float(), ctypes.c_double()
        while self._L.gwcp_profile_get(self._h, i, ctypes.byref(name), ctypes.byref(ms), ctypes.byref(by)) == 0:
            out.append((name.value.decode(), float(ms.value), float(by.value)))
            i += 1
        return out

    def timeline(self) -> list[tuple[str, float, float]]:
        """(name, start ms after the first kernel, duration ms) of each profiled kernel."""
        out = []
        at = ctypes.c_float()
        for i, (name, ms, _) in enumerate(self.profile()):
            if self._L.gwcp_profile_start(self._h, i, ctypes.byref(at)) != 0:
                break
            out.append((name, float(at.value), ms))
        return out

    def counters(self) -> dict:
        a = (ctypes.c_uint64 * 10)()
        self._L.gwcp_counters_ex(self._h, a, 10)
        keys = ("accesses", "sync_entries", "critical_sections", "in_section_accesses", "clock_versions",
                "partner_tests", "loop_visits", "joins", "tiles_read", "tiles_written")
        return dict(zip(keys, [int(v) for v in a]))

    def debug_alloc_limit(self, nbytes: int):
        """Test hook: cap the context's cached device buffers at nbytes (0 = no cap)."""
        rc = self._L.gwcp_debug_alloc_limit(self._h, nbytes)
        if rc:
            raise GwcpError(rc, "gwcp_debug_alloc_limit")

    def clock_bytes(self) -> dict:
        """Bytes of the last compute's clock versions: as dense rows, as stored, as reserved."""
        a = (ctypes.c_uint64 * 3)()
        rc = self._L.gwcp_clock_bytes(self._h, a)
        if rc:
            raise GwcpError(rc, "gwcp_clock_bytes")
        return dict(dense=int(a[0]), stored=int(a[1]), reserved=int(a[2]))


def debug_wait_timeout(device: int, spin_limit: int) -> int:
    """Runs the analysis' bounded device wait on a row nothing completes; returns the kernel's
    status (ERR_TIMEOUT when the wait gave up as it must)."""
    st = ctypes.c_int(0)
    rc = load_library().gwcp_debug_wait_timeout(device, spin_limit, ctypes.byref(st))
    if rc:
        raise GwcpError(rc, "gwcp_debug_wait_timeout")
    return int(st.value)


def rank_scores(theta, feat, stream=None):
    """Scores of feature rows (CUDA tensors: theta [5313] float32, feat [n, 16] float32)."""
    import torch

    out = torch.empty(feat.shape[0], dtype=torch.float32, device=feat.device)
    rc = load_library().gwcp_rank_scores(theta.data_ptr(), feat.data_ptr(), feat.shape[0], out.data_ptr(),
                                         _stream_ptr(stream))
    if rc:
        raise GwcpError(rc, "gwcp_rank_scores")
    return out


def rank_grad(theta, feat, labels, pos_weight: float, stream=None):
    """(gradient [5313] float32 CUDA tensor, loss) of the mean weighted logistic loss."""
    import torch

    g = torch.empty(RANK_PARAMS, dtype=torch.float32, device=feat.device)
    loss = torch.empty(1, dtype=torch.float32, device=feat.device)
    rc = load_library().gwcp_rank_grad(theta.data_ptr(), feat.data_ptr(), labels.data_ptr(), feat.shape[0],
                                       float(pos_weight), g.data_ptr(), loss.data_ptr(), _stream_ptr(stream))
    if rc:
        raise GwcpError(rc, "gwcp_rank_grad")
    torch.cuda.synchronize(feat.device)
    return g, float(loss.item())


def rank_train(theta, feat, labels, epochs: int, batch: int, lr: float, pos_weight: float, stream=None):
    """Adam training of theta (CUDA tensor, in place) on feature rows and 0/1 labels (CUDA
    tensors, rows already shuffled); returns the mean batch loss of each epoch."""
    losses = np.zeros(epochs, dtype=np.float32)
    o = TrainOptions(epochs, batch, lr, pos_weight)
    rc = load_library().gwcp_rank_train(theta.data_ptr(), feat.data_ptr(), labels.data_ptr(), feat.shape[0],
                                        ctypes.byref(o), losses.ctypes.data_as(ctypes.POINTER(ctypes.c_float)),
                                        _stream_ptr(stream))
    if rc:
        raise GwcpError(rc, "gwcp_rank_train")
    return losses


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


def _trace_desc(events, geo) -> tuple[TraceDesc, object]:
    """A gwcp_trace_desc for a host numpy trace or a torch CUDA tensor; returns it with the
    object that must stay alive while the pool uses it."""
    num_agents, agents_per_block, granularity = geo
    g = Geometry(num_agents, agents_per_block, granularity, 0)
    if isinstance(events, np.ndarray):
        a = np.ascontiguousarray(events)
        if a.dtype.itemsize != 16:
            raise ValueError("events must be 16-byte records")
        return TraceDesc(a.ctypes.data, len(a), g, 0, 0), a
    if not events.is_cuda and not events.is_pinned():
        raise ValueError("tensor must be on the GPU or in pinned host memory")
    n = events.numel() * events.element_size() // 16
    return TraceDesc(events.data_ptr(), n, g, 1 if events.is_cuda else 0, 0), events


class Pool:
    """Batched and served analysis (gwcp_pool): lanes of contexts that run independent
    traces concurrently on one GPU, admitted by device memory."""

    def __init__(self, device: int = 0, lanes: int = 16, mem_budget: int = 0, race_capacity: int = 0,
                 pack_walkers: bool = True, compress_versions: bool = False):
        L = load_library()
        opt = PoolOptions(lanes, int(pack_walkers), mem_budget, race_capacity, int(compress_versions))
        h = ctypes.c_void_p()
        rc = L.gwcp_pool_create(ctypes.byref(h), device, ctypes.byref(opt))
        if rc:
            raise GwcpError(rc, "gwcp_pool_create")
        self._h, self._L = h, L
        self._live = {}  # ticket -> (descriptor, trace keep-alive, output array)

    def close(self):
        if getattr(self, "_h", None):
            self._L.gwcp_pool_destroy(self._h)
            self._h = None
            self._live.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def now(self) -> float:
        return float(self._L.gwcp_pool_now(self._h))

    def device_bytes(self) -> int:
        return int(self._L.gwcp_pool_device_bytes(self._h))

    def submit(self, events, geo, cap: int, out: np.ndarray | None = None) -> int:
        """Queues one trace (host numpy array, pinned host tensor or CUDA tensor); geo =
        (num_agents, agents_per_block, granularity). Up to `cap` races are kept, in `out`
        (a reusable C-contiguous (>= cap, 2) uint64 array) when given."""
        d, keep = _trace_desc(events, geo)
        if out is None:
            out = np.zeros((max(cap, 1), 2), dtype=np.uint64)
        elif out.dtype != np.uint64 or out.ndim != 2 or out.shape[0] < cap or not out.flags.c_contiguous:
            raise ValueError("out must be a C-contiguous (>= cap, 2) uint64 array")
        t = ctypes.c_uint64(0)
        rc = self._L.gwcp_pool_submit(self._h, ctypes.byref(d), out.ctypes.data_as(ctypes.c_void_p), cap,
                                      ctypes.byref(t))
        if rc:
            raise GwcpError(rc, "gwcp_pool_submit")
        self._live[t.value] = (d, keep, out, cap)
        return int(t.value)

    def wait(self, ticket: int, block: bool = True):
        """Returns None if not finished (block=False), else (races (k, 2) uint64 array of
        (earlier, later) truncated to the cap, RequestInfo)."""
        info = RequestInfo()
        rc = self._L.gwcp_pool_wait(self._h, ticket, int(block), ctypes.byref(info))
        if rc == 1:
            return None
        if rc:
            raise GwcpError(rc, "gwcp_pool_wait")
        _, _, out, cap = self._live.pop(ticket)
        return out[: min(info.n_races, cap)] if info.rc in (GWCP_OK, ERR_CAPACITY) else out[:0], info

    def run_batch(self, traces, caps, outs=None):
        """traces: list of (events, geo); returns a list of (races, rc, n_races). outs: optional
        reusable (>= cap, 2) uint64 arrays, one per trace, that the races are written into."""
        n = len(traces)
        descs = (TraceDesc * n)()
        keep = []
        if outs is None:
            outs = [np.zeros((max(c, 1), 2), dtype=np.uint64) for c in caps]
        for i, (ev, geo) in enumerate(traces):
            d, k = _trace_desc(ev, geo)
            descs[i] = d
            keep.append(k)
            if outs[i].shape[0] < caps[i] or outs[i].dtype != np.uint64 or not outs[i].flags.c_contiguous:
                raise ValueError("outs[i] must be a C-contiguous (>= cap, 2) uint64 array")
        optr = (ctypes.c_void_p * n)(*[o.ctypes.data for o in outs])
        cap = (ctypes.c_uint64 * n)(*caps)
        nr = (ctypes.c_uint64 * n)()
        rcs = (ctypes.c_int32 * n)()
        self._L.gwcp_pool_run_batch(self._h, descs, n, optr, cap, nr, rcs)
        return [(outs[i][: min(nr[i], caps[i])], int(rcs[i]), int(nr[i])) for i in range(n)]

    def set_active_lanes(self, k: int):
        rc = self._L.gwcp_pool_set_active_lanes(self._h, k)
        if rc:
            raise GwcpError(rc, "gwcp_pool_set_active_lanes")

    def autotune(self, traces):
        """Picks the number of active lanes that runs `traces` fastest; returns (best, {lanes: s})."""
        n = len(traces)
        descs = (TraceDesc * n)()
        keep = []
        for i, (ev, geo) in enumerate(traces):
            d, k = _trace_desc(ev, geo)
            descs[i] = d
            keep.append(k)
        best = ctypes.c_uint32(0)
        secs = (ctypes.c_double * 8)()
        rc = self._L.gwcp_pool_autotune(self._h, descs, n, ctypes.byref(best), secs)
        if rc:
            raise GwcpError(rc, "gwcp_pool_autotune")
        cand = (1, 2, 4, 8, 12, 16, 24, 32)
        return int(best.value), {c: float(secs[i]) for i, c in enumerate(cand) if secs[i] > 0}

    def settings(self) -> tuple[int, bool]:
        """(active lanes, tile walkers packed two CTAs per SM)."""
        a, pk = ctypes.c_uint32(0), ctypes.c_uint32(0)
        self._L.gwcp_pool_settings(self._h, ctypes.byref(a), ctypes.byref(pk))
        return int(a.value), bool(pk.value)

    def clock_modes(self) -> dict:
        """Chosen clock mode per width class {ceil(log2(W)): mode} (modes other than AUTO)."""
        m = (ctypes.c_uint32 * 16)()
        self._L.gwcp_pool_clock_modes(self._h, m)
        return {c: int(m[c]) for c in range(16) if m[c]}
