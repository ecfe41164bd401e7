"""FSE on overlapping tiles, GB300-native (sm_103a CUDA behind a C ABI).

This module is a thin ctypes binding of ``include/fse.h``: it marshals
arguments (torch tensors for device memory and streams, numpy arrays for host
memory) and raises on error statuses.  Every step of the method runs in the
library's CUDA kernels; there is no Python or CPU fallback, and importing the
binding fails loudly when the library has not been built.
"""
import ctypes
import os

import numpy as np

from . import build as _build

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libfse.so")

OK, EINVAL, EDEGENERATE, ENOMEM, EBUSY, ETIMEOUT, ECUDA, ENOTFOUND, ECANCELLED = 0, -1, -2, -3, -4, -5, -6, -7, -8
ORDER = {"phased": 0, "raster": 1, "independent": 2}
TILING = {"alg1": 0, "vertical": 1}
OPT_EXEC_MODE, OPT_TIMEOUT_MS, OPT_CTAS_PER_SM, OPT_USE_GRAPH, OPT_DEBUG_CAPTURE, OPT_KERNEL_TIMING = 1, 2, 3, 4, 5, 6
OPT_F64_WARPS, OPT_F32_LAYOUT, OPT_TMA_STAGING, OPT_DEBUG_TMA_STALL = 7, 8, 9, 10
OPT_F32_UNROLL, OPT_F64_UNROLL, OPT_CLASS_LAUNCH, OPT_SERVER_CLASSES = 11, 12, 13, 14
OPT_ROOT_WINDOW = 15
EXEC = {"dag": 0, "levels": 1, "per_block": 2}
REQ_QUEUED, REQ_RUNNING, REQ_DONE, REQ_FAILED = 0, 1, 2, 3


class FseError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"fse error {code}: {msg}")
        self.code = code


class Tile(ctypes.Structure):
    _fields_ = [(n, ctypes.c_int32) for n in ("x", "y", "w", "h", "ex", "ey", "ew", "eh")]


class Params(ctypes.Structure):
    _fields_ = [("block", ctypes.c_int32), ("border", ctypes.c_int32), ("fft", ctypes.c_int32),
                ("K", ctypes.c_int32), ("rho", ctypes.c_double), ("delta", ctypes.c_double),
                ("gamma", ctypes.c_double), ("order", ctypes.c_int32), ("n_tiles", ctypes.c_int32),
                ("overlap", ctypes.c_int32), ("precision", ctypes.c_int32),
                ("tiling", ctypes.c_int32)]


class Job(ctypes.Structure):
    _fields_ = [("image", ctypes.c_void_p), ("mask", ctypes.c_void_p), ("out", ctypes.c_void_p),
                ("out_f32", ctypes.c_void_p), ("out_f64", ctypes.c_void_p), ("W", ctypes.c_int32), ("H", ctypes.c_int32),
                ("pitch", ctypes.c_int32), ("p", Params)]


class Stats(ctypes.Structure):
    _fields_ = [("lost_blocks", ctypes.c_int64), ("core_lost_blocks", ctypes.c_int64),
                ("empty_blocks", ctypes.c_int64), ("pixels", ctypes.c_int64),
                ("bin_iterations", ctypes.c_int64), ("jobs", ctypes.c_int32),
                ("tiles", ctypes.c_int32), ("launches", ctypes.c_int32),
                ("graph_replayed", ctypes.c_int32), ("device_ms", ctypes.c_float),
                ("exec_ms", ctypes.c_float), ("class_blocks", ctypes.c_int64 * 3),
                ("class_bin_iterations", ctypes.c_int64 * 3)]

    def as_dict(self):
        d = {n: getattr(self, n) for n, _ in self._fields_}
        for n in ("class_blocks", "class_bin_iterations"):
            d[n] = list(d[n])
        return d


class ServerCfg(ctypes.Structure):
    _fields_ = [("arena_bytes", ctypes.c_size_t), ("max_queue", ctypes.c_int32),
                ("max_resident", ctypes.c_int32), ("max_batch", ctypes.c_int32)]


EXPORTS = ["fse_plan_tiles", "fse_plan_tiles_vertical", "fse_context_create", "fse_context_destroy", "fse_context_set_option",
           "fse_extrapolate_batch", "fse_extrapolate_host", "fse_server_create", "fse_submit",
           "fse_poll", "fse_wait", "fse_server_latencies", "fse_server_destroy", "fse_last_error",
           "fse_debug_fetch", "fse_debug_wait_probe", "fse_context_kernel_times",
           "fse_extrapolate_noalloc", "fse_autotune", "fse_context_class_times", "fse_cancel", "fse_server_debug_state"]

_lib = None


def load(path=LIB_PATH):
    """Loads the built library (``build()`` first); raises if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"libfse.so not built at {path}: run paper_2207_00238_gb300.build.build()")
    L = ctypes.CDLL(path)
    P, i32, vp = ctypes.POINTER, ctypes.c_int32, ctypes.c_void_p
    L.fse_plan_tiles.argtypes = [i32, i32, i32, i32, P(Tile), i32, P(i32)]
    L.fse_plan_tiles_vertical.argtypes = [i32, i32, i32, i32, P(Tile), i32, P(i32)]
    L.fse_context_create.argtypes = [P(vp), ctypes.c_int, ctypes.c_size_t, ctypes.c_char_p]
    L.fse_context_destroy.argtypes = [vp]
    L.fse_context_destroy.restype = None
    L.fse_context_set_option.argtypes = [vp, i32, ctypes.c_int64]
    L.fse_extrapolate_batch.argtypes = [vp, P(Job), i32, vp, P(Stats)]
    L.fse_extrapolate_host.argtypes = [vp, P(Job), i32, vp, P(Stats)]
    L.fse_server_create.argtypes = [P(vp), vp, P(ServerCfg)]
    L.fse_submit.argtypes = [vp, P(Job), P(ctypes.c_uint64)]
    L.fse_poll.argtypes = [vp, ctypes.c_uint64, P(i32)]
    L.fse_cancel.argtypes = [vp, ctypes.c_uint64]
    L.fse_server_debug_state.argtypes = [vp, P(ctypes.c_int64), i32]
    L.fse_server_debug_state.restype = i32
    L.fse_wait.argtypes = [vp, ctypes.c_uint64, i32, P(Stats)]
    L.fse_server_latencies.argtypes = [vp, P(ctypes.c_double), i32]
    L.fse_server_latencies.restype = i32
    L.fse_server_destroy.argtypes = [vp]
    L.fse_server_destroy.restype = None
    L.fse_last_error.restype = ctypes.c_char_p
    L.fse_debug_fetch.argtypes = [vp, P(i32), P(i32), i32, P(i32)]
    L.fse_debug_fetch.restype = i32
    L.fse_debug_wait_probe.argtypes = [vp, i32]
    L.fse_extrapolate_noalloc.argtypes = [P(Job), i32, vp]
    L.fse_autotune.argtypes = [vp, P(Job), i32, vp, i32, P(ctypes.c_double), i32]
    L.fse_autotune.restype = i32
    L.fse_context_kernel_times.argtypes = [vp, P(ctypes.c_float), i32]
    L.fse_context_kernel_times.restype = i32
    L.fse_context_class_times.argtypes = [vp, P(ctypes.c_float), i32]
    L.fse_context_class_times.restype = i32
    _lib = L
    return L


def build(force=False):
    return _build.build(force=force)


def _check(rc):
    if rc < 0:
        raise FseError(rc, load().fse_last_error().decode())
    return rc


def plan_tiles(W, H, N, d, tiling="alg1"):
    """Algorithm 1 (or the vertical stripes) + overlap d.  Returns int32 array
    [N, 8] (x, y, w, h, ex, ey, ew, eh)."""
    L = load()
    arr = (Tile * max(N, 1))()
    n = ctypes.c_int32(0)
    fn = L.fse_plan_tiles_vertical if tiling == "vertical" else L.fse_plan_tiles
    _check(fn(W, H, N, d, arr, max(N, 1), ctypes.byref(n)))
    return np.array([[getattr(arr[i], f) for f, _ in Tile._fields_] for i in range(n.value)],
                    np.int32).reshape(-1, 8)


def extrapolate_noalloc(jobs, stream=None):
    """fse_extrapolate_noalloc: the batch pass without any allocation, for
    callers that cannot allocate device memory.  Device pointers of the
    current device; returns once the work on `stream` has finished."""
    arr = (Job * len(jobs))(*jobs)
    _check(load().fse_extrapolate_noalloc(arr, len(jobs), stream))


def make_params(block, border, fft, K, rho=0.8, delta=0.5, gamma=0.5, order="phased",
                n_tiles=1, overlap=32, precision=32, tiling="alg1", **_):
    return Params(block, border, fft, K, rho, delta, gamma,
                  ORDER[order] if isinstance(order, str) else int(order), n_tiles, overlap, precision,
                  TILING[tiling] if isinstance(tiling, str) else int(tiling))


def _ptr(t):
    if t is None:
        return None
    if hasattr(t, "data_ptr"):
        return t.data_ptr()
    return t.ctypes.data


def make_job(image, mask, out, params, out_f32=None, out_f64=None):
    """image/mask/out: 2-D uint8 (torch CUDA tensors for the device path, numpy
    arrays for the host path), same shape and row pitch."""
    H, W = image.shape[-2], image.shape[-1]
    pitch = image.stride(0) if hasattr(image, "stride") and callable(image.stride) else image.strides[0]
    if not isinstance(params, Params):
        params = make_params(**params)
    return Job(_ptr(image), _ptr(mask), _ptr(out), _ptr(out_f32), _ptr(out_f64), W, H, pitch, params)


class Context:
    """One GPU, one device arena.  Not thread-safe; use one per thread."""

    def __init__(self, device=0, arena_bytes=1 << 30, tune_cache=None):
        L = load()
        h = ctypes.c_void_p()
        _check(L.fse_context_create(ctypes.byref(h), device, arena_bytes,
                                    tune_cache.encode() if tune_cache else None))
        self.h = h
        self.device = device

    def close(self):
        if self.h:
            load().fse_context_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_option(self, key, value):
        _check(load().fse_context_set_option(self.h, key, int(value)))

    def exec_mode(self, mode):
        self.set_option(OPT_EXEC_MODE, EXEC[mode])

    def extrapolate(self, jobs, stream=None, stats=True):
        """Device-pointer batch (fse_extrapolate_batch)."""
        arr = (Job * len(jobs))(*jobs)
        st = Stats() if stats else None
        _check(load().fse_extrapolate_batch(self.h, arr, len(jobs), stream,
                                            ctypes.byref(st) if st is not None else None))
        return st.as_dict() if st is not None else None

    def extrapolate_host(self, jobs, stream=None, stats=False):
        """Host-pointer batch (fse_extrapolate_host): copies in, runs, copies out."""
        arr = (Job * len(jobs))(*jobs)
        st = Stats() if stats else None
        _check(load().fse_extrapolate_host(self.h, arr, len(jobs), stream,
                                           ctypes.byref(st) if st is not None else None))
        return st.as_dict() if st is not None else None

    def debug_fetch(self, cap):
        rec = np.zeros((cap, 4), np.int32)
        useq = np.zeros((cap, 256), np.int32)
        kmax = ctypes.c_int32(0)
        P = ctypes.POINTER(ctypes.c_int32)
        n = _check(load().fse_debug_fetch(self.h, rec.ctypes.data_as(P), useq.ctypes.data_as(P), cap,
                                          ctypes.byref(kmax)))
        K = kmax.value
        useq = useq.ravel()[: cap * K].reshape(cap, K) if K else np.zeros((cap, 0), np.int32)
        return rec[:n], useq[:n]

    def autotune(self, jobs, stream=None, reps=3):
        """fse_autotune: picks and applies the fastest launch configuration for
        this job mix; returns the timed candidates (class, layout, ctas, ms)."""
        arr = (Job * len(jobs))(*jobs)
        cap = 64
        tr = (ctypes.c_double * (4 * cap))()
        n = _check(load().fse_autotune(self.h, arr, len(jobs), stream, reps, tr, cap))
        return [tuple(tr[4 * i:4 * i + 4]) for i in range(min(n, cap))]

    def kernel_times(self, cap=4096):
        """Iteration-kernel milliseconds per call since FSE_OPT_KERNEL_TIMING was set."""
        ms = (ctypes.c_float * cap)()
        n = _check(load().fse_context_kernel_times(self.h, ms, cap))
        return [ms[i] for i in range(n)]

    def class_times(self, cap=4096):
        """Per-class iteration-kernel milliseconds [[F=32, F=64, FP64], ...] of
        each timed call (does not forget them; kernel_times does)."""
        ms = (ctypes.c_float * (3 * cap))()
        n = _check(load().fse_context_class_times(self.h, ms, cap))
        return [[ms[3 * i + k] for k in range(3)] for i in range(n)]

    def wait_probe(self, timeout_us):
        return load().fse_debug_wait_probe(self.h, timeout_us)


class Server:
    """Continuous-batching request server (fse_server_*).  Host buffers."""

    def __init__(self, ctx, arena_bytes=4 << 30, max_queue=256, max_resident=64, max_batch=16):
        L = load()
        h = ctypes.c_void_p()
        cfg = ServerCfg(arena_bytes, max_queue, max_resident, max_batch)
        _check(L.fse_server_create(ctypes.byref(h), ctx.h, ctypes.byref(cfg)))
        self.h = h
        self._keep = {}

    def submit(self, image, mask, out, params, out_f32=None):
        """image/mask/out: numpy uint8 arrays (out must stay alive until wait)."""
        job = make_job(image, mask, out, params, out_f32=out_f32)
        t = ctypes.c_uint64(0)
        _check(load().fse_submit(self.h, ctypes.byref(job), ctypes.byref(t)))
        self._keep[t.value] = (out, out_f32)
        return t.value

    def cancel(self, ticket):
        _check(load().fse_cancel(self.h, ticket))

    def poll(self, ticket):
        st = ctypes.c_int32(0)
        _check(load().fse_poll(self.h, ticket, ctypes.byref(st)))
        return st.value

    def wait(self, ticket, timeout_ms=-1):
        st = Stats()
        rc = load().fse_wait(self.h, ticket, timeout_ms, ctypes.byref(st))
        if rc == OK:
            self._keep.pop(ticket, None)
        _check(rc)
        return st.as_dict()

    def debug_state(self):
        """fse_server_debug_state: per class and per occupied slot counters."""
        buf = (ctypes.c_int64 * 2064)()
        n = _check(load().fse_server_debug_state(self.h, buf, 2064))
        a = list(buf[:n])
        slots = [a[16 + 8 * i:24 + 8 * i] for i in range(256)]
        return {"f32": a[0:8], "f64": a[8:16], "slots": [s for s in slots if s[0] != -1]}

    def latencies(self, cap=1 << 20):
        buf = (ctypes.c_double * cap)()
        n = _check(load().fse_server_latencies(self.h, buf, cap))
        return np.frombuffer(buf, dtype=np.float64, count=n).copy()

    def close(self):
        if self.h:
            load().fse_server_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
