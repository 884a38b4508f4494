"""GB300-native CudaChain: planar convex hulls on the GPU (sm_103a).

Thin ctypes binding over ``libcch.so`` (C ABI in ``include/cch.h``).  The
binding only marshals arguments: every step of the hull runs in the CUDA
kernels of ``csrc/``.  There is no CPU fallback -- if the library is missing
or cannot be loaded, every call raises.

PyTorch supplies device memory and streams; tensors must be contiguous
``[n, 2]`` int32 or float64 on a CUDA device.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libcch.so")

CCH_I32 = 1
CCH_F64 = 2
STATUS = {0: "ok", -1: "invalid argument", -2: "unsupported dtype", -3: "non-finite coordinate",
          -4: "out of range", -5: "out of memory", -6: "CUDA error", -7: "device wait timeout",
          -8: "server busy", -9: "unknown ticket"}

_lock = threading.Lock()
_lib = None


class ServeConfig(ctypes.Structure):
    """cch_serve_config."""
    _fields_ = [("budget_bytes", ctypes.c_size_t), ("num_streams", ctypes.c_int32),
                ("max_pending", ctypes.c_int32), ("max_batch", ctypes.c_int32), ("dtype", ctypes.c_int32)]


class TuneParams(ctypes.Structure):
    """cch_tune_params."""
    _fields_ = [("small_max", ctypes.c_int32), ("stair_div", ctypes.c_int32), ("stair_min", ctypes.c_int32),
                ("stair_max", ctypes.c_int32), ("a1_len_min", ctypes.c_int32), ("cls_per_sm", ctypes.c_int32)]

    def as_dict(self) -> dict:
        return {f: int(getattr(self, f)) for f, _ in self._fields_}


class Done(ctypes.Structure):
    """cch_done."""
    _fields_ = [("ticket", ctypes.c_uint64), ("status", ctypes.c_int32), ("count", ctypes.c_int32),
                ("idx", ctypes.POINTER(ctypes.c_int32)), ("latency_ms", ctypes.c_double)]


class CchError(RuntimeError):
    def __init__(self, code: int, what: str = ""):
        self.code = int(code)
        super().__init__(f"{what}: {STATUS.get(self.code, 'status')} ({self.code})")


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is not built; run "
                               "`python -c 'import __graft_entry__ as g; g.build()'`")
        lib = ctypes.CDLL(LIB_PATH)
        vp, i64, i32, u32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_uint32
        lib.cch_status_string.restype = ctypes.c_char_p
        lib.cch_status_string.argtypes = [ctypes.c_int]
        lib.cch_hull.restype = ctypes.c_int
        lib.cch_hull.argtypes = [vp, i64, ctypes.c_int, vp, vp, vp]
        lib.cch_hull_batched.restype = ctypes.c_int
        lib.cch_hull_batched.argtypes = [vp, vp, i32, ctypes.c_int, vp, vp, vp]
        lib.cch_hull_noalloc.restype = ctypes.c_int
        lib.cch_hull_noalloc.argtypes = [vp, i64, ctypes.c_int, vp, vp, vp]
        lib.cch_hull_host.restype = ctypes.c_int
        lib.cch_hull_host.argtypes = [vp, i64, ctypes.c_int, vp, vp, vp]
        lib.cch_hull_f32soa.restype = ctypes.c_int
        lib.cch_hull_f32soa.argtypes = [vp, vp, i64, vp, vp, vp]
        lib.cch_hull_stages.restype = ctypes.c_int
        lib.cch_hull_stages.argtypes = [vp, i64, ctypes.c_int, u32, vp, vp, vp, vp, vp, vp, vp]
        lib.cch_workspace_bytes.restype = ctypes.c_size_t
        lib.cch_workspace_bytes.argtypes = [i64, ctypes.c_int]
        lib.cch_release_workspace.restype = None
        lib.cch_release_workspace.argtypes = []
        lib.cch_profile.restype = ctypes.c_int
        lib.cch_profile.argtypes = [ctypes.c_int]
        lib.cch_profile_stages.restype = ctypes.c_int
        lib.cch_profile_stages.argtypes = [ctypes.c_uint32]
        lib.cch_profile_read.restype = ctypes.c_int
        lib.cch_profile_read.argtypes = [vp, ctypes.c_int, vp]
        lib.cch_launch_count.restype = ctypes.c_uint64
        lib.cch_launch_count.argtypes = []
        lib.cch_selftest_wait.restype = ctypes.c_int
        lib.cch_selftest_wait.argtypes = [vp, vp]
        tp = ctypes.POINTER(TuneParams)
        lib.cch_tune_bucket.restype = ctypes.c_int
        lib.cch_tune_bucket.argtypes = [i64, i32]
        for name in ("cch_tune_set", "cch_tune_get"):
            getattr(lib, name).restype = ctypes.c_int
            getattr(lib, name).argtypes = [ctypes.c_char_p, i32, i32, i32, i32, tp]
        lib.cch_tune_clear.restype = ctypes.c_int
        lib.cch_tune_clear.argtypes = []
        for name in ("cch_tune_save", "cch_tune_load"):
            getattr(lib, name).restype = ctypes.c_int
            getattr(lib, name).argtypes = [ctypes.c_char_p]
        lib.cch_autotune_batched.restype = ctypes.c_int
        lib.cch_autotune_batched.argtypes = [vp, vp, i32, i32, vp, vp, vp, i32, tp]
        for name in ("cch_serve_create", "cch_serve_submit", "cch_serve_poll", "cch_serve_release",
                     "cch_serve_stats", "cch_serve_destroy"):
            getattr(lib, name).restype = ctypes.c_int
        lib.cch_serve_create.argtypes = [ctypes.POINTER(ServeConfig), ctypes.POINTER(vp)]
        lib.cch_serve_submit.argtypes = [vp, vp, i64, ctypes.POINTER(ctypes.c_uint64)]
        lib.cch_serve_submit_device.restype = ctypes.c_int
        lib.cch_serve_submit_device.argtypes = [vp, vp, i64, vp, ctypes.POINTER(ctypes.c_uint64)]
        lib.cch_serve_poll.argtypes = [vp, ctypes.POINTER(Done), ctypes.c_int, ctypes.POINTER(ctypes.c_int)]
        lib.cch_serve_release.argtypes = [vp, ctypes.c_uint64]
        lib.cch_serve_stats.argtypes = [vp, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double),
                                        ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int64)]
        lib.cch_serve_destroy.argtypes = [vp]
        _lib = lib
        return lib


def lib():
    """The loaded C library (ctypes.CDLL)."""
    return _load()


def _check(rc: int, what: str):
    if rc != 0:
        raise CchError(rc, what)


def _dtype_code(t) -> int:
    import torch
    if t.dtype == torch.int32:
        return CCH_I32
    if t.dtype == torch.float64:
        return CCH_F64
    raise TypeError(f"points must be int32 or float64, got {t.dtype}")


def _stream_handle(stream=None) -> int:
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return int(s.cuda_stream)


def _check_points(points):
    if not points.is_cuda:
        raise ValueError("points must be a CUDA tensor (use hull_host for host arrays)")
    if points.dim() != 2 or points.shape[1] != 2 or not points.is_contiguous():
        raise ValueError("points must be a contiguous [n, 2] tensor")


def hull_async(points, out_idx=None, out_count=None, stream=None):
    """Enqueue one hull on `stream` (default: current stream).

    Returns (out_idx int32[max(n,1)], out_count int32[1]) device tensors; the
    first out_count[0] entries of out_idx are the hull indices once the stream
    reaches them.  A negative count is a device-side error code."""
    import torch
    _check_points(points)
    n = points.shape[0]
    dev = points.device
    if out_idx is None:
        out_idx = torch.empty(max(n, 1), dtype=torch.int32, device=dev)
    if out_count is None:
        out_count = torch.empty(1, dtype=torch.int32, device=dev)
    rc = _load().cch_hull(points.data_ptr() if n else None, n, _dtype_code(points),
                          out_idx.data_ptr(), out_count.data_ptr(), _stream_handle(stream))
    _check(rc, "cch_hull")
    return out_idx, out_count


def hull(points, stream=None):
    """Hull vertex indices (int32 CUDA tensor, CCW from the lexicographic
    minimum).  Synchronises the stream to read the count."""
    out_idx, out_count = hull_async(points, stream=stream)
    h = int(out_count.item())
    if h < 0:
        raise CchError(h, "cch_hull (device)")
    return out_idx[:h]


def hull_f32soa_async(x, y, out_idx=None, out_count=None, stream=None):
    """Enqueue the hull of the points (x[i], y[i]) given as two float32 CUDA
    vectors (the paper's input form).  Round 1 reads the two vectors
    directly; later stages carry the coordinates widened exactly to float64,
    so the result is hull_async's on torch.stack([x, y], 1).double().
    Returns (out_idx, out_count) device tensors as hull_async does."""
    import torch
    for t in (x, y):
        if not t.is_cuda or t.dtype != torch.float32 or t.dim() != 1 or not t.is_contiguous():
            raise ValueError("x and y must be contiguous 1-D float32 CUDA tensors")
    if x.shape[0] != y.shape[0]:
        raise ValueError("x and y must have the same length")
    n = x.shape[0]
    dev = x.device
    if out_idx is None:
        out_idx = torch.empty(max(n, 1), dtype=torch.int32, device=dev)
    if out_count is None:
        out_count = torch.empty(1, dtype=torch.int32, device=dev)
    rc = _load().cch_hull_f32soa(x.data_ptr() if n else None, y.data_ptr() if n else None, n,
                                 out_idx.data_ptr(), out_count.data_ptr(), _stream_handle(stream))
    _check(rc, "cch_hull_f32soa")
    return out_idx, out_count


def hull_f32soa(x, y, stream=None):
    """Hull vertex indices of float32 SoA points (synchronises)."""
    out_idx, out_count = hull_f32soa_async(x, y, stream=stream)
    h = int(out_count.item())
    if h < 0:
        raise CchError(h, "cch_hull_f32soa (device)")
    return out_idx[:h]


def hull_batched_async(points, offsets, out_idx=None, out_counts=None, stream=None):
    """Enqueue the hulls of sets points[offsets[s]:offsets[s+1]].
    Returns (out_idx, out_counts) device tensors; set s's indices (local to
    the set) start at out_idx[offsets[s]]."""
    import torch
    _check_points(points)
    off = np.ascontiguousarray(np.asarray(offsets, dtype=np.int64))
    nsets = off.shape[0] - 1
    N = int(off[-1]) if nsets >= 0 else 0
    dev = points.device
    if out_idx is None:
        out_idx = torch.empty(max(N, 1), dtype=torch.int32, device=dev)
    if out_counts is None:
        out_counts = torch.empty(max(nsets, 1), dtype=torch.int32, device=dev)
    rc = _load().cch_hull_batched(points.data_ptr() if N else None, off.ctypes.data, nsets,
                                  _dtype_code(points), out_idx.data_ptr(), out_counts.data_ptr(),
                                  _stream_handle(stream))
    _check(rc, "cch_hull_batched")
    return out_idx, out_counts


def hull_batched(points, offsets, stream=None):
    """List of per-set hull index tensors (synchronises)."""
    out_idx, out_counts = hull_batched_async(points, offsets, stream=stream)
    counts = out_counts.cpu().numpy()
    res = []
    for s in range(len(offsets) - 1):
        h = int(counts[s])
        if h < 0:
            raise CchError(h, f"cch_hull_batched set {s}")
        o = int(offsets[s])
        res.append(out_idx[o:o + h])
    return res


def hull_host(points: np.ndarray, stream=None) -> np.ndarray:
    """End to end from host memory: copy in, hull, copy out (numpy int32)."""
    p = np.ascontiguousarray(points)
    if p.dtype == np.int32:
        dt = CCH_I32
    elif p.dtype == np.float64:
        dt = CCH_F64
    else:
        raise TypeError("points must be int32 or float64")
    n = p.shape[0]
    out = np.empty(max(n, 1), dtype=np.int32)
    cnt = np.zeros(1, dtype=np.int32)
    rc = _load().cch_hull_host(p.ctypes.data if n else None, n, dt, out.ctypes.data,
                               cnt.ctypes.data, _stream_handle(stream))
    _check(rc, "cch_hull_host")
    return out[:int(cnt[0])].copy()


def hull_host_ptr(host_ptr: int, n: int, dtype_code: int, out_idx_ptr: int, out_count_ptr: int,
                  stream=None) -> int:
    """cch_hull_host on raw host pointers (e.g. pinned tensors); returns the status."""
    return _load().cch_hull_host(host_ptr, n, dtype_code, out_idx_ptr, out_count_ptr,
                                 _stream_handle(stream))


def stages(points, exact_only: bool = False, prefilter: bool = True, blocked: bool = False,
           octagon: bool = False, stream=None) -> dict:
    """Run one hull and return its intermediate sets (synchronises).

    exact_only  every float64 quadrilateral test in exact arithmetic (no FP32 filter)
    prefilter   drop SPA-dominated points already in round 1 (default); with
                False the round-1 sets are exactly the paper's R1..R4
    blocked     ``spa`` is the paper's chunked GPU SPA (Sec. 2.2.2: 1024
                chunks per region, each restarting at its first point) on the
                paper's round-1 sets (implies prefilter=False); the hull is
                the same
    octagon     round 1 discards the points strictly inside the octagon of the
                four extremes and the four diagonal extremes (implies
                prefilter=False); ``diag`` holds the diagonal extremes used
                (-1 where none)

    ``r1`` list of 4 int32 arrays (round-1 survivors per region, index order),
    ``spa`` list of 4 int32 arrays (SPA survivors per region, sorted order),
    ``hull`` int32 array, ``counts`` int64[16], ``status``, ``passes`` (radix
    passes of the multi-block sort, 0 on the shared-memory path)."""
    import torch
    _check_points(points)
    n = points.shape[0]
    dev = points.device
    m = max(n, 1)
    r1 = torch.empty(m, dtype=torch.int32, device=dev)
    r1r = torch.empty(m, dtype=torch.int32, device=dev)
    spa = torch.empty(m, dtype=torch.int32, device=dev)
    out_idx = torch.empty(m, dtype=torch.int32, device=dev)
    out_count = torch.empty(1, dtype=torch.int32, device=dev)
    counts = np.zeros(16, dtype=np.int64)
    rc = _load().cch_hull_stages(points.data_ptr() if n else None, n, _dtype_code(points),
                                 (1 if exact_only else 0) | (0 if prefilter else 2) | (4 if blocked else 0)
                                 | (8 if octagon else 0),
                                 r1.data_ptr(), r1r.data_ptr(),
                                 spa.data_ptr(), counts.ctypes.data, out_idx.data_ptr(),
                                 out_count.data_ptr(), _stream_handle(stream))
    _check(rc, "cch_hull_stages")
    s1 = int(counts[0])
    r1_idx = r1[:s1].cpu().numpy()
    r1_reg = r1r[:s1].cpu().numpy()
    spa_all = spa[:int(counts[5:9].sum())].cpu().numpy()
    spa_list, o = [], 0
    for r in range(4):
        c = int(counts[5 + r])
        spa_list.append(spa_all[o:o + c])
        o += c
    h = int(out_count.item())
    return {
        "r1": [r1_idx[r1_reg == r + 1] for r in range(4)],
        "r1_counts": counts[1:5].copy(),
        "spa": spa_list,
        "hull": out_idx[:max(h, 0)].cpu().numpy(),
        "count": h,
        "counts": counts,
        "status": int(counts[9]),
        "passes": int(counts[10]),
        "diag": counts[11:15].copy(),
    }


STAGE_NAMES = ("k_extremes", "k_stairs", "k_classify", "gather", "small", "big", "chain", "blocked_spa")


def profile(enable: bool = True):
    """Record CUDA events around the pipeline stages of every later call."""
    _check(_load().cch_profile(1 if enable else 0), "cch_profile")


def profile_stages(names) -> None:
    """Record events only around the named stages (see STAGE_NAMES)."""
    mask = 0
    for n in names:
        mask |= 1 << STAGE_NAMES.index(n)
    _check(_load().cch_profile_stages(mask), "cch_profile_stages")


def profile_read() -> tuple[dict, int]:
    """Summed milliseconds per stage since the last read, and the call count."""
    ms = np.zeros(len(STAGE_NAMES), dtype=np.float64)
    calls = np.zeros(1, dtype=np.int64)
    k = _load().cch_profile_read(ms.ctypes.data, len(STAGE_NAMES), calls.ctypes.data)
    if k < 0:
        raise CchError(k, "cch_profile_read")
    return {STAGE_NAMES[i]: float(ms[i]) for i in range(k)}, int(calls[0])


def tune_set(params: dict, dtype_code: int, batched: bool, bucket: int, gpu: str | None = None, sms: int = 0):
    """Table entry of (gpu, sms, dtype, batched, bucket); gpu None = the current device."""
    p = TuneParams(**params)
    _check(_load().cch_tune_set(gpu.encode() if gpu else None, sms, dtype_code, int(batched), bucket,
                                ctypes.byref(p)), "cch_tune_set")


def tune_get(dtype_code: int, batched: bool, bucket: int, gpu: str | None = None, sms: int = 0):
    """(params dict, found) for the key; the defaults when there is no entry."""
    p = TuneParams()
    rc = _load().cch_tune_get(gpu.encode() if gpu else None, sms, dtype_code, int(batched), bucket, ctypes.byref(p))
    if rc not in (0, -9):
        raise CchError(rc, "cch_tune_get")
    return p.as_dict(), rc == 0


def autotune_batched(points, offsets, out_idx=None, out_counts=None, reps: int = 3, stream=None) -> dict:
    """Measure the run-time choices on this batch and keep the fastest for its key."""
    import torch
    _check_points(points)
    off = np.ascontiguousarray(offsets, dtype=np.int64)
    nsets = off.shape[0] - 1
    n = int(off[-1])
    if out_idx is None:
        out_idx = torch.empty(max(n, 1), dtype=torch.int32, device=points.device)
    if out_counts is None:
        out_counts = torch.empty(max(nsets, 1), dtype=torch.int32, device=points.device)
    best = TuneParams()
    _check(_load().cch_autotune_batched(points.data_ptr() if n else None, off.ctypes.data, nsets, _dtype_code(points),
                                        out_idx.data_ptr(), out_counts.data_ptr(), _stream_handle(stream), reps,
                                        ctypes.byref(best)), "cch_autotune_batched")
    return best.as_dict()


def launch_count() -> int:
    """Kernels launched by the library so far."""
    return int(_load().cch_launch_count())


def workspace_bytes(n: int, dtype_code: int = CCH_F64) -> int:
    return int(_load().cch_workspace_bytes(n, dtype_code))


def release_workspace():
    _load().cch_release_workspace()


class Server:
    """Hull server (cch_serve_*): requests are admitted by a device-memory
    budget and batched onto a pool of streams as they arrive.

    ``submit`` copies a ``[n, 2]`` array -- a host array, or a CUDA tensor,
    which stays in device memory (cch_serve_submit_device, ordered after the
    current stream) -- and returns a ticket; ``poll`` returns the finished
    requests as ``(ticket, status, hull, latency_ms)`` with ``hull`` a NumPy
    copy (the server's copy is released at once)."""

    def __init__(self, dtype=np.float64, budget_bytes: int = 0, num_streams: int = 0, max_pending: int = 0,
                 max_batch: int = 0):
        self.dtype = np.dtype(dtype)
        code = CCH_F64 if self.dtype == np.float64 else CCH_I32 if self.dtype == np.int32 else None
        if code is None:
            raise TypeError("points must be int32 or float64")
        cfg = ServeConfig(budget_bytes, num_streams, max_pending, max_batch, code)
        h = ctypes.c_void_p()
        _check(_load().cch_serve_create(ctypes.byref(cfg), ctypes.byref(h)), "cch_serve_create")
        self._h = h

    def submit(self, points, stream=None) -> int:
        if getattr(points, "is_cuda", False):
            import torch
            _check_points(points)
            if points.dtype != (torch.float64 if self.dtype == np.float64 else torch.int32):
                raise TypeError("device points must match the server's dtype")
            t = ctypes.c_uint64()
            _check(_load().cch_serve_submit_device(self._h, points.data_ptr() if points.shape[0] else None,
                                                   points.shape[0], _stream_handle(stream), ctypes.byref(t)),
                   "cch_serve_submit_device")
            return int(t.value)
        p = np.ascontiguousarray(points, dtype=self.dtype)
        if p.ndim != 2 or p.shape[1] != 2:
            raise ValueError("points must be [n, 2]")
        t = ctypes.c_uint64()
        _check(_load().cch_serve_submit(self._h, p.ctypes.data, p.shape[0], ctypes.byref(t)), "cch_serve_submit")
        return int(t.value)

    def poll(self, max_results: int = 256):
        arr = (Done * max_results)()
        k = ctypes.c_int()
        lib_ = _load()
        _check(lib_.cch_serve_poll(self._h, arr, max_results, ctypes.byref(k)), "cch_serve_poll")
        out = []
        for i in range(k.value):
            d = arr[i]
            h = np.ctypeslib.as_array(d.idx, shape=(d.count,)).copy() if d.count > 0 else np.zeros(0, np.int32)
            out.append((int(d.ticket), int(d.status), h, float(d.latency_ms)))
            _check(lib_.cch_serve_release(self._h, d.ticket), "cch_serve_release")
        return out

    def stats(self) -> dict:
        p50, p99, hps = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
        n = ctypes.c_int64()
        _check(_load().cch_serve_stats(self._h, ctypes.byref(p50), ctypes.byref(p99), ctypes.byref(hps),
                                       ctypes.byref(n)), "cch_serve_stats")
        return {"p50_ms": p50.value, "p99_ms": p99.value, "hulls_per_s": hps.value, "finished": n.value}

    def close(self):
        if self._h:
            _check(_load().cch_serve_destroy(self._h), "cch_serve_destroy")
            self._h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
