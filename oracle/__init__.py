"""CPU oracle for the CudaChain convex hull -- TEST INFRASTRUCTURE ONLY.

Only the test suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product library never does: the
CUDA path and this oracle share no code.

Contents
  * ``hull(points)``      -- the definition of the output (strict convex hull
    vertex indices, CCW, starting at the lexicographic (x, y) minimum, each
    vertex the smallest index among identical points), by Andrew's monotone
    chain (the paper's reference [4], Sec. 1) on exact predicates, in C.
  * ``method(points)``    -- the paper's procedure step by step (Sec. 2.1
    steps 1-7, Table 1, Sec. 2.1.1, Fig. 2), returning every intermediate set.
  * ``orient(a, b, c)``   -- the exact orientation predicate used by both.
  * ``bruteforce``        -- O(n^3) hull and O(n^2) SPA by exact rationals, the
    pins for the C code.
  * ``blocked_spa(points)`` -- the SPA of the paper's GPU implementation
    (Sec. 2.2.2): each region's sorted points in 1024 consecutive chunks,
    Fig. 2's rule restarted at every chunk's first point.
  * ``diag_extremes(points)``, ``octagon_round1(points, diag)`` -- round 1
    with the Akl-Toussaint octagon (the paper's reference [17]) in place of
    the quadrilateral: the four diagonal extremes and the round-1 / SPA sets
    without the points strictly inside the octagon.
  * ``parallel_hull(points)`` -- the multi-core CPU baseline the benchmark
    times beside the oracle (OpenMP: octagon filter, parallel merge sort,
    Andrew's chain; ``cch_cpu_parallel.c`` includes the oracle's source for
    its exact predicates); the tests check it returns exactly ``hull``.

Parity status: every function here is pinned by tests in ``tests/test_oracle*.py``
against brute force on exact rationals, closed forms and invariants, except
the survivor COUNTS of Fig. 11, which the paper prints only as a plot
(parity unpinned for those counts).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "cch_oracle.c")
_LIB = os.path.join(_HERE, "libcchoracle.so")
_PSRC = os.path.join(_HERE, "cch_cpu_parallel.c")
_PLIB = os.path.join(_HERE, "libcchpar.so")
_lock = threading.Lock()
_lib = None
_plib = None

I32 = 1
F64 = 2


def build(force: bool = False) -> str:
    """Compile the C oracle with gcc (-ffp-contract=off keeps every product
    and sum separately rounded, which the exact predicate relies on)."""
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math",
           "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


def build_parallel(force: bool = False):
    """Compile the multi-core CPU baseline (OpenMP; it includes the oracle's
    source).  Returns the library path, or None where gcc has no OpenMP."""
    newest = max(os.path.getmtime(_SRC), os.path.getmtime(_PSRC))
    if not force and os.path.exists(_PLIB) and os.path.getmtime(_PLIB) >= newest:
        return _PLIB
    tmp = _PLIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-ffp-contract=off", "-fno-fast-math",
           "-fPIC", "-shared", "-o", tmp, _PSRC, "-lm"]
    r = subprocess.run(cmd, capture_output=True, text=True, cwd=_HERE)
    if r.returncode != 0:
        return None
    os.replace(tmp, _PLIB)
    return _PLIB


def _load_parallel():
    global _plib
    with _lock:
        if _plib is None:
            path = build_parallel()
            if path is None:
                return None
            lib = ctypes.CDLL(path)
            vp, i64 = ctypes.c_void_p, ctypes.c_int64
            lib.cpu_parallel_hull_i32.restype = i64
            lib.cpu_parallel_hull_i32.argtypes = [vp, i64, vp, ctypes.c_int]
            lib.cpu_parallel_hull_f64.restype = i64
            lib.cpu_parallel_hull_f64.argtypes = [vp, i64, vp, ctypes.c_int]
            lib.cpu_parallel_threads.restype = ctypes.c_int
            lib.cpu_parallel_threads.argtypes = []
            _plib = lib
    return _plib


def parallel_available() -> bool:
    return _load_parallel() is not None


def parallel_threads() -> int:
    return _load_parallel().cpu_parallel_threads()


def parallel_hull(points, threads: int = 0) -> np.ndarray:
    """The multi-core CPU baseline (quadrilateral filter, parallel merge
    sort, Andrew's chain on the oracle's predicates): the same indices as
    hull().  threads = 0 uses every core OpenMP offers."""
    p, dt = _prep(points)
    n = p.shape[0]
    out = np.empty(max(n, 1), dtype=np.int32)
    lib = _load_parallel()
    if lib is None:
        raise RuntimeError("the parallel CPU baseline needs gcc with OpenMP")
    fn = lib.cpu_parallel_hull_i32 if dt == I32 else lib.cpu_parallel_hull_f64
    h = fn(p.ctypes.data, n, out.ctypes.data, int(threads))
    return out[:h].copy()


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB)
            i64, i32p = ctypes.c_int64, ctypes.POINTER(ctypes.c_int32)
            vp = ctypes.c_void_p
            lib.oracle_orient_i32.restype = ctypes.c_int
            lib.oracle_orient_i32.argtypes = [ctypes.c_int32] * 6
            lib.oracle_orient_f64.restype = ctypes.c_int
            lib.oracle_orient_f64.argtypes = [ctypes.c_double] * 6
            lib.oracle_hull_i32.restype = i64
            lib.oracle_hull_i32.argtypes = [vp, i64, vp]
            lib.oracle_hull_f64.restype = i64
            lib.oracle_hull_f64.argtypes = [vp, i64, vp]
            lib.oracle_method.restype = i64
            lib.oracle_method.argtypes = [ctypes.c_int, vp, i64] + [vp] * 8
            del i32p
            _lib = lib
    return _lib


def _prep(points):
    p = np.ascontiguousarray(points)
    if p.ndim != 2 or p.shape[1] != 2:
        raise ValueError("points must have shape [n, 2]")
    if p.dtype == np.int32:
        return p, I32
    if p.dtype == np.float64:
        return p, F64
    raise TypeError(f"unsupported dtype {p.dtype}; use int32 or float64")


def orient(a, b, c, dtype=np.float64) -> int:
    """Exact sign of (b - a) x (c - a): +1 left turn, -1 right turn, 0 collinear."""
    lib = _load()
    if np.dtype(dtype) == np.int32:
        return lib.oracle_orient_i32(int(a[0]), int(a[1]), int(b[0]), int(b[1]),
                                     int(c[0]), int(c[1]))
    return lib.oracle_orient_f64(float(a[0]), float(a[1]), float(b[0]), float(b[1]),
                                 float(c[0]), float(c[1]))


def hull(points) -> np.ndarray:
    """Strict convex hull vertex indices (int32), CCW from the lexicographic
    (x, y) minimum; ties between identical points resolved to the smallest
    index.  n = 0 gives an empty array."""
    p, dt = _prep(points)
    n = p.shape[0]
    out = np.empty(max(n, 1), dtype=np.int32)
    lib = _load()
    fn = lib.oracle_hull_i32 if dt == I32 else lib.oracle_hull_f64
    h = fn(p.ctypes.data, n, out.ctypes.data)
    return out[:h].copy()


def method(points) -> dict:
    """The paper's procedure step by step; returns the intermediates:

    ``ext``      int32[4]  P_minx, P_miny, P_maxx, P_maxy (E1..E4)
    ``region``   int8[n]   0 (interior, R0) or 1..4 (Sec. 2.1.1)
    ``r1``       list of 4 int32 arrays: round-1 survivors per region, index order
    ``sorted``   list of 4 int32 arrays: the same, sorted per Table 1 (stable)
    ``spa``      list of 4 int32 arrays: SPA survivors (Fig. 2), sorted order
    ``hull``     int32[h]  final hull
    """
    p, dt = _prep(points)
    n = p.shape[0]
    m = max(n, 1)
    ext = np.full(4, -1, dtype=np.int32)
    region = np.zeros(m, dtype=np.int8)
    r1 = np.zeros(m, dtype=np.int32)
    r1c = np.zeros(4, dtype=np.int64)
    srt = np.zeros(m, dtype=np.int32)
    spa = np.zeros(m, dtype=np.int32)
    spac = np.zeros(4, dtype=np.int64)
    hl = np.zeros(m, dtype=np.int32)
    lib = _load()
    h = lib.oracle_method(dt, p.ctypes.data, n, ext.ctypes.data, region.ctypes.data,
                          r1.ctypes.data, r1c.ctypes.data, srt.ctypes.data,
                          spa.ctypes.data, spac.ctypes.data, hl.ctypes.data)

    def split(a, c):
        out, o = [], 0
        for k in range(4):
            out.append(a[o:o + int(c[k])].copy())
            o += int(c[k])
        return out

    return {
        "ext": ext,
        "region": region[:n].copy(),
        "r1": split(r1, r1c),
        "sorted": split(srt, r1c),
        "spa": split(spa, spac),
        "hull": hl[:h].copy(),
    }


# ------------------------------------------------- the paper's blocked SPA

def blocked_spa(points, nchunks: int = 1024, m: dict | None = None) -> list:
    """SPA as the paper's GPU implementation runs it (Sec. 2.2.2): one thread
    block of BLOCK_SIZE = 1024 threads per region; thread t checks the
    consecutive points [t L, (t + 1) L) of the region's sorted points,
    L = ceil(m / 1024), with Fig. 2's rule -- a point is discarded when its
    compared coordinate is strictly worse than the running value t, and t
    takes every kept point's value -- restarted at the chunk's first point
    (which is kept).  The region arrays of Sec. 2.2.2 hold the region's
    points only (the extremes are interior, R0), so chunk 0 also starts at
    its own first point.

    Returns a list of 4 int32 arrays: the kept points of R1..R4 in sorted
    (Table 1) order.  Compared coordinates (Fig. 2): R1 keeps y <= t, R2 keeps
    x >= t, R3 keeps y >= t, R4 keeps x <= t; written here as one "smaller is
    better" value v (R1 y, R2 -x, R3 -y, R4 x), a point is kept iff v is at
    most the minimum of v over the earlier points of its chunk.
    ``m`` may pass a precomputed ``method(points)``."""
    p, _ = _prep(points)
    if m is None:
        m = method(points)
    out = []
    for k in range(4):
        s = m["sorted"][k]
        n = len(s)
        if n == 0:
            out.append(np.zeros(0, dtype=np.int32))
            continue
        coord = p[s, 1] if k in (0, 2) else p[s, 0]
        v = -coord if k in (1, 2) else coord
        v = v.astype(np.float64) if p.dtype == np.float64 else v.astype(np.int64)
        L = (n + nchunks - 1) // nchunks
        keep = np.zeros(n, dtype=bool)
        for lo in range(0, n, L):
            c = v[lo:lo + L]
            run = np.minimum.accumulate(c)
            excl = np.concatenate(([c[0]], run[:-1]))     # the first point is its own start value
            keep[lo:lo + L] = c <= excl
        out.append(s[keep].astype(np.int32))
    return out


# ------------------------------------------- round 1 with the octagon

def _f32_views(p):
    """FP32 views of the coordinates, as the octagon mode defines them:
    float64 with the significand truncated to 24 bits (exponent rebiased;
    magnitudes below 2^-126 become zero of their sign), int32 rounded to the
    nearest float.  Written from the IEEE 754 encodings with integer numpy
    operations (float64 values of magnitude below 2^128)."""
    if p.dtype == np.int32:
        return p.astype(np.float32)
    b = np.ascontiguousarray(p, dtype=np.float64).view(np.uint64)
    hi = (b >> np.uint64(32)).astype(np.int64)
    lo = (b & np.uint64(0xFFFFFFFF)).astype(np.int64)
    sign = hi & 0x80000000
    t = (hi & 0x7FFFFFFF) - 0x38000000
    mag = ((t << 3) | (lo >> 29)) & 0x7FFFFFFF
    bits = np.where(t < 0, sign, sign | mag).astype(np.uint32)
    return bits.view(np.float32)


def diag_extremes(points) -> np.ndarray:
    """The diagonal extremes of the octagon mode: per direction the point with
    the smallest FP32 score of its views -- D1 X+Y, D2 Y-X, D3 -(X+Y), D4 X-Y
    (each a single IEEE float32 operation, -0 ordered before +0 as the
    order words do) -- ties to the smallest index.  int32[4]; empty set: -1."""
    p, _ = _prep(points)
    if p.shape[0] == 0:
        return np.full(4, -1, dtype=np.int32)
    v = _f32_views(p)
    X, Y = v[:, 0], v[:, 1]
    with np.errstate(all="ignore"):
        scores = [X + Y, Y - X, -(X + Y), X - Y]
    out = np.zeros(4, dtype=np.int32)
    for k, sc in enumerate(scores):
        u = sc.astype(np.float32).view(np.uint32).astype(np.int64)
        order = np.where(u & 0x80000000, (~u) & 0xFFFFFFFF, u | 0x80000000)   # IEEE order of the bits
        out[k] = int(np.lexsort((np.arange(len(order)), order))[0])
    return out


def octagon_round1(points, diag, m: dict | None = None) -> dict:
    """Round 1 with the octagon: vertices E1 D1 E2 D2 E3 D3 E4 D4, where
    diag[r] is D_r's index (-1: none, the vertex is then E_{r+1}).  A point
    strictly inside the octagon (strictly left of every edge of nonzero
    length, exact orientation) is discarded.  Returns ``r1`` and ``spa``:
    ``method``'s sets without those points (a point strictly inside cannot
    beat, in its region's SPA order, a point that is not, so the SPA
    survivors of the reduced sets are the paper's survivors outside the
    octagon), and the vertex list ``verts``."""
    p, _ = _prep(points)
    if m is None:
        m = method(points)
    E = [int(i) for i in m["ext"]]
    verts = []
    for r in range(4):
        verts.append(E[r])
        verts.append(int(diag[r]) if diag[r] >= 0 else E[(r + 1) % 4])
    pl = p.tolist()
    edges = [(pl[verts[k]], pl[verts[(k + 1) % 8]]) for k in range(8)]
    edges = [(a, b) for a, b in edges if a != b]

    def inside(i):
        q = pl[i]
        return all(orient(a, b, q, p.dtype) > 0 for a, b in edges)

    def keep(arr):
        return np.array([i for i in arr.tolist() if not inside(i)], dtype=np.int32)

    return {"r1": [keep(a) for a in m["r1"]], "spa": [keep(a) for a in m["spa"]], "verts": verts}


def octagon_diag(points, m: dict | None = None) -> np.ndarray:
    """The diagonal extremes the octagon mode uses: D_r of ``diag_extremes``
    when it lies strictly outside the quadrilateral edge E_r -> E_{r+1} (and
    that edge has nonzero length), else -1."""
    p, _ = _prep(points)
    if m is None:
        m = method(points)
    if p.shape[0] == 0:
        return np.full(4, -1, dtype=np.int32)
    d = diag_extremes(points)
    E = [int(i) for i in m["ext"]]
    pl = p.tolist()
    out = np.full(4, -1, dtype=np.int32)
    for r in range(4):
        a, b = pl[E[r]], pl[E[(r + 1) % 4]]
        if a != b and orient(a, b, pl[int(d[r])], p.dtype) < 0:
            out[r] = d[r]
    return out
