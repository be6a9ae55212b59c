"""CPU oracle for the integer convex-hull preconditioner (Cadenas & Megson).

TEST INFRASTRUCTURE ONLY.  Only the tests, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline / reference leg may import this package.  It shares no
code with the CUDA library and never imports it.

``oracle.c`` holds the integer part (Algorithm 1, the Lemma 1 chains and
polyline, Andrew's monotone-chain hull, Melkman's hull of a simple polyline,
Steps 1-2 for points anywhere in int32, an O(m^3) brute-force hull, the
culling-polygon start array).  ``learned.py`` holds the floating-point part of
the learned culling (histogram, MLP forward/backward in float64, extreme
points).  Every function cites the passage of the paper it follows; arrays are
numpy int32 of shape (n, 2) for points and (p, 2) for L.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

ORC_OK = 0
ORC_ERR_ARG = -1
ORC_ERR_RANGE = -2


def build(force: bool = False) -> str:
    """Compile oracle.c into liboracle.so with gcc (no GPU code involved)."""
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    subprocess.check_call(["gcc", "-O2", "-std=gnu11", "-shared", "-fPIC",
                           "-o", tmp, _SRC, "-lm"])
    os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            P = ctypes.c_void_p
            i64, i32 = ctypes.c_int64, ctypes.c_int32
            sigs = {
                "oracle_reduce": (ctypes.c_int, [P, i64, i32, P]),
                "oracle_reduce_from": (ctypes.c_int, [P, i64, i32, P, P]),
                "oracle_chain": (i64, [P, i32, P, P]),
                "oracle_mask": (None, [P, i32, P]),
                "oracle_polyline": (i64, [P, i32, P]),
                "oracle_melkman": (i64, [P, i64, P]),
                "oracle_hull_box": (i64, [P, i64, P]),
                "oracle_reduce_rows": (None, [P, i32, P]),
                "oracle_hull_points": (i64, [P, i64, P]),
                "oracle_hull_chain": (i64, [P, i32, P]),
                "oracle_hull_brute": (i64, [P, i64, P]),
                "oracle_polygon_init": (ctypes.c_int, [P, i32, i32, P]),
                "oracle_chain_from": (None, [P, P, i32, P, P, P]),
                "oracle_best_offsets": (None, [P, i64, ctypes.c_int, ctypes.c_int, ctypes.c_int, P]),
                "oracle_label_batch": (ctypes.c_int, [P, P, P, i64, ctypes.c_int, ctypes.c_int,
                                                      ctypes.c_int, P, P]),
            }
            for name, (res, args) in sigs.items():
                f = getattr(lib, name)
                f.restype = res
                f.argtypes = args
            _lib = lib
    return _lib


def _pts(a) -> np.ndarray:
    a = np.ascontiguousarray(np.asarray(a, dtype=np.int32).reshape(-1, 2))
    return a


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


class OracleRangeError(ValueError):
    """A point lies outside [1, p]^2 (the square of side p, Section 2.1)."""


def reduce(pts, p: int) -> np.ndarray:
    """Algorithm 1 (Reduction of Points), Section 2.1: L of shape (p, 2),
    row x-1 = (min y, max y) over points with that x, else (p+1, -1)."""
    pts = _pts(pts)
    L = np.empty((p, 2), dtype=np.int32)
    rc = _load().oracle_reduce(_ptr(pts), pts.shape[0], p, _ptr(L))
    if rc == ORC_ERR_RANGE:
        raise OracleRangeError("point outside [1,p]^2")
    if rc != ORC_OK:
        raise ValueError(f"oracle_reduce: bad arguments ({rc})")
    return L


def reduce_from(pts, p: int, Linit) -> np.ndarray:
    """Algorithm 1 started from a given array instead of (p+1, -1)."""
    pts = _pts(pts)
    Linit = np.ascontiguousarray(np.asarray(Linit, dtype=np.int32).reshape(p, 2))
    L = np.empty((p, 2), dtype=np.int32)
    rc = _load().oracle_reduce_from(_ptr(pts), pts.shape[0], p, _ptr(Linit), _ptr(L))
    if rc == ORC_ERR_RANGE:
        raise OracleRangeError("point outside [1,p]^2")
    if rc != ORC_OK:
        raise ValueError(f"oracle_reduce_from: bad arguments ({rc})")
    return L


def chain(L) -> tuple[np.ndarray, np.ndarray]:
    """Lemma 1 scan of L: (lower, upper) chains, each (s, 2) int32, the valid
    columns' (x, ly) and (x, hy) in increasing x."""
    L = np.ascontiguousarray(np.asarray(L, dtype=np.int32).reshape(-1, 2))
    p = L.shape[0]
    lo = np.empty((p, 2), dtype=np.int32)
    up = np.empty((p, 2), dtype=np.int32)
    s = _load().oracle_chain(_ptr(L), p, _ptr(lo), _ptr(up))
    return lo[:s].copy(), up[:s].copy()


def chain_points(pts) -> tuple[np.ndarray, np.ndarray]:
    """The Lemma 1 chains straight from the points, for sides too large for
    an array L of p entries: for each distinct x in increasing order,
    (x, min y) and (x, max y) of the points with that x.  The same result as
    chain(reduce(pts, p)) without the O(p) array."""
    pts = _pts(pts)
    if pts.shape[0] == 0:
        e = np.zeros((0, 2), dtype=np.int32)
        return e, e.copy()
    x, y = pts[:, 0].astype(np.int64), pts[:, 1].astype(np.int64)
    o = np.lexsort((y, x))
    x, y = x[o], y[o]
    first = np.ones(x.shape[0], dtype=bool)
    first[1:] = x[1:] != x[:-1]
    last = np.ones(x.shape[0], dtype=bool)
    last[:-1] = x[1:] != x[:-1]
    lo = np.stack([x[first], y[first]], 1).astype(np.int32)
    up = np.stack([x[last], y[last]], 1).astype(np.int32)
    return lo, up


def reduce_rows(L) -> np.ndarray:
    """The second scan along y (Section 2, Fig. 4): Algorithm 1 over the rx
    points of L (its valid (x, ly) and (x, hy)) with x and y exchanged; row
    y-1 of the result = (min x, max x), else (p+1, -1)."""
    L = np.ascontiguousarray(np.asarray(L, dtype=np.int32).reshape(-1, 2))
    p = L.shape[0]
    R = np.empty((p, 2), dtype=np.int32)
    _load().oracle_reduce_rows(_ptr(L), p, _ptr(R))
    return R


def rx_points(L) -> np.ndarray:
    """The reduced set of the scan along x: the Lemma 1 polyline's vertices."""
    return polyline(L)


def rxy_points(R) -> np.ndarray:
    """The reduced set after the second scan: (lo, y) then (hi, y) when they
    differ, for each valid row y in increasing order."""
    R = np.ascontiguousarray(np.asarray(R, dtype=np.int32).reshape(-1, 2))
    q = polyline(R)  # rows play the part of columns
    return np.ascontiguousarray(q[:, ::-1])


def tree_words(p: int, w: int) -> list[int]:
    """Words per level of the w-ary tree of bit words over p columns
    (Section 4, "Extraction using a tree structure"): level 0 has one bit per
    column, each level above one bit per word of the level below, up to a
    single word."""
    words, n = [], p
    while True:
        n = -(-n // w)
        words.append(n)
        if n <= 1:
            return words


def mask(L) -> np.ndarray:
    """Bit array M ("Extraction using an array of bits"): uint32 words,
    column i at bit (i-1)&31 of word (i-1)>>5."""
    L = np.ascontiguousarray(np.asarray(L, dtype=np.int32).reshape(-1, 2))
    p = L.shape[0]
    M = np.empty(((p + 31) // 32,), dtype=np.uint32)
    _load().oracle_mask(_ptr(L), p, _ptr(M))
    return M


def polyline(L) -> np.ndarray:
    """Lemma 1 polygonal chain over the valid entries of L."""
    L = np.ascontiguousarray(np.asarray(L, dtype=np.int32).reshape(-1, 2))
    p = L.shape[0]
    out = np.empty((2 * p + 1, 2), dtype=np.int32)
    s = _load().oracle_polyline(_ptr(L), p, _ptr(out))
    return out[:s].copy()


def hull_points(pts) -> np.ndarray:
    """Strict hull vertices of the point set (sort + Andrew), CCW from the
    lexicographic minimum."""
    pts = _pts(pts)
    n = pts.shape[0]
    out = np.empty((max(2 * n, 2), 2), dtype=np.int32)
    h = _load().oracle_hull_points(_ptr(pts), n, _ptr(out))
    return out[:h].copy()


def hull_chain(L) -> np.ndarray:
    """Hull of the reduced set, Andrew's scan run on the Lemma 1 polyline
    (already ordered: no sort)."""
    L = np.ascontiguousarray(np.asarray(L, dtype=np.int32).reshape(-1, 2))
    p = L.shape[0]
    out = np.empty((2 * p + 2, 2), dtype=np.int32)
    h = _load().oracle_hull_chain(_ptr(L), p, _ptr(out))
    return out[:h].copy()


def melkman(poly) -> np.ndarray:
    """Melkman's on-line hull of a simple polyline (the hull algorithm of
    Section 3, Fig. 10), strict vertices CCW from the lexicographic minimum.
    The vertices must be distinct and the polyline simple; the Lemma 1
    polyline is."""
    poly = _pts(poly)
    m = poly.shape[0]
    out = np.empty((max(m, 1) + 1, 2), dtype=np.int32)
    h = _load().oracle_melkman(_ptr(poly), m, _ptr(out))
    return out[:h].copy()


def hull_box(pts) -> np.ndarray:
    """Steps 1-2 of the general procedure (Section 2): bounding box,
    translation into it, Algorithm 1 with the columns along the shorter side,
    the hull of the reduced set, mapped back.  Points anywhere in int32."""
    pts = _pts(pts)
    n = pts.shape[0]
    if n == 0:
        return np.empty((0, 2), dtype=np.int32)
    side = int(min(int(pts[:, 0].max()) - int(pts[:, 0].min()),
                   int(pts[:, 1].max()) - int(pts[:, 1].min()))) + 1
    out = np.empty((2 * side + 2, 2), dtype=np.int32)
    h = _load().oracle_hull_box(_ptr(pts), n, _ptr(out))
    if h < 0:
        raise ValueError("oracle_hull_box: a side of the box exceeds 2^30")
    return out[:h].copy()


def hull_brute(pts) -> np.ndarray:
    """O(m^3) hull from the definition of a hull edge (small inputs)."""
    pts = _pts(pts)
    n = pts.shape[0]
    out = np.empty((max(n, 1) + 1, 2), dtype=np.int32)
    h = _load().oracle_hull_brute(_ptr(pts), n, _ptr(out))
    return out[:h].copy()


def hull(pts, p: int) -> np.ndarray:
    """The whole path: Algorithm 1, then the hull of the reduced set."""
    return hull_chain(reduce(pts, p))


def polygon_init(poly, p: int) -> np.ndarray:
    """Start array for Algorithm 1 from a convex culling polygon (strict
    vertices, CCW from the lexicographic minimum): column x in the polygon's
    x-range starts at (floor(b(x))+1, ceil(u(x))-1), other columns at
    (p+1, -1)."""
    poly = _pts(poly)
    Linit = np.empty((p, 2), dtype=np.int32)
    _load().oracle_polygon_init(_ptr(poly), poly.shape[0], p, _ptr(Linit))
    return Linit


def chain_from(L, Linit) -> tuple[np.ndarray, np.ndarray]:
    """Chains of a culled reduction: a lower point where ly fell below its
    start value, an upper point where hy rose above it."""
    L = np.ascontiguousarray(np.asarray(L, dtype=np.int32).reshape(-1, 2))
    Linit = np.ascontiguousarray(np.asarray(Linit, dtype=np.int32).reshape(-1, 2))
    p = L.shape[0]
    lo = np.empty((p, 2), dtype=np.int32)
    up = np.empty((p, 2), dtype=np.int32)
    cnt = np.zeros(2, dtype=np.int64)
    _load().oracle_chain_from(_ptr(L), _ptr(Linit), p, _ptr(lo), _ptr(up), _ptr(cnt))
    return lo[:cnt[0]].copy(), up[:cnt[1]].copy()


def best_offsets(H, K: int = 16, sub: int = 9, rounds: int = 2) -> np.ndarray:
    """Training label of the learned culling proposal (not in the paper): per
    sector of directions, the offset (units of pi/K from the sector centre)
    whose extreme hull vertex maximises the area of the polygon of the K
    extreme vertices (coordinate ascent over `sub` candidates per sector)."""
    H = _pts(H)
    out = np.zeros(K, dtype=np.float32)
    _load().oracle_best_offsets(_ptr(H), H.shape[0], K, sub, rounds, _ptr(out))
    return out


def label_batch(pts, offsets, ps, K: int = 16, sub: int = 9, rounds: int = 2):
    """Labels (B, K) float32 and oracle hull sizes (B,) of a ragged batch."""
    pts = _pts(pts)
    off = np.ascontiguousarray(np.asarray(offsets, dtype=np.int64))
    pp = np.ascontiguousarray(np.asarray(ps, dtype=np.int32))
    B = pp.shape[0]
    out = np.zeros((B, K), dtype=np.float32)
    hs = np.zeros(B, dtype=np.int64)
    rc = _load().oracle_label_batch(_ptr(pts), _ptr(off), _ptr(pp), B, K, sub, rounds, _ptr(out),
                                    _ptr(hs))
    if rc == ORC_ERR_RANGE:
        raise OracleRangeError("point outside [1,p]^2")
    return out, hs
