"""Thin ctypes binding of libch.so (C ABI in include/ch.h).

Argument marshalling only: every step of the hull path runs in the library's
CUDA kernels.  PyTorch supplies device memory and the current CUDA stream.
The functions keep the C names; outputs and workspaces the caller does not
pass are allocated here with torch (the C calls never allocate).

Importing this module does not touch the GPU.  The first call loads
libch.so and raises ``RuntimeError`` if it cannot (no silent fallback).
"""
from __future__ import annotations

import ctypes
import os
import threading

import torch

from . import _build

CH_OK = 0
CH_ERR_ARG = -1
CH_ERR_RANGE = -2
CH_ERR_CAPACITY = -3
CH_ERR_TIMEOUT = -4
CH_ERR_CUDA = -5
CH_ERR_WORKSPACE = -6

_lock = threading.Lock()
_lib = None


class ChError(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = code
        super().__init__(f"{where}: {strerror(code)} ({code})")


def _declare(lib):
    P, i32, i64, sz = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_size_t
    szp = ctypes.POINTER(ctypes.c_size_t)
    sigs = {
        "ch_strerror": (ctypes.c_char_p, [ctypes.c_int]),
        "ch_version": (ctypes.c_int, []),
        "ch_sync_status": (ctypes.c_int, [P]),
        "ch_clear_status": (ctypes.c_int, [P]),
        "ch_trace_set": (ctypes.c_int, [ctypes.POINTER(ctypes.c_void_p), ctypes.c_int]),
        "ch_plan_info": (ctypes.c_int, [i64, i32, ctypes.POINTER(i32), ctypes.POINTER(i32)]),
        "ch_batched_workspace_size": (ctypes.c_int, [i32, P, P, i32, szp]),
        "ch_batched_prepare": (ctypes.c_int, [i32, P, P, i32, P, sz, P]),
        "ch_batched_prepare_shape": (ctypes.c_int, [i32, P, P, i32, i32, P, sz, P]),
        "ch_hull_batched": (ctypes.c_int, [P, P, P, i32, P, P, P, P, sz, P]),
        "ch_reduce_batched": (ctypes.c_int, [P, P, P, i32, P, P, P, sz, P]),
        "ch_chain_batched": (ctypes.c_int, [P, P, P, i32, P, P, P, P]),
        "ch_reduce_workspace_size": (ctypes.c_int, [i64, i32, szp]),
        "ch_reduce": (ctypes.c_int, [P, i64, i32, P, P, sz, P]),
        "ch_chain_workspace_size": (ctypes.c_int, [i32, szp]),
        "ch_chain": (ctypes.c_int, [P, i32, P, P, P, P, P, sz, P]),
        "ch_hull_workspace_size": (ctypes.c_int, [i32, szp]),
        "ch_hull": (ctypes.c_int, [P, P, P, i32, P, P, P, sz, P]),
        "ch_convex_hull_workspace_size": (ctypes.c_int, [i64, i32, szp]),
        "ch_convex_hull": (ctypes.c_int, [P, i64, i32, P, P, P, P, P, P, P, sz, P]),
        "ch_convex_hull_host_workspace_size": (ctypes.c_int, [i64, i32, szp]),
        "ch_convex_hull_host": (ctypes.c_int, [P, i64, i32, P, ctypes.POINTER(ctypes.c_int32), P, sz, P]),
        "ch_mlp_forward": (ctypes.c_int, [P, P, i32, P, P, P, P]),
        "ch_mlp_loss": (ctypes.c_int, [P, P, i32, P, P, P]),
        "ch_mlp_backward_workspace_size": (ctypes.c_int, [i32, szp]),
        "ch_mlp_backward": (ctypes.c_int, [P, P, P, P, P, i32, P, P, sz, P]),
        "ch_mlp_adam": (ctypes.c_int, [P, P, P, P, i32, ctypes.c_float, ctypes.c_float,
                                       ctypes.c_float, ctypes.c_float, P]),
        "ch_chain_noalloc": (ctypes.c_int, [P, i32, P, P, P, P, P]),
        "ch_bbox_workspace_size": (ctypes.c_int, [szp]),
        "ch_bbox": (ctypes.c_int, [P, i64, P, P, sz, P]),
        "ch_convex_hull_box_workspace_size": (ctypes.c_int, [i64, P, szp]),
        "ch_convex_hull_box": (ctypes.c_int, [P, i64, P, P, P, P, sz, P]),
        "ch_cull_workspace_size": (ctypes.c_int, [i32, szp]),
        "ch_cull_propose": (ctypes.c_int, [P, i64, i32, P, P, P, P, P, P, P, P, P, P, sz, P]),
        "ch_hull_learned_workspace_size": (ctypes.c_int, [i64, i32, szp]),
        "ch_hull_learned_kernel_count": (ctypes.c_int, [i64, i32, i32, ctypes.POINTER(i32)]),
        "ch_hull_learned": (ctypes.c_int, [P, i64, i32, P, P, P, P, P, P, P, P, P, P, sz, P]),
        "ch_polyline_workspace_size": (ctypes.c_int, [i32, szp]),
        "ch_polyline": (ctypes.c_int, [P, i32, P, P, P, sz, P]),
        "ch_hull_melkman_workspace_size": (ctypes.c_int, [i32, szp]),
        "ch_hull_melkman": (ctypes.c_int, [P, P, i32, P, P, P, sz, P]),
        "ch_convex_hull_melkman_workspace_size": (ctypes.c_int, [i64, i32, szp]),
        "ch_convex_hull_melkman": (ctypes.c_int, [P, i64, i32, P, P, P, P, P, P, sz, P]),
        "ch_sparse_workspace_size": (ctypes.c_int, [i64, i32, szp, szp]),
        "ch_sparse_kernel_count": (ctypes.c_int, [i64, i32, ctypes.POINTER(i32)]),
        "ch_convex_hull_sparse": (ctypes.c_int, [P, i64, i32, P, P, P, P, P, P, sz, P]),
        "ch_reduce_rows": (ctypes.c_int, [P, i32, P, P]),
        "ch_reduce_u16": (ctypes.c_int, [P, i64, i32, P, P, sz, P]),
        "ch_convex_hull_u16": (ctypes.c_int, [P, i64, i32, P, P, P, P, P, P, P, sz, P]),
        "ch_convex_hull_rxy_workspace_size": (ctypes.c_int, [i64, i32, szp]),
        "ch_convex_hull_rxy": (ctypes.c_int, [P, i64, i32, P, P, P, P, P, sz, P]),
    }
    for name, (res, args) in sigs.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    return lib


def library_path() -> str:
    return _build.LIB


def lib():
    """The loaded libch.so (built first if absent)."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.LIB
            if not os.path.exists(path):
                path = _build.build()
            try:
                _lib = _declare(ctypes.CDLL(path))
            except OSError as e:
                raise RuntimeError(f"libch.so could not be loaded from {path}: {e}") from e
    return _lib


def strerror(code: int) -> str:
    return lib().ch_strerror(int(code)).decode()


def _check(rc: int, where: str):
    if rc != CH_OK:
        raise ChError(rc, where)


def _ptr(t):
    """Device pointer of a CUDA tensor (None -> NULL); a host tensor is an
    error, so host memory never reaches a kernel through a device argument."""
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError("device arguments must be CUDA tensors")
    return ctypes.c_void_p(t.data_ptr())


def _host_ptr(t):
    """Pointer of a CPU tensor, for the host arguments of ch_convex_hull_host."""
    if t.is_cuda:
        raise ValueError("host arguments must be CPU tensors")
    return ctypes.c_void_p(t.data_ptr())


def _stream(stream):
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _dev(t):
    if not t.is_cuda:
        raise ValueError("expected a CUDA tensor")
    return t.device


def _size(fn, *args) -> int:
    out = ctypes.c_size_t(0)
    _check(fn(*args, ctypes.byref(out)), fn.__name__)
    return int(out.value)


def _ws(nbytes: int, device, ws):
    if ws is not None:
        if ws.numel() * ws.element_size() < nbytes:
            raise ChError(CH_ERR_WORKSPACE, "workspace")
        return ws
    return torch.empty(max(nbytes, 1), dtype=torch.uint8, device=device)


def _pts(pts):
    if (not pts.is_cuda or pts.dtype != torch.int32 or pts.dim() != 2 or pts.shape[1] != 2
            or not pts.is_contiguous()):
        raise ValueError("points must be a contiguous int32 CUDA tensor of shape (n, 2)")
    return pts


def ch_sync_status(stream=None) -> int:
    """Status of the calls made on `stream` (default: torch's current stream)
    since its last read; waits for that stream and clears its word."""
    return int(lib().ch_sync_status(_stream(stream)))


def ch_clear_status(stream=None):
    _check(lib().ch_clear_status(_stream(stream)), "ch_clear_status")


def ch_trace_set(events):
    """Profiling aid: a list of (start, end) torch.cuda.Event pairs (timing
    enabled, already recorded once so their handles exist); every reduction
    kernel launched afterwards is bracketed by the next pair.  [] turns it off."""
    flat = [e.cuda_event for pair in events for e in pair]
    arr = (ctypes.c_void_p * max(1, len(flat)))(*flat)
    _check(lib().ch_trace_set(arr, len(events)), "ch_trace_set")


def ch_plan_info(n: int, p: int):
    """(form, kernels): how ch_convex_hull runs n points of side p on the
    current device, and how many kernels one call launches."""
    form, kern = ctypes.c_int32(0), ctypes.c_int32(0)
    _check(lib().ch_plan_info(int(n), int(p), ctypes.byref(form), ctypes.byref(kern)), "ch_plan_info")
    return int(form.value), int(kern.value)


def ch_reduce_workspace_size(n: int, p: int) -> int:
    return _size(lib().ch_reduce_workspace_size, int(n), int(p))


def ch_reduce(pts, p: int, L=None, workspace=None, stream=None):
    """Algorithm 1: returns L (p, 2) int32 on the points' device."""
    pts = _pts(pts)
    dev = _dev(pts)
    n = pts.shape[0]
    if L is None:
        L = torch.empty((p, 2), dtype=torch.int32, device=dev)
    ws = _ws(ch_reduce_workspace_size(n, p), dev, workspace)
    _check(lib().ch_reduce(_ptr(pts), n, int(p), _ptr(L), _ptr(ws), ws.numel(), _stream(stream)),
           "ch_reduce")
    return L


def ch_chain_workspace_size(p: int) -> int:
    return _size(lib().ch_chain_workspace_size, int(p))


def _check_chain_args(L, p, lower, upper, counts, mask):
    """The chain step's arrays: contiguous int32 CUDA tensors, L with at least
    p rows of 2, lower and upper with room for p rows of 2, counts for 2
    values and mask (when given) for ceil(p / 32) words; ValueError else."""
    need = (("L", L, 2 * p), ("lower", lower, 2 * p), ("upper", upper, 2 * p),
            ("counts", counts, 2), ("mask", mask, (p + 31) // 32))
    for name, t, k in need:
        if t is None:
            if name != "mask":
                raise ValueError(f"{name} is required")
            continue
        if not t.is_cuda or t.dtype != torch.int32 or not t.is_contiguous():
            raise ValueError(f"{name} must be a contiguous int32 CUDA tensor")
        if t.numel() < k:
            raise ValueError(f"{name} holds {t.numel()} int32 values, {k} needed for p = {p}")


def ch_chain(L, p: int | None = None, lower=None, upper=None, counts=None, mask=None,
             workspace=None, stream=None, with_mask: bool = False):
    """Lemma 1 chains of L: returns (lower, upper, counts[, mask]); lower and
    upper have capacity p rows, the first counts[0] of which are valid."""
    dev = _dev(L)
    p = int(L.shape[0] if p is None else p)
    if lower is None:
        lower = torch.empty((p, 2), dtype=torch.int32, device=dev)
    if upper is None:
        upper = torch.empty((p, 2), dtype=torch.int32, device=dev)
    if counts is None:
        counts = torch.empty(2, dtype=torch.int32, device=dev)
    if with_mask and mask is None:
        mask = torch.empty(((p + 31) // 32,), dtype=torch.int32, device=dev)
    if p >= 1:
        _check_chain_args(L, p, lower, upper, counts, mask)
    ws = _ws(ch_chain_workspace_size(p), dev, workspace)
    _check(lib().ch_chain(_ptr(L), p, _ptr(lower), _ptr(upper), _ptr(counts), _ptr(mask),
                          _ptr(ws), ws.numel(), _stream(stream)), "ch_chain")
    if mask is not None:
        return lower, upper, counts, mask
    return lower, upper, counts


CH_CHAIN_NOALLOC_MAX_P = 1 << 24  # the header's #define of the same name


def ch_chain_noalloc(L, p: int, lower, upper, counts, mask=None, stream=None):
    """ch_chain with the library's own fixed scratch (no workspace, no
    allocation in the call); outputs are the caller's tensors.  p above
    CH_CHAIN_NOALLOC_MAX_P is refused by the library (CH_ERR_CAPACITY)
    before any array is touched."""
    if 1 <= int(p) <= CH_CHAIN_NOALLOC_MAX_P:
        _check_chain_args(L, int(p), lower, upper, counts, mask)
    _check(lib().ch_chain_noalloc(_ptr(L), int(p), _ptr(lower), _ptr(upper), _ptr(counts),
                                  _ptr(mask), _stream(stream)), "ch_chain_noalloc")


def ch_hull_workspace_size(p: int) -> int:
    return _size(lib().ch_hull_workspace_size, int(p))


def ch_hull(lower, upper, counts, p: int, hull=None, hull_count=None, workspace=None,
            stream=None):
    """Strict hull of the chains: returns (hull (2p, 2) capacity, hull_count (1,))."""
    dev = _dev(lower)
    if hull is None:
        hull = torch.empty((2 * p, 2), dtype=torch.int32, device=dev)
    if hull_count is None:
        hull_count = torch.empty(1, dtype=torch.int32, device=dev)
    ws = _ws(ch_hull_workspace_size(p), dev, workspace)
    _check(lib().ch_hull(_ptr(lower), _ptr(upper), _ptr(counts), int(p), _ptr(hull),
                         _ptr(hull_count), _ptr(ws), ws.numel(), _stream(stream)), "ch_hull")
    return hull, hull_count


def ch_convex_hull_workspace_size(n: int, p: int) -> int:
    return _size(lib().ch_convex_hull_workspace_size, int(n), int(p))


def ch_convex_hull(pts, p: int, L=None, lower=None, upper=None, counts=None, hull=None,
                   hull_count=None, workspace=None, stream=None):
    """All three steps; returns (hull, hull_count).  L/lower/upper/counts are
    written when given (else kept in the workspace)."""
    pts = _pts(pts)
    dev = _dev(pts)
    n = pts.shape[0]
    if hull is None:
        hull = torch.empty((2 * p, 2), dtype=torch.int32, device=dev)
    if hull_count is None:
        hull_count = torch.empty(1, dtype=torch.int32, device=dev)
    ws = _ws(ch_convex_hull_workspace_size(n, p), dev, workspace)
    _check(lib().ch_convex_hull(_ptr(pts), n, int(p), _ptr(L), _ptr(lower), _ptr(upper),
                                _ptr(counts), _ptr(hull), _ptr(hull_count), _ptr(ws), ws.numel(),
                                _stream(stream)), "ch_convex_hull")
    return hull, hull_count


def pack_u16(pts):
    """int32 (n, 2) points in [1, 65536]^2 -> the packed 16-bit format of
    ch_convex_hull_u16: one int32 word (x - 1) | (y - 1) << 16 per point
    (a view of little-endian uint16 pairs (x - 1, y - 1))."""
    x = (pts[:, 0] - 1).to(torch.int32)
    y = (pts[:, 1] - 1).to(torch.int32)
    return ((y << 16) | (x & 0xFFFF)).contiguous()


def _pts16(pts):
    if not pts.is_cuda or pts.dtype != torch.int32 or pts.dim() != 1 or not pts.is_contiguous():
        raise ValueError("packed points must be a contiguous int32 CUDA tensor of shape (n,)")
    return pts


def ch_reduce_u16(pts, p: int, L=None, workspace=None, stream=None):
    """Algorithm 1 on packed 16-bit points (see pack_u16): L (p, 2)."""
    pts = _pts16(pts)
    dev = _dev(pts)
    if L is None:
        L = torch.empty((p, 2), dtype=torch.int32, device=dev)
    ws = _ws(ch_reduce_workspace_size(pts.shape[0], p), dev, workspace)
    _check(lib().ch_reduce_u16(_ptr(pts), pts.shape[0], int(p), _ptr(L), _ptr(ws), ws.numel(),
                               _stream(stream)), "ch_reduce_u16")
    return L


def ch_convex_hull_u16(pts, p: int, L=None, lower=None, upper=None, counts=None, hull=None,
                       hull_count=None, workspace=None, stream=None):
    """The fused path on packed 16-bit points; returns (hull, hull_count)."""
    pts = _pts16(pts)
    dev = _dev(pts)
    if hull is None:
        hull = torch.empty((2 * p, 2), dtype=torch.int32, device=dev)
    if hull_count is None:
        hull_count = torch.empty(1, dtype=torch.int32, device=dev)
    ws = _ws(ch_convex_hull_workspace_size(pts.shape[0], p), dev, workspace)
    _check(lib().ch_convex_hull_u16(_ptr(pts), pts.shape[0], int(p), _ptr(L), _ptr(lower),
                                    _ptr(upper), _ptr(counts), _ptr(hull), _ptr(hull_count),
                                    _ptr(ws), ws.numel(), _stream(stream)), "ch_convex_hull_u16")
    return hull, hull_count


def ch_convex_hull_host_workspace_size(n: int, p: int) -> int:
    return _size(lib().ch_convex_hull_host_workspace_size, int(n), int(p))


def ch_convex_hull_host(host_pts, p: int, workspace, stream=None, host_hull=None):
    """End to end from host memory (a CPU int32 (n, 2) tensor, pinned for
    speed): returns the hull as a CPU int32 (h, 2) tensor."""
    if host_pts.is_cuda or host_pts.dtype != torch.int32 or not host_pts.is_contiguous():
        raise ValueError("host_pts must be a contiguous CPU int32 tensor of shape (n, 2)")
    n = host_pts.shape[0]
    if host_hull is None:
        host_hull = torch.empty((2 * p, 2), dtype=torch.int32)
    cnt = ctypes.c_int32(0)
    _check(lib().ch_convex_hull_host(_host_ptr(host_pts), n, int(p), _host_ptr(host_hull),
                                     ctypes.byref(cnt), _ptr(workspace), workspace.numel(),
                                     _stream(stream)), "ch_convex_hull_host")
    return host_hull[: cnt.value]


# ------------------------------------------------------------------ batched


def ch_polyline_workspace_size(p: int) -> int:
    return _size(lib().ch_polyline_workspace_size, int(p))


def ch_polyline(L, p: int | None = None, poly=None, count=None, workspace=None, stream=None):
    """Lemma 1 polyline of L: returns (poly, count); poly has capacity 2p
    rows, the first count[0] of which are the vertices."""
    dev = _dev(L)
    p = int(L.shape[0] if p is None else p)
    if poly is None:
        poly = torch.empty((2 * p, 2), dtype=torch.int32, device=dev)
    if count is None:
        count = torch.empty(1, dtype=torch.int32, device=dev)
    ws = _ws(ch_polyline_workspace_size(p), dev, workspace)
    _check(lib().ch_polyline(_ptr(L), p, _ptr(poly), _ptr(count), _ptr(ws), ws.numel(),
                             _stream(stream)), "ch_polyline")
    return poly, count


def ch_hull_melkman_workspace_size(p: int) -> int:
    return _size(lib().ch_hull_melkman_workspace_size, int(p))


def ch_hull_melkman(poly, count, p: int, hull=None, hull_count=None, workspace=None, stream=None):
    """Melkman's hull of the simple polyline poly[:count[0]] (count: device
    int32 tensor); returns (hull, hull_count)."""
    dev = _dev(poly)
    if hull is None:
        hull = torch.empty((max(2 * int(p), 2), 2), dtype=torch.int32, device=dev)
    if hull_count is None:
        hull_count = torch.empty(1, dtype=torch.int32, device=dev)
    need = ch_hull_melkman_workspace_size(p)
    ws = _ws(need, dev, workspace) if need or workspace is not None else None
    _check(lib().ch_hull_melkman(_ptr(poly), _ptr(count), int(p), _ptr(hull), _ptr(hull_count),
                                 _ptr(ws), 0 if ws is None else ws.numel(), _stream(stream)),
           "ch_hull_melkman")
    return hull, hull_count


def ch_convex_hull_melkman_workspace_size(n: int, p: int) -> int:
    return _size(lib().ch_convex_hull_melkman_workspace_size, int(n), int(p))


def ch_convex_hull_melkman(pts, p: int, L=None, poly=None, poly_count=None, hull=None,
                           hull_count=None, workspace=None, stream=None):
    """Algorithm 1, the Lemma 1 polyline and Melkman's hull in one call;
    returns (hull, hull_count)."""
    pts = _pts(pts)
    dev = _dev(pts)
    if hull is None:
        hull = torch.empty((2 * p, 2), dtype=torch.int32, device=dev)
    if hull_count is None:
        hull_count = torch.empty(1, dtype=torch.int32, device=dev)
    ws = _ws(ch_convex_hull_melkman_workspace_size(pts.shape[0], p), dev, workspace)
    _check(lib().ch_convex_hull_melkman(_ptr(pts), pts.shape[0], int(p), _ptr(L), _ptr(poly),
                                        _ptr(poly_count), _ptr(hull), _ptr(hull_count), _ptr(ws),
                                        ws.numel(), _stream(stream)), "ch_convex_hull_melkman")
    return hull, hull_count


def ch_sparse_workspace_size(n: int, p: int):
    """(bytes, persistent_bytes) of the sparse path's workspace: the leading
    persistent_bytes must be zero before the first call and stay zero after
    each call that records no error."""
    a, b = ctypes.c_size_t(0), ctypes.c_size_t(0)
    _check(lib().ch_sparse_workspace_size(int(n), int(p), ctypes.byref(a), ctypes.byref(b)),
           "ch_sparse_workspace_size")
    return int(a.value), int(b.value)


def ch_sparse_kernel_count(n: int, p: int) -> int:
    k = ctypes.c_int32(0)
    _check(lib().ch_sparse_kernel_count(int(n), int(p), ctypes.byref(k)), "ch_sparse_kernel_count")
    return int(k.value)


def ch_sparse_workspace(n: int, p: int, device="cuda"):
    """A zero-filled workspace for ch_convex_hull_sparse."""
    nbytes, _ = ch_sparse_workspace_size(n, p)
    return torch.zeros(max(nbytes, 1), dtype=torch.uint8, device=device)


def ch_convex_hull_sparse(pts, p: int, workspace, lower=None, upper=None, counts=None, hull=None,
                          hull_count=None, stream=None):
    """The path through the tree of bit words (sparse regime p > n); the
    workspace comes from ch_sparse_workspace and is reused across calls.
    Returns (hull, hull_count)."""
    pts = _pts(pts)
    dev = _dev(pts)
    n = pts.shape[0]
    if hull is None:
        hull = torch.empty((max(2 * min(p, max(n, 1)), 2), 2), dtype=torch.int32, device=dev)
    if hull_count is None:
        hull_count = torch.empty(1, dtype=torch.int32, device=dev)
    need, _ = ch_sparse_workspace_size(n, p)
    if workspace.numel() * workspace.element_size() < need:
        raise ChError(CH_ERR_WORKSPACE, "ch_convex_hull_sparse")
    _check(lib().ch_convex_hull_sparse(_ptr(pts), n, int(p), _ptr(lower), _ptr(upper), _ptr(counts),
                                       _ptr(hull), _ptr(hull_count), _ptr(workspace),
                                       workspace.numel(), _stream(stream)), "ch_convex_hull_sparse")
    return hull, hull_count


def ch_reduce_rows(L, p: int | None = None, R=None, stream=None):
    """The second scan along y over the rx points of L: R (p, 2)."""
    dev = _dev(L)
    p = int(L.shape[0] if p is None else p)
    if R is None:
        R = torch.empty((p, 2), dtype=torch.int32, device=dev)
    _check(lib().ch_reduce_rows(_ptr(L), p, _ptr(R), _stream(stream)), "ch_reduce_rows")
    return R


def ch_convex_hull_rxy_workspace_size(n: int, p: int) -> int:
    return _size(lib().ch_convex_hull_rxy_workspace_size, int(n), int(p))


def ch_convex_hull_rxy(pts, p: int, L=None, R=None, hull=None, hull_count=None, workspace=None,
                       stream=None):
    """Algorithm 1 along x, the second scan along y, the hull of the rxy
    points; returns (hull, hull_count)."""
    pts = _pts(pts)
    dev = _dev(pts)
    if hull is None:
        hull = torch.empty((2 * p, 2), dtype=torch.int32, device=dev)
    if hull_count is None:
        hull_count = torch.empty(1, dtype=torch.int32, device=dev)
    ws = _ws(ch_convex_hull_rxy_workspace_size(pts.shape[0], p), dev, workspace)
    _check(lib().ch_convex_hull_rxy(_ptr(pts), pts.shape[0], int(p), _ptr(L), _ptr(R), _ptr(hull),
                                    _ptr(hull_count), _ptr(ws), ws.numel(), _stream(stream)),
           "ch_convex_hull_rxy")
    return hull, hull_count


def _host_sizes(offsets, ps):
    import numpy as np
    off = np.ascontiguousarray(np.asarray(offsets, dtype=np.int64))
    pp = np.ascontiguousarray(np.asarray(ps, dtype=np.int32))
    return off, pp


def ch_batched_workspace_size(offsets, ps, chunk_mult: int = 64) -> int:
    off, pp = _host_sizes(offsets, ps)
    out = ctypes.c_size_t(0)
    _check(lib().ch_batched_workspace_size(pp.shape[0], off.ctypes.data_as(ctypes.c_void_p),
                                           pp.ctypes.data_as(ctypes.c_void_p), int(chunk_mult),
                                           ctypes.byref(out)), "ch_batched_workspace_size")
    return int(out.value)


CH_BATCH_FOLD_DEFAULT = 512  # the header's #define of the same name
CH_BATCH_FOLD_SHAPES = (0, 384, 512, 640, 768, 896)


def ch_batched_prepare(offsets, ps, workspace, chunk_mult: int = 64, stream=None,
                       fold_threads: int | None = None):
    """Plan the batch (host arrays offsets (B+1,), ps (B,)) into `workspace`;
    fold_threads (None: the library's default) picks the CTA shape, see
    ch_batched_prepare_shape in include/ch.h."""
    off, pp = _host_sizes(offsets, ps)
    if fold_threads is None:
        _check(lib().ch_batched_prepare(pp.shape[0], off.ctypes.data_as(ctypes.c_void_p),
                                        pp.ctypes.data_as(ctypes.c_void_p), int(chunk_mult),
                                        _ptr(workspace), workspace.numel(), _stream(stream)),
               "ch_batched_prepare")
    else:
        _check(lib().ch_batched_prepare_shape(pp.shape[0], off.ctypes.data_as(ctypes.c_void_p),
                                              pp.ctypes.data_as(ctypes.c_void_p), int(chunk_mult),
                                              int(fold_threads), _ptr(workspace),
                                              workspace.numel(), _stream(stream)),
               "ch_batched_prepare_shape")


def ch_hull_batched(pts, offsets, ps, hull_out, hull_offsets, hull_counts, workspace,
                    stream=None):
    """Hulls of all sets of the prepared batch (device tensors)."""
    pts = _pts(pts)
    B = int(ps.shape[0])
    _check(lib().ch_hull_batched(_ptr(pts), _ptr(offsets), _ptr(ps), B, _ptr(hull_out),
                                 _ptr(hull_offsets), _ptr(hull_counts), _ptr(workspace),
                                 workspace.numel(), _stream(stream)), "ch_hull_batched")
    return hull_out, hull_counts


def ch_reduce_batched(pts, offsets, ps, L_out, L_offsets, workspace, stream=None):
    """Algorithm 1 for all sets of the prepared batch: set s writes its L
    (ps[s] int32 pairs) at L_out[L_offsets[s]] (device tensors)."""
    pts = _pts(pts)
    B = int(ps.shape[0])
    _check(lib().ch_reduce_batched(_ptr(pts), _ptr(offsets), _ptr(ps), B, _ptr(L_out),
                                   _ptr(L_offsets), _ptr(workspace), workspace.numel(),
                                   _stream(stream)), "ch_reduce_batched")
    return L_out


def ch_chain_batched(L, L_offsets, ps, lower, upper, counts, stream=None):
    """Lemma 1 chains of all sets from their L (layout of ch_reduce_batched);
    counts: int32 (B, 2)."""
    B = int(ps.shape[0])
    _check(lib().ch_chain_batched(_ptr(L), _ptr(L_offsets), _ptr(ps), B, _ptr(lower), _ptr(upper),
                                  _ptr(counts), _stream(stream)), "ch_chain_batched")
    return lower, upper, counts


def L_offsets_of(ps):
    """int64 (B+1,) offsets giving set s ps[s] pairs (the layout of L and of
    the chains in the batched reduce and chain calls)."""
    import numpy as np
    pp = np.asarray(ps.cpu() if hasattr(ps, "cpu") else ps, dtype=np.int64)
    out = np.zeros(pp.shape[0] + 1, dtype=np.int64)
    np.cumsum(pp, out=out[1:])
    return out


def hull_capacity_offsets(offsets, ps):
    """int64 (B+1,) output offsets giving each set min(n, 2p) pairs."""
    import numpy as np
    off, pp = _host_sizes(offsets, ps)
    cap = np.minimum(np.diff(off), 2 * pp.astype(np.int64))
    out = np.zeros(pp.shape[0] + 1, dtype=np.int64)
    np.cumsum(cap, out=out[1:])
    return out


# ---------------------------------------------------------------- MLP
CH_MLP_IN, CH_MLP_HID, CH_MLP_K = 1024, 256, 16
CH_MLP_PARAMS = CH_MLP_IN * CH_MLP_HID + CH_MLP_HID + CH_MLP_HID * CH_MLP_HID + CH_MLP_HID \
    + CH_MLP_HID * CH_MLP_K + CH_MLP_K


def _f32(t, shape=None, name="tensor"):
    if t.dtype != torch.float32 or not t.is_contiguous() or not t.is_cuda:
        raise ValueError(f"{name} must be a contiguous float32 CUDA tensor")
    if shape is not None and tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name} must have shape {tuple(shape)}, got {tuple(t.shape)}")
    return t


def ch_mlp_forward(params, X, H1=None, H2=None, Y=None, stream=None):
    """Returns (H1, H2, Y) of the batch X (M, 1024)."""
    _f32(params, (CH_MLP_PARAMS,), "params")
    M = X.shape[0]
    _f32(X, (M, CH_MLP_IN), "X")
    dev = X.device
    H1 = H1 if H1 is not None else torch.empty((M, CH_MLP_HID), dtype=torch.float32, device=dev)
    H2 = H2 if H2 is not None else torch.empty((M, CH_MLP_HID), dtype=torch.float32, device=dev)
    Y = Y if Y is not None else torch.empty((M, CH_MLP_K), dtype=torch.float32, device=dev)
    _check(lib().ch_mlp_forward(_ptr(params), _ptr(X), M, _ptr(H1), _ptr(H2), _ptr(Y),
                                _stream(stream)), "ch_mlp_forward")
    return H1, H2, Y


def ch_mlp_loss(Y, T, dY=None, loss=None, stream=None):
    """Returns (loss (1,), dY) for targets T (M, 16)."""
    M = Y.shape[0]
    _f32(Y, (M, CH_MLP_K), "Y")
    _f32(T, (M, CH_MLP_K), "T")
    dY = dY if dY is not None else torch.empty_like(Y)
    loss = loss if loss is not None else torch.empty(1, dtype=torch.float32, device=Y.device)
    _check(lib().ch_mlp_loss(_ptr(Y), _ptr(T), M, _ptr(dY), _ptr(loss), _stream(stream)),
           "ch_mlp_loss")
    return loss, dY


def ch_mlp_backward(params, X, H1, H2, dY, grads=None, workspace=None, stream=None):
    M = X.shape[0]
    grads = grads if grads is not None else torch.empty_like(params)
    ws = _ws(_size(lib().ch_mlp_backward_workspace_size, M), X.device, workspace)
    _check(lib().ch_mlp_backward(_ptr(params), _ptr(X), _ptr(H1), _ptr(H2), _ptr(dY), M,
                                 _ptr(grads), _ptr(ws), ws.numel(), _stream(stream)),
           "ch_mlp_backward")
    return grads


def ch_mlp_adam(params, grads, m, v, step: int, lr: float, beta1: float = 0.9,
                beta2: float = 0.999, eps: float = 1e-8, stream=None):
    _check(lib().ch_mlp_adam(_ptr(params), _ptr(grads), _ptr(m), _ptr(v), int(step), lr, beta1,
                             beta2, eps, _stream(stream)), "ch_mlp_adam")


# ---------------------------------------------------------------- learned culling
def ch_cull_workspace_size(p: int) -> int:
    return _size(lib().ch_cull_workspace_size, int(p))


def ch_cull_propose(pts, p: int, params=None, workspace=None, stream=None):
    """The culling proposal and its intermediate results, as a dict of device
    tensors: Linit (p, 2), features (1024,), net_out (16,), for both
    direction sets (0 sector centres, 1 network) dirs (2, 2, 16) and
    extremes (2, 16) int64, and for the polygon used poly (16, 2) with
    poly_count (1,) and chosen (1,) (1 network, 0 centres, -1 no network)."""
    pts = _pts(pts)
    dev = _dev(pts)
    if params is not None:
        _f32(params, (CH_MLP_PARAMS,), "params")
    out = {
        "Linit": torch.empty((p, 2), dtype=torch.int32, device=dev),
        "features": torch.empty(CH_MLP_IN, dtype=torch.float32, device=dev),
        "net_out": torch.zeros(CH_MLP_K, dtype=torch.float32, device=dev),
        "dirs": torch.empty((2, 2, CH_MLP_K), dtype=torch.float32, device=dev),
        "poly": torch.zeros((CH_MLP_K, 2), dtype=torch.int32, device=dev),
        "poly_count": torch.empty(1, dtype=torch.int32, device=dev),
        "extremes": torch.empty((2, CH_MLP_K), dtype=torch.int64, device=dev),
        "chosen": torch.empty(1, dtype=torch.int32, device=dev),
    }
    ws = _ws(ch_cull_workspace_size(p), dev, workspace)
    o = out
    _check(lib().ch_cull_propose(_ptr(pts), pts.shape[0], int(p), _ptr(params), _ptr(o["Linit"]),
                                 _ptr(o["features"]), _ptr(o["net_out"]), _ptr(o["dirs"]),
                                 _ptr(o["poly"]), _ptr(o["poly_count"]), _ptr(o["extremes"]),
                                 _ptr(o["chosen"]), _ptr(ws), ws.numel(), _stream(stream)),
           "ch_cull_propose")
    return out


def ch_hull_learned_workspace_size(n: int, p: int) -> int:
    return _size(lib().ch_hull_learned_workspace_size, int(n), int(p))


def ch_hull_learned_kernel_count(n: int, p: int, with_net: bool) -> int:
    k = ctypes.c_int32(0)
    _check(lib().ch_hull_learned_kernel_count(int(n), int(p), int(bool(with_net)), ctypes.byref(k)),
           "ch_hull_learned_kernel_count")
    return int(k.value)


def cull_stats_tensor(device="cuda"):
    """Device buffer for ch_hull_learned's ch_cull_stats (16 bytes as int64 (2,))."""
    return torch.zeros(2, dtype=torch.int64, device=device)


def cull_stats(t) -> dict:
    """The fields of a ch_cull_stats buffer: culled (points strictly inside the
    culling polygon), poly_vertices and chosen (1 network, 0 sector centres,
    -1 no network)."""
    w = t.cpu().view(torch.int32)
    return {"culled": int(t[0].item()), "poly_vertices": int(w[2]), "chosen": int(w[3])}


def ch_hull_learned(pts, p: int, params=None, L=None, Linit=None, lower=None, upper=None,
                    counts=None, hull=None, hull_count=None, stats=None, workspace=None,
                    stream=None):
    """The whole path with the culling proposal; returns (hull, hull_count).
    stats: None, or a cull_stats_tensor() the call fills in."""
    pts = _pts(pts)
    dev = _dev(pts)
    n = pts.shape[0]
    if params is not None:
        _f32(params, (CH_MLP_PARAMS,), "params")
    if stats is not None and (stats.dtype != torch.int64 or stats.numel() != 2
                              or not stats.is_contiguous()):
        raise ValueError("stats must be a contiguous int64 CUDA tensor of 2 elements")
    if hull is None:
        hull = torch.empty((2 * p, 2), dtype=torch.int32, device=dev)
    if hull_count is None:
        hull_count = torch.empty(1, dtype=torch.int32, device=dev)
    ws = _ws(ch_hull_learned_workspace_size(n, p), dev, workspace)
    _check(lib().ch_hull_learned(_ptr(pts), n, int(p), _ptr(params), _ptr(L), _ptr(Linit),
                                 _ptr(lower), _ptr(upper), _ptr(counts), _ptr(hull),
                                 _ptr(hull_count), _ptr(stats), _ptr(ws), ws.numel(),
                                 _stream(stream)),
           "ch_hull_learned")
    return hull, hull_count


# ---------------------------------------------------------------- any integer points
def ch_bbox(pts, box=None, workspace=None, stream=None):
    """(xmin, xmax, ymin, ymax) of the points as a device int32 tensor (4,)."""
    pts = _pts(pts)
    dev = _dev(pts)
    box = box if box is not None else torch.empty(4, dtype=torch.int32, device=dev)
    ws = _ws(_size(lib().ch_bbox_workspace_size), dev, workspace)
    _check(lib().ch_bbox(_ptr(pts), pts.shape[0], _ptr(box), _ptr(ws), ws.numel(), _stream(stream)),
           "ch_bbox")
    return box


def _host_box(box):
    import numpy as np
    b = np.ascontiguousarray(np.asarray(box, dtype=np.int32).reshape(4))
    return b, b.ctypes.data_as(ctypes.c_void_p)


def ch_convex_hull_box_workspace_size(n: int, box) -> int:
    b, bp = _host_box(box)
    return _size(lib().ch_convex_hull_box_workspace_size, int(n), bp)


def ch_convex_hull_box(pts, box, hull=None, hull_count=None, workspace=None, stream=None):
    """Hull of points anywhere in int32 given their bounding box (host values
    xmin, xmax, ymin, ymax); returns (hull, hull_count)."""
    pts = _pts(pts)
    dev = _dev(pts)
    b, bp = _host_box(box)
    side = int(min(int(b[1]) - int(b[0]), int(b[3]) - int(b[2]))) + 1
    if hull is None:
        hull = torch.empty((2 * max(side, 1) + 2, 2), dtype=torch.int32, device=dev)
    if hull_count is None:
        hull_count = torch.empty(1, dtype=torch.int32, device=dev)
    ws = _ws(ch_convex_hull_box_workspace_size(pts.shape[0], b), dev, workspace)
    _check(lib().ch_convex_hull_box(_ptr(pts), pts.shape[0], bp, _ptr(hull), _ptr(hull_count),
                                    _ptr(ws), ws.numel(), _stream(stream)), "ch_convex_hull_box")
    return hull, hull_count


def convex_hull(pts, stream=None):
    """Hull of any int32 points: ch_bbox, a 16-byte read of the box (the one
    synchronisation), then ch_convex_hull_box.  Returns the vertices as a
    device tensor (h, 2), counter-clockwise from the lexicographic minimum."""
    pts = _pts(pts)
    if pts.shape[0] == 0:
        return torch.empty((0, 2), dtype=torch.int32, device=pts.device)
    box = ch_bbox(pts, stream=stream).cpu().numpy()
    hull, hc = ch_convex_hull_box(pts, box, stream=stream)
    return hull[: int(hc.item())]
