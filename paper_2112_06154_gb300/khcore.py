"""Thin Python binding of the C ABI in ``include/khcore.h``.

Functions carry the C names and only marshal arguments: every step of the
path runs in the CUDA library ``_build/libkhcore.so``.  Host arrays are numpy;
device arrays are torch CUDA tensors (their ``data_ptr()`` is passed with
``KH_DEVICE_PTR``).  Loading fails loudly when the library is missing; there
is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

KH_OK = 0
KH_EINVAL = -1
KH_EGRAPH = -2
KH_ENOMEM = -3
KH_ECUDA = -4
KH_ETIMEOUT = -5
KH_EINTERNAL = -6
KH_DEVICE_PTR = 1
KH_PROF_BFS = 0
KH_PROF_LEVEL1 = 1
KH_PROF_LEVELU = 2
KH_PROF_FRONTIER = 3
KH_PROF_PEEL = 4
KH_PROF_KINDS = 5
KH_OP_HDEG2 = 0
KH_VAR_AUTO = 0
KH_VAR_CTA = 1
KH_VAR_SLICED = 2
KH_VAR_SLICED_SMALL = 3
KH_OP_PEEL_COMPACT = 1
KH_COMPACT_OFF = 1
KH_COMPACT_ALWAYS = 2
KH_OP_LEVEL_UNION = 2
KH_LEVELU_STEPPED = 1
KH_LEVELU_FREE = 2
KH_LEVELU_GROUPED = 3
KH_OP_HDEG2_SWEEP = 3
KH_SWEEP_OFF = 1
KH_SWEEP_FROM = 2
PROF_NAMES = ["bfs", "level1", "levelU", "frontier", "peel"]

_ERRNAMES = {KH_EINVAL: "KH_EINVAL", KH_EGRAPH: "KH_EGRAPH", KH_ENOMEM: "KH_ENOMEM",
             KH_ECUDA: "KH_ECUDA", KH_ETIMEOUT: "KH_ETIMEOUT", KH_EINTERNAL: "KH_EINTERNAL"}

# (name, restype, argtypes) of every entry point declared in include/khcore.h
_P = ctypes.c_void_p
_PP = ctypes.POINTER(ctypes.c_void_p)
_I64P = ctypes.POINTER(ctypes.c_int64)
SIGNATURES = [
    ("kh_ctx_create", ctypes.c_int, [_PP, ctypes.c_int, _P]),
    ("kh_ctx_destroy", ctypes.c_int, [_P]),
    ("kh_last_error", ctypes.c_char_p, [_P]),
    ("kh_debug_fail_alloc", ctypes.c_int, [_P, ctypes.c_int64]),
    ("kh_graph_load_csr", ctypes.c_int, [_P, ctypes.c_int64, _P, _P, ctypes.c_uint32, _PP]),
    ("kh_graph_free", ctypes.c_int, [_P]),
    ("kh_graph_load_batch", ctypes.c_int, [_P, ctypes.c_int32, _P, _P, _P, _P, ctypes.c_uint32, _PP]),
    ("kh_graph_n", ctypes.c_int, [_P, _I64P]),
    ("kh_footprint", ctypes.c_int, [ctypes.c_int64, ctypes.c_int64, ctypes.c_int32, ctypes.c_int64,
                                    ctypes.c_double, ctypes.c_double, _I64P, _I64P]),
    ("kh_set_h", ctypes.c_int, [_P, ctypes.c_int32]),
    ("kh_set_sampling", ctypes.c_int, [_P, ctypes.c_uint64, ctypes.c_int64, ctypes.c_double,
                                       ctypes.c_double]),
    ("kh_get_M", ctypes.c_int, [_P, _I64P]),
    ("kh_ranks", ctypes.c_int, [_P, _P, ctypes.c_uint32]),
    ("kh_hdegree_exact", ctypes.c_int, [_P, _P, ctypes.c_uint32]),
    ("kh_sampled_counts", ctypes.c_int, [_P, ctypes.c_int32, ctypes.c_int32, _P, ctypes.c_uint32]),
    ("kh_estimate", ctypes.c_int, [_P, _P, _P, _P, ctypes.c_uint32]),
    ("kh_core_exact", ctypes.c_int, [_P, _P, ctypes.c_uint32]),
    ("kh_core_sampled", ctypes.c_int, [_P, _P, ctypes.c_uint32]),
    ("kh_peel_info", ctypes.c_int, [_P, _P, _I64P, _I64P]),
    ("kh_prof_enable", ctypes.c_int, [_P, ctypes.c_int32]),
    ("kh_prof_read", ctypes.c_int, [_P, ctypes.c_int32, ctypes.POINTER(ctypes.c_double), _I64P,
                                    ctypes.POINTER(ctypes.c_double)]),
    ("kh_peel_stats", ctypes.c_int, [_P, _P, _P, _I64P]),
    ("kh_dense", ctypes.c_int, [_P, ctypes.c_int32, _P, ctypes.c_int32, _P, _P,
                                ctypes.POINTER(ctypes.c_int32)]),
    ("kh_dense_pruned", ctypes.c_int, [_P, ctypes.c_int32, _P, ctypes.c_int32, _P, ctypes.c_double,
                                       _P, _P, ctypes.POINTER(ctypes.c_int32), _P]),
    ("kh_prof_trace", ctypes.c_int, [_P, ctypes.c_int32, _P, ctypes.c_int64, _I64P]),
    ("kh_prof_trace_bytes", ctypes.c_int, [_P, ctypes.c_int32, _P, ctypes.c_int64, _I64P]),
    ("kh_launch_count", ctypes.c_int, [_P, _I64P]),
    ("kh_hdegree_exact_noalloc", ctypes.c_int, [ctypes.c_int64, _P, _P, ctypes.c_int32, _P, _P]),
    ("kh_set_variant", ctypes.c_int, [_P, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                      ctypes.c_int32]),
    ("kh_get_variant", ctypes.c_int, [_P, ctypes.c_int32, ctypes.POINTER(ctypes.c_int32),
                                      ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int32),
                                      ctypes.POINTER(ctypes.c_double)]),
    ("kh_sync", ctypes.c_int, [_P]),
]

_lib = None


class KhError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{_ERRNAMES.get(code, code)}: {msg}")
        self.code = code


def lib_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = False):
    """Load libkhcore.so (optionally building it first)."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.LIB
    if not os.path.exists(path):
        if build_if_missing:
            _build.build()
        else:
            raise ImportError(f"CUDA library not built: {path} (run __graft_entry__.build())")
    lib = ctypes.CDLL(path)
    for name, res, args in SIGNATURES:
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


class Ctx:
    """Owner of a ``kh_ctx*``."""

    def __init__(self, handle):
        self.handle = handle

    def error(self) -> str:
        return load().kh_last_error(self.handle).decode(errors="replace")

    def close(self):
        if self.handle:
            load().kh_ctx_destroy(self.handle)
            self.handle = None


class Graph:
    """Owner of a ``kh_graph*`` (keeps its context alive)."""

    def __init__(self, ctx: Ctx, handle, n: int):
        self.ctx = ctx
        self.handle = handle
        self.n = n

    def close(self):
        if self.handle:
            load().kh_graph_free(self.handle)
            self.handle = None


def _check(rc, ctx: Ctx):
    if rc != KH_OK:
        raise KhError(rc, ctx.error() if ctx is not None else "")


def _is_torch(x):
    return type(x).__module__.startswith("torch")


def _ptr(x):
    """(pointer, is_device) for a numpy array or a torch tensor."""
    if x is None:
        return None, False
    if _is_torch(x):
        if not x.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return ctypes.c_void_p(x.data_ptr()), x.is_cuda
    if not x.flags.c_contiguous:
        raise ValueError("array must be C-contiguous")
    return ctypes.c_void_p(x.ctypes.data), False


def kh_ctx_create(device: int = 0, stream=None) -> Ctx:
    """``stream``: a torch.cuda.Stream, a raw cudaStream_t int, or None."""
    h = ctypes.c_void_p()
    s = None
    if stream is not None:
        s = ctypes.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))
    rc = load().kh_ctx_create(ctypes.byref(h), device, s)
    if rc != KH_OK:
        raise KhError(rc, "kh_ctx_create failed")
    return Ctx(h)


def kh_ctx_destroy(ctx: Ctx):
    ctx.close()


def kh_debug_fail_alloc(ctx: Ctx, k: int):
    """Make the k-th device allocation of this context fail once with KH_ENOMEM (0: off)."""
    rc = load().kh_debug_fail_alloc(ctx.handle, k)
    if rc:
        raise KhError(rc, "kh_debug_fail_alloc")


def kh_last_error(ctx: Ctx) -> str:
    return ctx.error()


def _csr_arrays(rowptr, col):
    """Typed, contiguous CSR arrays whose sizes agree: the C ABI takes rowptr[n]
    as the length of col, so a shorter col would be read past its end."""
    if _is_torch(rowptr) or _is_torch(col):
        import torch
        if not (_is_torch(rowptr) and _is_torch(col)):
            raise KhError(KH_EINVAL, "rowptr and col must both be torch tensors or both numpy")
        if rowptr.dtype != torch.int64 or col.dtype != torch.int32:
            raise KhError(KH_EINVAL, "rowptr must be int64 and col int32")
        rowptr, col = rowptr.contiguous(), col.contiguous()
        if rowptr.numel() < 1 or int(rowptr[-1].item()) != col.numel():
            raise KhError(KH_EGRAPH, "rowptr[-1] must equal the length of col")
        return rowptr, col
    rowptr = np.ascontiguousarray(rowptr, dtype=np.int64)
    col = np.ascontiguousarray(col, dtype=np.int32)
    if rowptr.ndim != 1 or rowptr.size < 1 or int(rowptr[-1]) != col.size:
        raise KhError(KH_EGRAPH, "rowptr[-1] must equal the length of col")
    return rowptr, col


def kh_graph_load_csr(ctx: Ctx, rowptr, col) -> Graph:
    """rowptr int64[n+1], col int32[nnz]: both numpy (host) or both torch CUDA tensors."""
    rowptr, col = _csr_arrays(rowptr, col)
    n = int(rowptr.shape[0]) - 1
    pr, dev = _ptr(rowptr)
    pc, _ = _ptr(col)
    h = ctypes.c_void_p()
    rc = load().kh_graph_load_csr(ctx.handle, n, pr, pc, KH_DEVICE_PTR if dev else 0,
                                  ctypes.byref(h))
    _check(rc, ctx)
    return Graph(ctx, h, n)


def kh_graph_free(g: Graph):
    g.close()


def kh_set_h(g: Graph, h: int):
    _check(load().kh_set_h(g.handle, h), g.ctx)


def kh_set_sampling(g: Graph, seed: int = 1, M: int = 0, eps: float = 0.5, delta: float = 0.05):
    _check(load().kh_set_sampling(g.handle, seed, M, eps, delta), g.ctx)


def kh_get_M(g: Graph) -> int:
    m = ctypes.c_int64()
    _check(load().kh_get_M(g.handle, ctypes.byref(m)), g.ctx)
    return int(m.value)


def _out(out, n, dtype, cols=None):
    if out is not None:
        return out
    shape = (n,) if cols is None else (n, max(cols, 0))
    return np.zeros(shape, dtype=dtype)


def kh_ranks(g: Graph, out=None):
    out = _out(out, g.n, np.uint8)
    p, dev = _ptr(out)
    _check(load().kh_ranks(g.handle, p, KH_DEVICE_PTR if dev else 0), g.ctx)
    return out


def kh_hdegree_exact(g: Graph, out=None):
    out = _out(out, g.n, np.int32)
    p, dev = _ptr(out)
    _check(load().kh_hdegree_exact(g.handle, p, KH_DEVICE_PTR if dev else 0), g.ctx)
    return out


def kh_sampled_counts(g: Graph, j_lo: int, j_hi: int, out=None):
    out = _out(out, g.n, np.int32, j_hi - j_lo + 1)
    p, dev = _ptr(out)
    _check(load().kh_sampled_counts(g.handle, j_lo, j_hi, p, KH_DEVICE_PTR if dev else 0), g.ctx)
    return out


def kh_estimate(g: Graph, est=None, level=None, bsize=None):
    """Returns (est uint64, level uint8, bsize int32)."""
    est = _out(est, g.n, np.uint64)
    dev = _ptr(est)[1]
    if level is None and not dev:
        level = np.zeros(g.n, np.uint8)
    if bsize is None and not dev:
        bsize = np.zeros(g.n, np.int32)
    pe, _ = _ptr(est)
    pl, _ = _ptr(level)
    pb, _ = _ptr(bsize)
    _check(load().kh_estimate(g.handle, pe, pl, pb, KH_DEVICE_PTR if dev else 0), g.ctx)
    return est, level, bsize


def kh_core_exact(g: Graph, out=None):
    out = _out(out, g.n, np.int32)
    p, dev = _ptr(out)
    _check(load().kh_core_exact(g.handle, p, KH_DEVICE_PTR if dev else 0), g.ctx)
    return out


def kh_core_sampled(g: Graph, out=None):
    out = _out(out, g.n, np.uint64)
    p, dev = _ptr(out)
    _check(load().kh_core_sampled(g.handle, p, KH_DEVICE_PTR if dev else 0), g.ctx)
    return out


def kh_peel_info(g: Graph, want_rounds: bool = True):
    """(round_of int32[n] or None, rounds, updates) of the last kh_core_* call."""
    ro = np.zeros(g.n, np.int32) if want_rounds else None
    rounds = ctypes.c_int64()
    updates = ctypes.c_int64()
    p, _ = _ptr(ro)
    _check(load().kh_peel_info(g.handle, p, ctypes.byref(rounds), ctypes.byref(updates)), g.ctx)
    return ro, int(rounds.value), int(updates.value)


KH_MAX_H = 16


def kh_dense(g: Graph, exact: bool, round_of, rounds: int):
    """EstDense (Alg. 7): (sum uint64[rounds], size int64[rounds], best)."""
    ro = np.ascontiguousarray(round_of, dtype=np.int32)
    if ro.size != g.n:
        raise KhError(KH_EINVAL, f"round_of has {ro.size} entries, the graph {g.n} nodes")
    total = np.zeros(max(rounds, 1), np.uint64)
    size = np.zeros(max(rounds, 1), np.int64)
    best = ctypes.c_int32(-1)
    _check(load().kh_dense(g.handle, 1 if exact else 0, ro.ctypes.data, rounds, total.ctypes.data,
                           size.ctypes.data, ctypes.byref(best)), g.ctx)
    return total[:rounds], size[:rounds], int(best.value)


def kh_dense_pruned(g: Graph, exact: bool, round_of, rounds: int, core, eps: float):
    """EstDense after dropping nodes with core < gamma max(core) (Sec. 6):
    (sum uint64[rounds], size int64[rounds], best, kept uint8[n])."""
    ro = np.ascontiguousarray(round_of, dtype=np.int32)
    c = np.ascontiguousarray(core, dtype=np.uint64)
    if ro.size != g.n or c.size != g.n:
        raise KhError(KH_EINVAL, f"round_of and core need {g.n} entries")
    total = np.zeros(max(rounds, 1), np.uint64)
    size = np.zeros(max(rounds, 1), np.int64)
    kept = np.zeros(max(g.n, 1), np.uint8)
    best = ctypes.c_int32(-1)
    _check(load().kh_dense_pruned(g.handle, 1 if exact else 0, ro.ctypes.data, rounds,
                                  c.ctypes.data, eps, total.ctypes.data, size.ctypes.data,
                                  ctypes.byref(best), kept.ctypes.data), g.ctx)
    return total[:rounds], size[:rounds], int(best.value), kept[:g.n]


def kh_peel_stats(g: Graph):
    """(refreshed int64[KH_MAX_H+1], changed int64[KH_MAX_H+1], stopped) of the last peel."""
    ref = np.zeros(KH_MAX_H + 1, np.int64)
    chg = np.zeros(KH_MAX_H + 1, np.int64)
    st = ctypes.c_int64()
    _check(load().kh_peel_stats(g.handle, ref.ctypes.data, chg.ctypes.data, ctypes.byref(st)), g.ctx)
    return ref, chg, int(st.value)


def kh_sync(g: Graph):
    _check(load().kh_sync(g.handle), g.ctx)


def kh_footprint(n: int, nnz: int, h: int, M: int = 0, eps: float = 0.5, delta: float = 0.05):
    """(M in force, upper bound of device bytes) of a sampled decomposition of a
    graph of n nodes and nnz adjacency entries, before loading it (host only)."""
    m = ctypes.c_int64()
    b = ctypes.c_int64()
    rc = load().kh_footprint(n, nnz, h, M, eps, delta, ctypes.byref(m), ctypes.byref(b))
    if rc != KH_OK:
        raise KhError(rc, "kh_footprint: bad sizes or sampling parameters")
    return int(m.value), int(b.value)


def kh_graph_n(g: Graph) -> int:
    n = ctypes.c_int64()
    _check(load().kh_graph_n(g.handle, ctypes.byref(n)), g.ctx)
    return int(n.value)


def kh_prof_enable(g: Graph, on: bool = True):
    _check(load().kh_prof_enable(g.handle, 1 if on else 0), g.ctx)


def kh_prof_read(g: Graph, kind: int):
    """(ms, launches, algorithmic bytes) accumulated for one kernel class."""
    ms = ctypes.c_double()
    n = ctypes.c_int64()
    b = ctypes.c_double()
    _check(load().kh_prof_read(g.handle, kind, ctypes.byref(ms), ctypes.byref(n), ctypes.byref(b)),
           g.ctx)
    return float(ms.value), int(n.value), float(b.value)


def kh_prof_trace(g: Graph, kind: int) -> np.ndarray:
    """Event time (ms) of every bracketed launch of one kernel class, in order."""
    n = ctypes.c_int64()
    _check(load().kh_prof_trace(g.handle, kind, None, 0, ctypes.byref(n)), g.ctx)
    out = np.zeros(max(n.value, 1), np.float32)
    _check(load().kh_prof_trace(g.handle, kind, out.ctypes.data, out.size, ctypes.byref(n)), g.ctx)
    return out[:n.value]


def kh_prof_trace_bytes(g: Graph, kind: int) -> np.ndarray:
    """Algorithmic bytes of every bracketed launch of one kernel class, in the
    order of kh_prof_trace (UINT64_MAX where not recorded)."""
    n = ctypes.c_int64()
    _check(load().kh_prof_trace_bytes(g.handle, kind, None, 0, ctypes.byref(n)), g.ctx)
    out = np.zeros(max(n.value, 1), np.uint64)
    _check(load().kh_prof_trace_bytes(g.handle, kind, out.ctypes.data, out.size, ctypes.byref(n)),
           g.ctx)
    return out[:n.value]


def kh_launch_count(g: Graph) -> int:
    n = ctypes.c_int64()
    _check(load().kh_launch_count(g.handle, ctypes.byref(n)), g.ctx)
    return int(n.value)


def kh_set_variant(g: Graph, variant: int, slices: int = 0, threads: int = 0,
                   op: int = KH_OP_HDEG2):
    """Force the layout of the h = 2 exact-degree pass (KH_VAR_AUTO: the tuner's),
    or another schedule setting by op: KH_OP_PEEL_COMPACT (compaction),
    KH_OP_LEVEL_UNION (level union), KH_OP_HDEG2_SWEEP (bit-parallel sweeps;
    KH_SWEEP_FROM with slices = the work bin)."""
    _check(load().kh_set_variant(g.handle, op, variant, slices, threads), g.ctx)


def kh_get_variant(g: Graph, op: int = KH_OP_HDEG2):
    """(variant, slices, threads, sample ms) of the layout in force (tunes if needed)."""
    v, sl, th = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
    ms = ctypes.c_double()
    _check(load().kh_get_variant(g.handle, op, ctypes.byref(v), ctypes.byref(sl), ctypes.byref(th),
                                 ctypes.byref(ms)), g.ctx)
    return int(v.value), int(sl.value), int(th.value), float(ms.value)


def kh_hdegree_exact_noalloc(rowptr, col, h: int, deg, stream=None) -> int:
    """Allocation-free exact h-degrees on device tensors (see include/khcore.h).

    rowptr int64[n+1], col int32[nnz] and deg int32[n] are contiguous 1-D CUDA
    tensors of the current device (KhError KH_EINVAL otherwise: the library
    reads them as such without checking); returns the C return code (0 on
    success)."""
    import torch
    for name, t, dt in (("rowptr", rowptr, torch.int64), ("col", col, torch.int32),
                        ("deg", deg, torch.int32)):
        if not _is_torch(t) or not t.is_cuda or t.dim() != 1 or not t.is_contiguous():
            raise KhError(KH_EINVAL, f"{name} must be a contiguous 1-D CUDA tensor")
        if t.dtype != dt:
            raise KhError(KH_EINVAL, f"{name} must be {dt}")
        if t.device.index != torch.cuda.current_device():
            raise KhError(KH_EINVAL, f"{name} must be on the current device")
    n = int(rowptr.shape[0]) - 1
    if n < 0 or deg.numel() != n:
        raise KhError(KH_EINVAL, "deg needs one entry per node (rowptr has n + 1)")
    if n > 0 and int(rowptr[-1].item()) != col.numel():
        raise KhError(KH_EGRAPH, "rowptr[-1] must equal the length of col")
    s = None
    if stream is not None:
        s = ctypes.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))
    return int(load().kh_hdegree_exact_noalloc(n, ctypes.c_void_p(rowptr.data_ptr()),
                                               ctypes.c_void_p(col.data_ptr()), h,
                                               ctypes.c_void_p(deg.data_ptr()), s))


def kh_graph_load_batch(ctx: Ctx, vtx_off, rowptr, col, h_per_graph=None) -> Graph:
    """Packed graphs (see include/khcore.h): vtx_off int64[g+1] and h_per_graph
    int32[g] on the host; rowptr/col numpy (host) or torch CUDA tensors."""
    vtx_off = np.ascontiguousarray(vtx_off, dtype=np.int64)
    hpg = None if h_per_graph is None else np.ascontiguousarray(h_per_graph, dtype=np.int32)
    rowptr, col = _csr_arrays(rowptr, col)
    if vtx_off.size < 1 or int(vtx_off[-1]) != int(rowptr.shape[0]) - 1:
        raise KhError(KH_EINVAL, "vtx_off[-1] must equal the number of nodes")
    if hpg is not None and hpg.size != vtx_off.size - 1:
        raise KhError(KH_EINVAL, "h_per_graph needs one entry per graph")
    pr, dev = _ptr(rowptr)
    pc, _ = _ptr(col)
    h = ctypes.c_void_p()
    rc = load().kh_graph_load_batch(ctx.handle, int(vtx_off.size - 1), _ptr(vtx_off)[0], pr, pc,
                                    _ptr(hpg)[0] if hpg is not None else None,
                                    KH_DEVICE_PTR if dev else 0, ctypes.byref(h))
    _check(rc, ctx)
    return Graph(ctx, h, int(vtx_off[-1]))
