"""CPU oracle for the (k,h)-core method -- TEST INFRASTRUCTURE ONLY.

The oracle is the plain single-threaded C program in ``khoracle.c``; this
module compiles it with gcc and exposes it through ctypes.  Only the tests,
``__graft_entry__.smoke()`` and the benchmark's CPU-baseline leg may import
it.  It shares no code with the CUDA library and never imports it.

Every function takes a graph as ``(rowptr int64[n+1], col int32[2m])`` numpy
arrays (symmetric CSR, sorted rows) and returns numpy arrays.  Citations of
the paper's passages are in ``khoracle.c``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "khoracle.c")
_LIB = os.path.join(_HERE, "_build", "libkhoracle.so")

SEQUENTIAL = 1
REFRESH_ALL = 2
DEFINITION = 4

_lib = None


def build(force: bool = False) -> str:
    """Compile khoracle.c into a shared library (gcc, -O2, no -march flags)."""
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-Wall",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is not None:
        return _lib
    lib = ctypes.CDLL(build())
    i64, i32, u32, u64 = ctypes.c_int64, ctypes.c_int32, ctypes.c_uint32, ctypes.c_uint64
    P = ctypes.c_void_p
    lib.kho_splitmix64_next.argtypes = [ctypes.POINTER(u64)]
    lib.kho_splitmix64_next.restype = u64
    lib.kho_ranks.argtypes = [i64, u64, P]
    lib.kho_ranks.restype = None
    lib.kho_budget_M.argtypes = [i64, ctypes.c_double, ctypes.c_double]
    lib.kho_budget_M.restype = i64
    lib.kho_hball.argtypes = [i64, P, P, P, i64, i32, P, P]
    lib.kho_hball.restype = i64
    lib.kho_hdegree_exact.argtypes = [i64, P, P, P, i32, P]
    lib.kho_hdegree_exact.restype = ctypes.c_int
    lib.kho_fixed_counts.argtypes = [i64, P, P, P, P, i32, i32, i32, P]
    lib.kho_fixed_counts.restype = ctypes.c_int
    lib.kho_estimate_def.argtypes = [i64, P, P, P, P, i32, i64, P, P, P]
    lib.kho_estimate_def.restype = ctypes.c_int
    lib.kho_estimate_dp.argtypes = [i64, P, P, P, P, i32, i64, P, P, P, P, P]
    lib.kho_estimate_dp.restype = ctypes.c_int
    lib.kho_core_exact.argtypes = [i64, P, P, i32, u32, P, P]
    lib.kho_core_exact.restype = i64
    lib.kho_core_sampled.argtypes = [i64, P, P, P, i32, i64, u32, P, P]
    lib.kho_core_sampled.restype = i64
    lib.kho_hdegree_some.argtypes = [i64, P, P, P, i32, P, i64, P]
    lib.kho_hdegree_some.restype = ctypes.c_int
    lib.kho_estimate_def_some.argtypes = [i64, P, P, P, P, i32, i64, P, i64, P, P, P]
    lib.kho_estimate_def_some.restype = ctypes.c_int
    lib.kho_dp_level.argtypes = [i64, P, P, P, i32, i64, P, P, P, i64, i64, P, P, P, P]
    lib.kho_dp_level.restype = ctypes.c_int
    lib.kho_dense_curve.argtypes = [i64, P, P, P, i32, i64, i32, P, i32, P, P]
    lib.kho_dense_curve.restype = ctypes.c_int
    lib.kho_dense_curve_pruned.argtypes = [i64, P, P, P, i32, i64, i32, P, i32, P,
                                           ctypes.c_double, P, P, P]
    lib.kho_dense_curve_pruned.restype = ctypes.c_int
    _lib = lib
    return lib


def _p(a):
    return None if a is None else ctypes.c_void_p(a.ctypes.data)


def _graph(rowptr, col):
    rowptr = np.ascontiguousarray(rowptr, dtype=np.int64)
    col = np.ascontiguousarray(col, dtype=np.int32)
    return rowptr, col, int(rowptr.size - 1)


def _alive(alive, n):
    if alive is None:
        return None
    return np.ascontiguousarray(alive, dtype=np.uint8)


def _check(rc, what):
    if rc < 0:
        raise RuntimeError(f"oracle {what} failed with code {rc}")


def splitmix64_stream(seed: int, count: int) -> np.ndarray:
    """First ``count`` outputs of SplitMix64 seeded with ``seed``."""
    lib = _load()
    st = ctypes.c_uint64(seed)
    return np.array([lib.kho_splitmix64_next(ctypes.byref(st)) for _ in range(count)],
                    dtype=np.uint64)


def ranks(n: int, seed: int) -> np.ndarray:
    r = np.zeros(max(n, 1), dtype=np.uint8)
    _load().kho_ranks(n, seed, _p(r))
    return r[:n]


def budget_M(n: int, eps: float, delta: float) -> int:
    return int(_load().kho_budget_M(n, eps, delta))


def hball(rowptr, col, v: int, h: int, alive=None) -> np.ndarray:
    rowptr, col, n = _graph(rowptr, col)
    al = _alive(alive, n)  # held until the C call returns
    out = np.zeros(max(n, 1), dtype=np.int32)
    dist = np.full(max(n, 1), -1, dtype=np.int32)
    s = _load().kho_hball(n, _p(rowptr), _p(col), _p(al), v, h, _p(out), _p(dist))
    return out[:s].copy()


def hdegree_exact(rowptr, col, h: int, alive=None) -> np.ndarray:
    rowptr, col, n = _graph(rowptr, col)
    al = _alive(alive, n)  # held until the C call returns
    deg = np.zeros(max(n, 1), dtype=np.int32)
    _check(_load().kho_hdegree_exact(n, _p(rowptr), _p(col), _p(al), h, _p(deg)),
           "hdegree_exact")
    return deg[:n]


def fixed_counts(rowptr, col, r, h: int, jlo: int, jhi: int, alive=None) -> np.ndarray:
    rowptr, col, n = _graph(rowptr, col)
    al = _alive(alive, n)  # held until the C call returns
    r = np.ascontiguousarray(r, dtype=np.uint8)
    nj = jhi - jlo + 1
    cnt = np.zeros((max(n, 1), nj), dtype=np.int32)
    _check(_load().kho_fixed_counts(n, _p(rowptr), _p(col), _p(al), _p(r), h,
                                    jlo, jhi, _p(cnt)), "fixed_counts")
    return cnt[:n]


def estimate_def(rowptr, col, r, h: int, M: int, alive=None):
    """(est uint64[n], k uint8[n], bsize int32[n]) from Def. 4.1 on N(v;h,X)."""
    rowptr, col, n = _graph(rowptr, col)
    al = _alive(alive, n)  # held until the C call returns
    r = np.ascontiguousarray(r, dtype=np.uint8)
    est = np.zeros(max(n, 1), dtype=np.uint64)
    k = np.zeros(max(n, 1), dtype=np.uint8)
    bs = np.zeros(max(n, 1), dtype=np.int32)
    _check(_load().kho_estimate_def(n, _p(rowptr), _p(col), _p(al), _p(r), h, M,
                                    _p(est), _p(k), _p(bs)), "estimate_def")
    return est[:n], k[:n], bs[:n]


def estimate_dp(rowptr, col, r, h: int, M: int, alive=None, levels: bool = False):
    """(est, k, bsize[, level_size int32[n,h], level_k uint8[n,h]]) via Alg. 2 levels."""
    rowptr, col, n = _graph(rowptr, col)
    al = _alive(alive, n)  # held until the C call returns
    r = np.ascontiguousarray(r, dtype=np.uint8)
    est = np.zeros(max(n, 1), dtype=np.uint64)
    k = np.zeros(max(n, 1), dtype=np.uint8)
    bs = np.zeros(max(n, 1), dtype=np.int32)
    ls = np.zeros((max(n, 1), h), dtype=np.int32) if levels else None
    lk = np.zeros((max(n, 1), h), dtype=np.uint8) if levels else None
    _check(_load().kho_estimate_dp(n, _p(rowptr), _p(col), _p(al), _p(r), h, M,
                                   _p(est), _p(k), _p(bs), _p(ls), _p(lk)), "estimate_dp")
    if levels:
        return est[:n], k[:n], bs[:n], ls[:n], lk[:n]
    return est[:n], k[:n], bs[:n]


def core_exact(rowptr, col, h: int, mode: int = 0):
    """(core int32[n], round_of int32[n], steps) of ExactCore."""
    rowptr, col, n = _graph(rowptr, col)
    core = np.zeros(max(n, 1), dtype=np.int32)
    rnd = np.zeros(max(n, 1), dtype=np.int32)
    steps = _load().kho_core_exact(n, _p(rowptr), _p(col), h, mode, _p(core), _p(rnd))
    _check(steps, "core_exact")
    return core[:n], rnd[:n], int(steps)


def core_sampled(rowptr, col, r, h: int, M: int, mode: int = 0):
    """(core uint64[n], round_of int32[n], steps) of Core (Alg. 4)."""
    rowptr, col, n = _graph(rowptr, col)
    r = np.ascontiguousarray(r, dtype=np.uint8)
    core = np.zeros(max(n, 1), dtype=np.uint64)
    rnd = np.zeros(max(n, 1), dtype=np.int32)
    steps = _load().kho_core_sampled(n, _p(rowptr), _p(col), _p(r), h, M, mode, _p(core), _p(rnd))
    _check(steps, "core_sampled")
    return core[:n], rnd[:n], int(steps)


def hdegree_some(rowptr, col, h: int, vertices, alive=None) -> np.ndarray:
    """deg_h(v; X) for the listed nodes only."""
    rowptr, col, n = _graph(rowptr, col)
    al = _alive(alive, n)  # held until the C call returns
    vs = np.ascontiguousarray(vertices, dtype=np.int32)
    deg = np.zeros(max(vs.size, 1), dtype=np.int32)
    _check(_load().kho_hdegree_some(n, _p(rowptr), _p(col), _p(al), h, _p(vs),
                                    vs.size, _p(deg)), "hdegree_some")
    return deg[:vs.size]


def estimate_def_some(rowptr, col, r, h: int, M: int, vertices, alive=None):
    """Def. 4.1 (est, k, bsize) for the listed nodes only."""
    rowptr, col, n = _graph(rowptr, col)
    al = _alive(alive, n)  # held until the C call returns
    r = np.ascontiguousarray(r, dtype=np.uint8)
    vs = np.ascontiguousarray(vertices, dtype=np.int32)
    m = max(vs.size, 1)
    est = np.zeros(m, dtype=np.uint64)
    k = np.zeros(m, dtype=np.uint8)
    bs = np.zeros(m, dtype=np.int32)
    _check(_load().kho_estimate_def_some(n, _p(rowptr), _p(col), _p(al), _p(r), h, M,
                                         _p(vs), vs.size, _p(est), _p(k), _p(bs)),
           "estimate_def_some")
    return est[:vs.size], k[:vs.size], bs[:vs.size]


def dense_curve(rowptr, col, r, h: int, M: int, exact: bool, round_of, rounds: int):
    """EstDense (Alg. 7): (sum uint64[rounds], size int64[rounds]) with
    sum[q] = sum of d(v; X_q) over X_q = {v : round_of[v] >= q}."""
    rowptr, col, n = _graph(rowptr, col)
    r = np.ascontiguousarray(r, dtype=np.uint8)
    ro = np.ascontiguousarray(round_of, dtype=np.int32)
    total = np.zeros(max(rounds, 1), dtype=np.uint64)
    size = np.zeros(max(rounds, 1), dtype=np.int64)
    _check(_load().kho_dense_curve(n, _p(rowptr), _p(col), _p(r), h, max(M, 1), 1 if exact else 0,
                                   _p(ro), rounds, _p(total), _p(size)), "dense_curve")
    return total[:rounds], size[:rounds]


def dense_curve_pruned(rowptr, col, r, h: int, M: int, exact: bool, round_of, rounds: int,
                       core, eps: float):
    """EstDense's faster variant (Sec. 6): nodes with c'(v) < gamma k' removed
    first (gamma = (1-eps)/(1+eps), k' = max c').  Returns (sum uint64[rounds],
    size int64[rounds], keep uint8[n]) over X'_q = {v kept : round_of[v] >= q}."""
    rowptr, col, n = _graph(rowptr, col)
    r = np.ascontiguousarray(r, dtype=np.uint8)
    ro = np.ascontiguousarray(round_of, dtype=np.int32)
    c = np.ascontiguousarray(core, dtype=np.uint64)
    total = np.zeros(max(rounds, 1), dtype=np.uint64)
    size = np.zeros(max(rounds, 1), dtype=np.int64)
    keep = np.zeros(max(n, 1), dtype=np.uint8)
    _check(_load().kho_dense_curve_pruned(n, _p(rowptr), _p(col), _p(r), h, max(M, 1),
                                          1 if exact else 0, _p(ro), rounds, _p(c), eps,
                                          _p(total), _p(size), _p(keep)), "dense_curve_pruned")
    return total[:rounds], size[:rounds], keep[:n]


def dp_level(rowptr, col, r, i: int, M: int, prev=None, v0: int = 0, v1: int = None):
    """One level of the list recursion (Alg. 2, Prop. 3.1) for nodes v0..v1-1 of
    the whole graph.  prev = (off int64[n+1], ids int32[], k uint8[n]) holds the
    level i-1 lists of every node (None for i = 1).  Returns (k uint8, size
    int32, est uint64, off int64[m+1], ids int32[]) for the m = v1 - v0 nodes,
    each list sorted by rank descending then id."""
    rowptr, col, n = _graph(rowptr, col)
    v1 = n if v1 is None else v1
    m = v1 - v0
    r = np.ascontiguousarray(r, dtype=np.uint8)
    k = np.zeros(max(m, 1), np.uint8)
    size = np.zeros(max(m, 1), np.int32)
    est = np.zeros(max(m, 1), np.uint64)
    slots = np.zeros(max(m, 1) * M, np.int32)
    if prev is not None:
        poff = np.ascontiguousarray(prev[0], dtype=np.int64)
        pids = np.ascontiguousarray(prev[1], dtype=np.int32)
        pk = np.ascontiguousarray(prev[2], dtype=np.uint8)
        if pids.size == 0:
            pids = np.zeros(1, np.int32)
    else:
        poff = pids = pk = None
    _check(_load().kho_dp_level(n, _p(rowptr), _p(col), _p(r), i, M, _p(poff), _p(pids),
                                _p(pk), v0, v1, _p(k), _p(size), _p(slots), _p(est)), "dp_level")
    k, size, est = k[:m], size[:m], est[:m]
    off = np.zeros(m + 1, np.int64)
    np.cumsum(size, out=off[1:])
    keep = (np.arange(M)[None, :] < size[:, None]) if m else np.zeros((0, M), bool)
    ids = slots[:m * M].reshape(m, M)[keep]
    return k, size, est, off, ids
