"""Write the SHA-256 digests of full-size oracle outputs.

Runs only the CPU oracle (``oracle/``) on the full-size seeded graphs:
  C2  Chung-Lu, n = 200,000, mean degree 20, exponent 2.5, maximum expected
      degree 5,000, graph seed 1002;
  C3  R-MAT scale 22, edge factor 16, a/b/c/d = .57/.19/.19/.05, graph seed 1003;
with rank seed 1 and M from Eq. (buffer) at eps = 0.5, delta = 0.05, and
records, per output vector, the SHA-256 of its raw little-endian bytes in
``fullsize_sha256.txt`` (next to this script).  The GPU tests hash the
library's output the same way, so an equal digest means an equal vector,
element by element.  The vectors themselves go to a cache folder (``--cache``,
default ``_cache/`` next to this script, not committed; also read from the
environment variable KH_ORACLE_CACHE) for a per-element comparison when a
digest differs; it holds the intermediate level lists too (several GB for C3).

Each oracle routine stays single-threaded; independent ranges of nodes run in
separate processes (``--jobs``):
  hdeg   exact h-degrees (Sec. 2): oracle.hdegree_some over node ranges;
  counts fixed-level counts j = 0..10 (Alg. 1 with the level forced to j):
         oracle.fixed_counts, one process;
  est    the level recursion (Prop. 3.1, Alg. 2) level by level with
         oracle.dp_level over node ranges, then Alg. 1: est, k[v,h], |B[v,h]|.

Usage: python tests/golden/make_fullsize.py [--jobs 8] [--cache DIR] [case ...]
"""
from __future__ import annotations

import argparse
import hashlib
import multiprocessing as mp
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
CACHE = os.environ.get("KH_ORACLE_CACHE") or os.path.join(HERE, "_cache")
DIGESTS = os.path.join(HERE, "fullsize_sha256.txt")
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

EPS, DELTA, RANK_SEED = 0.5, 0.05, 1

# case -> (graph, kind, h)
CASES = {
    "c2_hdeg_h2": ("c2", "hdeg", 2),
    "c2_hdeg_h3": ("c2", "hdeg", 3),
    "c2_counts_h2": ("c2", "counts", 2),
    "c2_counts_h3": ("c2", "counts", 3),
    "c2_est_h2": ("c2", "est", 2),
    "c2_est_h3": ("c2", "est", 3),
    "c3_hdeg_h2": ("c3", "hdeg", 2),
    "c3_est_h2": ("c3", "est", 2),
    "c3_est_h3": ("c3", "est", 3),
    "c3_est_h4": ("c3", "est", 4),
}
CITE = {"hdeg": "Sec. 2 (deg_h = |N(v;h)| - 1)",
        "counts": "Alg. 1 with the level forced to j = 0..10",
        "est": "Prop. 3.1 + Alg. 2 levels, then Alg. 1"}


def make_graph(name):
    from paper_2112_06154_gb300 import graphgen as gg
    if name == "c2":
        return gg.chung_lu(200_000, 20, 2.5, 5000, 1002)
    return gg.rmat(22, 16, 0.57, 0.19, 0.19, 1003)


def digest(a) -> str:
    a = np.ascontiguousarray(a)
    return hashlib.sha256(a.astype(a.dtype.newbyteorder("<"), copy=False).tobytes()).hexdigest()


def graph_files(name):
    rp_f = os.path.join(CACHE, f"{name}_rowptr.npy")
    cl_f = os.path.join(CACHE, f"{name}_col.npy")
    if not (os.path.exists(rp_f) and os.path.exists(cl_f)):
        rp, cl = make_graph(name)
        np.save(rp_f, rp)
        np.save(cl_f, cl)
    return rp_f, cl_f


# ------------------------------------------------------------- workers (spawn)

def _hdeg_chunk(args):
    import oracle as O
    rp_f, cl_f, h, v0, v1 = args
    rp = np.load(rp_f, mmap_mode="r")
    cl = np.load(cl_f, mmap_mode="r")
    return v0, O.hdegree_some(rp, cl, h, np.arange(v0, v1, dtype=np.int32))


def _level_chunk(args):
    import oracle as O
    rp_f, cl_f, i, M, prev_files, v0, v1 = args
    rp = np.load(rp_f, mmap_mode="r")
    cl = np.load(cl_f, mmap_mode="r")
    r = O.ranks(rp.size - 1, RANK_SEED)
    prev = None
    if prev_files is not None:
        prev = tuple(np.load(f, mmap_mode="r") for f in prev_files)
    return (v0,) + O.dp_level(rp, cl, r, i, M, prev, v0, v1)


def _counts_job(args):
    import oracle as O
    rp_f, cl_f, h = args
    rp = np.load(rp_f)
    cl = np.load(cl_f)
    r = O.ranks(rp.size - 1, RANK_SEED)
    return O.fixed_counts(rp, cl, r, h, 0, 10)


# ------------------------------------------------------------------- drivers

def ranges(n, chunk):
    return [(v0, min(n, v0 + chunk)) for v0 in range(0, n, chunk)]


def run_hdeg(pool, name, h):
    rp_f, cl_f = graph_files(name)
    n = np.load(rp_f, mmap_mode="r").size - 1
    out = np.zeros(n, np.int32)
    for v0, deg in pool.imap_unordered(_hdeg_chunk, [(rp_f, cl_f, h, a, b)
                                                     for a, b in ranges(n, 8192)]):
        out[v0:v0 + deg.size] = deg
    return {"deg": out}


def run_counts(pool, name, h):
    rp_f, cl_f = graph_files(name)
    return {"cnt": pool.apply(_counts_job, ((rp_f, cl_f, h),))}


def run_est(pool, name, h):
    import oracle as O
    rp_f, cl_f = graph_files(name)
    n = np.load(rp_f, mmap_mode="r").size - 1
    M = O.budget_M(n, EPS, DELTA)
    prev_files = None
    for i in range(1, h + 1):
        lvl_files = [os.path.join(CACHE, f"{name}_M{M}_level{i}_{part}.npy")
                     for part in ("off", "ids", "k")]
        est_f = os.path.join(CACHE, f"{name}_M{M}_level{i}_est.npy")
        if all(os.path.exists(f) for f in lvl_files + [est_f]):
            prev_files = lvl_files
            continue
        k = np.zeros(n, np.uint8)
        size = np.zeros(n, np.int32)
        est = np.zeros(n, np.uint64)
        parts = {}
        jobs = [(rp_f, cl_f, i, M, prev_files, a, b) for a, b in ranges(n, 16384)]
        for v0, kk, sz, e, off, ids in pool.imap_unordered(_level_chunk, jobs):
            k[v0:v0 + kk.size] = kk
            size[v0:v0 + kk.size] = sz
            est[v0:v0 + kk.size] = e
            parts[v0] = ids
        off = np.zeros(n + 1, np.int64)
        np.cumsum(size, out=off[1:])
        ids = np.concatenate([parts[v0] for v0 in sorted(parts)]) if parts else np.zeros(0, np.int32)
        del parts
        for f, a in zip(lvl_files, (off, ids, k)):
            np.save(f, a)
        np.save(est_f, est)
        prev_files = lvl_files
        print(f"  {name} level {i} done", flush=True)
    k = np.load(prev_files[2])
    off = np.load(prev_files[0])
    est = np.load(os.path.join(CACHE, f"{name}_M{M}_level{h}_est.npy"))
    return {"est": est, "level": k, "bsize": np.diff(off).astype(np.int32)}


def read_digests():
    rows = {}
    if os.path.exists(DIGESTS):
        with open(DIGESTS) as f:
            for line in f:
                if line.startswith("#") or not line.strip():
                    continue
                p = line.split()
                rows[(p[0], p[1])] = line.rstrip("\n")
    return rows


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--jobs", type=int, default=os.cpu_count() or 4)
    ap.add_argument("--cache", default=None)
    ap.add_argument("cases", nargs="*")
    args = ap.parse_args()
    global CACHE
    if args.cache:
        CACHE = os.path.abspath(args.cache)
        os.environ["KH_ORACLE_CACHE"] = CACHE  # the spawned workers read it too
    os.makedirs(CACHE, exist_ok=True)
    todo = args.cases or list(CASES)
    rows = read_digests()
    ctx = mp.get_context("spawn")
    with ctx.Pool(args.jobs) as pool:
        for case in todo:
            gname, kind, h = CASES[case]
            t0 = time.time()
            out = {"hdeg": run_hdeg, "counts": run_counts, "est": run_est}[kind](pool, gname, h)
            secs = time.time() - t0
            for field, a in out.items():
                np.save(os.path.join(CACHE, f"{case}_{field}.npy"), a)
                rows[(case, field)] = (f"{case} {field} {a.dtype.name} {'x'.join(map(str, a.shape))} "
                                       f"{digest(a)}  # {CITE[kind]}; oracle {secs:.0f} s")
            print(f"{case}: {secs:.0f} s", flush=True)
            with open(DIGESTS, "w") as f:
                f.write("# case field dtype shape sha256  # passage; oracle wall time\n")
                f.write("# written by tests/golden/make_fullsize.py from the CPU oracle only\n")
                for key in sorted(rows):
                    f.write(rows[key] + "\n")


if __name__ == "__main__":
    main()
