#!/usr/bin/env python
"""Benchmark of the (k,h)-core hot path on one GB300 (or N replicas).

Default workload (--workload rmat): the R-MAT scale-22 graph (4,194,304
nodes; 16 * 2^22 edge draws with a = 0.57, b = c = 0.19, d = 0.05,
symmetrised, deduplicated, self-loops dropped, ids permuted; graph seed 1003),
eps = 0.5, delta = 0.05 (M = 841), rank seed 1.  One step is one pass of the
hot path over that graph:
  ranks; exact h-degrees at h = 2; adaptive estimates (level recursion and
  Alg. 1) at h = 2, 3 and 4; the sampled (k,3)-core decomposition (Core,
  Alg. 4, bucket-synchronous).
--workload chung_lu runs the Chung-Lu n = 200,000 graph (m ~ 2M, exponent
2.5, maximum expected degree 5,000, graph seed 1002) with, for h = 2 and 3:
ranks, exact h-degrees, fixed-level counts j = 0..10, the adaptive estimate
and the sampled core; then the exact (k,2)-core.

The metric is h-degree updates per second: one update is one completed
(re)computation of one alive node's h-degree, or of its B[., h] and estimate
(a full-graph pass counts n; a refine that stopped early with only a lower
bound does not count).  ms_per_step is the device time of one whole pass.

--impl reference times the CPU oracle (single thread) on a bounded sample of
the same workload: exact h = 2 degrees and Def. 4.1 estimates at h = 2 of a
seeded sample of nodes per step.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

UNIT = "updates/s"
NOMINAL_HBM_GBS = 7900.0  # GB300 HBM3e nominal bandwidth (context beside the measured peak)
EPS, DELTA, RANK_SEED = 0.5, 0.05, 1
J_LO, J_HI = 0, 10
E2E_STEPS = 3  # end-to-end steps (graph upload included), capped to keep the run short

# kernel class -> the kernels it brackets (kh_prof_read kinds)
CLASS_KERNELS = {
    "bfs": "k_hdeg, k_hdeg2_slice, k_hdeg2_small, k_sweep_* (exact h-degrees)",
    "level1": "k_level1, k_level1_heavy (level-1 lists)",
    "levelU": "k_levelU (level >= 2 lists, hashed union with trim)",
    "frontier": "k_mark_nbrs, k_ball_hop, k_stale_*, k_apply_loss",
    "peel": "k_min_alive, k_collect, k_select, k_finish",
}


class Workload:
    """A headline workload: its graph, one step through the C ABI, its config."""

    def __init__(self, key):
        self.key = key
        if key == "rmat":
            self.name = "rmat_scale22_ef16_h2exact_h234estimate_k3core"
            self.metric = "(k,h)-core decomposition on R-MAT scale 22: h-degree updates/s"
            self.graph_desc = ("R-MAT scale 22, edge factor 16, a/b/c/d = .57/.19/.19/.05, "
                               "symmetrised, deduplicated, ids permuted (synthetic stand-in for "
                               "the paper's social and web graphs)")
            self.graph_seed = 1003
            self.step_desc = ("ranks; exact h-degrees at h=2; adaptive estimate at h=2,3,4; "
                              "sampled (k,3)-core")
        else:
            self.name = "chung_lu_n200k_m2M_gamma2.5_h2_h3"
            self.metric = "(k,h)-core decomposition on Chung-Lu n=200k: h-degree updates/s"
            self.graph_desc = "Chung-Lu power law (synthetic stand-in for the paper's social graphs)"
            self.graph_seed = 1002
            self.step_desc = ("per h in (2,3): ranks, exact h-degrees, fixed-level counts j=0..10, "
                              "adaptive estimate, sampled core; plus exact (k,2)-core")

    def make_graph(self):
        from paper_2112_06154_gb300 import graphgen as gg
        if self.key == "rmat":
            return gg.rmat(22, 16, 0.57, 0.19, 0.19, self.graph_seed)
        return gg.chung_lu(200_000, 20, 2.5, 5000, self.graph_seed)

    def config(self, rp, cl, M):
        deg = np.diff(rp)
        return {
            "workload": self.name, "graph": self.graph_desc,
            "n": int(rp.size - 1), "m": int(cl.size // 2), "max_deg": int(deg.max()),
            "isolated": int((deg == 0).sum()), "eps": EPS, "delta": DELTA, "M": int(M),
            "rank_seed": RANK_SEED, "graph_seed": self.graph_seed, "step": self.step_desc,
            "l2": "inputs larger than L2 (col array %d MB) and L2 flushed (512 MB write) "
                  "between timed steps" % (cl.nbytes >> 20),
        }

    def step(self, K, graph, n, out=None):
        """One pass; out=None: host outputs (e2e).  Returns completed updates."""
        dev = out is not None
        o = (lambda k: out[k]) if dev else (lambda k: None)
        updates = 0
        if self.key == "rmat":
            K.kh_set_h(graph, 2)
            K.kh_ranks(graph, o("r"))
            K.kh_hdegree_exact(graph, o("deg"))
            updates += n
            for h in (2, 3, 4):
                K.kh_set_h(graph, h)
                if dev:
                    K.kh_estimate(graph, out["est%d" % h], out["lvl%d" % h], out["bs%d" % h])
                else:
                    K.kh_estimate(graph)
                updates += n
            K.kh_set_h(graph, 3)
            K.kh_core_sampled(graph, o("cs"))
            updates += K.kh_peel_info(graph, False)[2]
            return updates
        for h in (2, 3):
            K.kh_set_h(graph, h)
            K.kh_ranks(graph, o("r"))
            K.kh_hdegree_exact(graph, o("deg"))
            K.kh_sampled_counts(graph, J_LO, J_HI, o("cnt"))
            if dev:
                K.kh_estimate(graph, out["est%d" % h], out["lvl%d" % h], out["bs%d" % h])
            else:
                K.kh_estimate(graph)
            K.kh_core_sampled(graph, o("cs"))
            updates += 3 * n + K.kh_peel_info(graph, False)[2]
        K.kh_set_h(graph, 2)
        K.kh_core_exact(graph, o("ce"))
        updates += K.kh_peel_info(graph, False)[2]
        return updates

    def device_outputs(self, n):
        import torch
        td = lambda *shape, dt: torch.empty(*shape, dtype=dt, device="cuda")
        out = {"r": td(n, dt=torch.uint8), "deg": td(n, dt=torch.int32),
               "cs": td(n, dt=torch.int64), "ce": td(n, dt=torch.int32),
               "cnt": td(n, J_HI - J_LO + 1, dt=torch.int32)}
        for h in (2, 3, 4):
            out["est%d" % h] = td(n, dt=torch.int64)
            out["lvl%d" % h] = td(n, dt=torch.uint8)
            out["bs%d" % h] = td(n, dt=torch.int32)
        return out

    def d2h_bytes(self, n):
        if self.key == "rmat":
            # ranks, degrees, 3 estimates (est, level, |B|), sampled core
            return n * (1 + 4 + 3 * (8 + 1 + 4) + 8)
        nj = J_HI - J_LO + 1
        return 2 * n * (1 + 4 + 4 * nj + 8 + 1 + 4 + 8) + 4 * n


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=2)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", choices=["ours", "reference"], default="ours")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-cpu", action="store_true")
    p.add_argument("--op", choices=["hdeg2", "hdeg3", "counts2", "est2", "est3", "est4",
                                    "sampled2", "sampled3", "sampled4", "exact2"],
                   help="run one operation once on the workload's graph (a target for profilers)")
    p.add_argument("--workload", choices=["rmat", "chung_lu", "rmat_ops", "c2_ops", "batch",
                                          "serve", "dense", "sweep"],
                   default="rmat",
                   help="rmat (default) / chung_lu: headline step; rmat_ops / c2_ops: single "
                        "operations on R-MAT 22 / Chung-Lu 200k; batch: 4096 preferential-attachment "
                        "graphs, batched vs one graph per call; serve: a Poisson request stream "
                        "through the server")
    p.add_argument("--rmat-scale", type=int, default=22,
                   help="--op only: R-MAT scale of the graph (a smaller case for profilers)")
    p.add_argument("--variant", default=None,
                   help="--op hdeg2/counts2 only: force the 2-degree layout: 'cta', 'sliced,S,T' or "
                        "'small,S,T' (sliced, small balls one warp each)")
    p.add_argument("--sweep", default=None,
                   help="--op hdeg2 only: 'off', or a work bin b: sources of 2-hop work >= 2^b - 1 "
                        "go to the bit-parallel sweeps (default: the tuner's choice)")
    p.add_argument("--union", default="auto",
                   help="schedule of the level-union kernel (kh_set_variant KH_OP_LEVEL_UNION): "
                        "auto, stepped, free, grouped or grouped:D (a lane group covers 1/D of "
                        "a list's expected keys)")
    p.add_argument("--prof", action="store_true",
                   help="--op only: bracket the kernel classes and print their times and "
                        "algorithmic bytes")
    p.add_argument("--requests", type=int, default=300)
    p.add_argument("--rate", type=float, default=200.0)
    p.add_argument("--pool", type=int, default=24)
    p.add_argument("--n-max", type=int, default=100_000)
    p.add_argument("--slots", type=int, default=4)
    p.add_argument("--batch-graphs", type=int, default=4096)
    p.add_argument("--exact-graphs", type=int, default=512)
    return p.parse_args()


def apply_union(K, G, args):
    mode = {"auto": K.KH_VAR_AUTO, "stepped": K.KH_LEVELU_STEPPED, "free": K.KH_LEVELU_FREE,
            "grouped": K.KH_LEVELU_GROUPED}
    name, _, div = getattr(args, "union", "auto").partition(":")
    K.kh_set_variant(G, mode[name], int(div or 0), op=K.KH_OP_LEVEL_UNION)


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


class Clocks:
    """nvidia-smi sampling during the timed region."""

    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        sm, smax, power, reasons = [], [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 8:
                continue
            try:
                sm.append(float(f[0]))
                smax.append(float(f[1]))
                power.append(float(f[2]))
            except ValueError:
                continue
            for nm, val in zip(names, f[4:8]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "power_w_max": max(power) if power else None,
                "samples": len(sm), "reasons": sorted(reasons)}


def load_peak():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


def profile_traffic(workload, kind_name, alg_bytes_per_launch):
    """DRAM bytes per launch of a kernel class on a workload, from the committed
    ncu summaries (None when the class is not listed).  A line gives either the
    bytes per launch, or 'ratio R': DRAM bytes per algorithmic byte measured on
    windows of launches, applied to this run's algorithmic bytes per launch."""
    path = os.path.join(ROOT, "profiles", "traffic_per_launch.txt")
    try:
        with open(path) as f:
            for line in f:
                parts = line.split()
                if line.startswith("#") or len(parts) < 3:
                    continue
                if parts[0] == workload and parts[1] == kind_name:
                    if parts[2] == "ratio" and len(parts) >= 4:
                        return float(parts[3]) * alg_bytes_per_launch
                    return float(parts[2])
    except OSError:
        pass
    return None


def aggregate_ranks(ms, updates, world, device):
    """Replicas: the slowest rank's time and the updates of all ranks."""
    if world <= 1:
        return ms, updates
    import torch
    import torch.distributed as dist
    t = torch.tensor([ms, updates], dtype=torch.float64, device=device)
    mx = t[0:1].clone()
    sm = t[1:2].clone()
    dist.all_reduce(mx, op=dist.ReduceOp.MAX)
    dist.all_reduce(sm, op=dist.ReduceOp.SUM)
    return float(mx[0]), float(sm[0])


# ----------------------------------------------------------------- our arm

def run_ours(args):
    import torch
    from paper_2112_06154_gb300 import khcore as K

    wl = Workload(args.workload)
    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:
        torch.cuda.set_device(0)
    dev = torch.cuda.current_device()
    K.load(build_if_missing=True)
    rp, cl = wl.make_graph()
    n = rp.size - 1
    stream = torch.cuda.Stream()
    ctx = K.kh_ctx_create(dev, stream)
    G = K.kh_graph_load_csr(ctx, rp, cl)
    K.kh_set_sampling(G, seed=RANK_SEED, M=0, eps=EPS, delta=DELTA)
    apply_union(K, G, args)
    M = K.kh_get_M(G)
    out = wl.device_outputs(n)
    flush = torch.empty(512 * 1024 * 1024, dtype=torch.uint8, device="cuda")

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()
        torch.cuda.synchronize()

    for _ in range(args.warmup):
        wl.step(K, G, n, out)
        K.kh_sync(G)
    clocks = Clocks(dev if world == 1 else local)
    total_ms = 0.0
    total_updates = 0
    launches0 = K.kh_launch_count(G)
    clocks.start()
    for _ in range(args.steps):
        with torch.cuda.stream(stream):
            flush.zero_()
        barrier()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        total_updates += wl.step(K, G, n, out)
        e1.record(stream)
        barrier()
        total_ms += e0.elapsed_time(e1)
    clk = clocks.stop()
    launches = K.kh_launch_count(G) - launches0

    # e2e: the same step through the C ABI with host buffers: the graph upload
    # from pinned host memory (and its validation), every output read back
    e2e = None
    if not args.no_e2e:
        prp = torch.from_numpy(rp).pin_memory()
        pcl = torch.from_numpy(cl).pin_memory()
        h2d = rp.nbytes + cl.nbytes
        d2h = wl.d2h_bytes(n)
        Gw = K.kh_graph_load_csr(ctx, prp, pcl)  # warm-up
        K.kh_set_sampling(Gw, seed=RANK_SEED, M=0, eps=EPS, delta=DELTA)
        apply_union(K, Gw, args)
        wl.step(K, Gw, n)
        Gw.close()
        barrier()
        t_e2e = 0.0
        upd_e2e = 0
        e2e_steps = max(1, min(args.steps, E2E_STEPS))
        for _ in range(e2e_steps):
            barrier()
            t0 = time.perf_counter()
            Ge = K.kh_graph_load_csr(ctx, prp, pcl)
            K.kh_set_sampling(Ge, seed=RANK_SEED, M=0, eps=EPS, delta=DELTA)
            apply_union(K, Ge, args)
            upd_e2e += wl.step(K, Ge, n)
            K.kh_sync(Ge)
            t_e2e += time.perf_counter() - t0
            Ge.close()
        e2e = {"value": upd_e2e / t_e2e, "unit": UNIT, "h2d_bytes_per_step": int(h2d),
               "d2h_bytes_per_step": int(d2h), "steps": e2e_steps,
               "ms_per_step": 1e3 * t_e2e / e2e_steps,
               "timing": "host wall clock around graph upload (pinned host arrays), the step "
                         "with host outputs, and a stream sync"}

    # roofline: one extra profiled step (kernel classes bracketed with CUDA
    # events on the library's stream, algorithmic bytes counted on the device)
    K.kh_prof_enable(G, True)
    wl.step(K, G, n, out)
    prof = {}
    for kind in range(K.KH_PROF_KINDS):
        ms, nl, byts = K.kh_prof_read(G, kind)
        prof[K.PROF_NAMES[kind]] = {"ms": ms, "launches": nl, "alg_bytes": byts}
    K.kh_prof_enable(G, False)
    dom = max(prof, key=lambda k: prof[k]["ms"])
    d = prof[dom]
    peak, peak_src = load_peak()
    achieved = (d["alg_bytes"] / 1e9) / (d["ms"] / 1e3) if d["ms"] > 0 else 0.0
    traffic = profile_traffic(wl.name, dom, d["alg_bytes"] / max(d["launches"], 1))
    roofline = {"bound": "hbm", "kernel": CLASS_KERNELS.get(dom, dom), "class": dom,
                "achieved": round(achieved, 2), "peak": peak,
                "unit": "GB/s", "frac": round(achieved / peak, 4),
                "nominal_peak": NOMINAL_HBM_GBS,
                "frac_of_nominal": round(achieved / NOMINAL_HBM_GBS, 4),
                "traffic": traffic,
                "alg_bytes_per_launch": d["alg_bytes"] / max(d["launches"], 1),
                "avg_launch_ms": d["ms"] / max(d["launches"], 1),
                "peak_source": f"{peak_src} hbm_gbs (copy)",
                "timing": "kernel-class CUDA events on the library stream, one profiled step "
                          "after the timed region",
                "classes": {k: {"ms": round(v["ms"], 3), "launches": v["launches"],
                                "alg_GB": round(v["alg_bytes"] / 1e9, 3),
                                "GBps": round(v["alg_bytes"] / 1e6 / v["ms"], 1) if v["ms"] else 0}
                            for k, v in prof.items()}}

    total_ms_max, updates_all = aggregate_ranks(total_ms, float(total_updates), world, "cuda")

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        cpu = cpu_baseline(wl, rp, cl, M, samples=4000)
    if rank == 0:
        line = {
            "metric": wl.metric, "value": updates_all / (total_ms_max / 1e3), "unit": UNIT,
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": total_ms_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "int32",
            "data": "synthetic (seeded generator; no dataset)",
            "config": wl.config(rp, cl, M), "roofline": roofline, "cpu_baseline": cpu,
            "e2e": e2e, "gpu_launches": int(launches), "clocks": clk,
            "updates_per_step": total_updates / args.steps,
        }
        print(json.dumps(line), flush=True)
    G.close()
    ctx.close()
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


# ----------------------------------------------------------------- CPU oracle

def oracle_sample(wl, rp, cl, M, count, seed):
    """The oracle on `count` seeded sample nodes of the workload's graph:
    exact h-degrees at h = 2 and the Def. 4.1 estimate at h = 2.  Returns
    (updates, seconds)."""
    import oracle as O
    n = rp.size - 1
    rng = np.random.default_rng(seed)
    vs = np.sort(rng.choice(n, size=min(count, n), replace=False)).astype(np.int32)
    r = O.ranks(n, RANK_SEED)
    t0 = time.perf_counter()
    O.hdegree_some(rp, cl, 2, vs)
    O.estimate_def_some(rp, cl, r, 2, M, vs)
    return 2 * vs.size, time.perf_counter() - t0


def cpu_baseline(wl, rp, cl, M, samples):
    """The oracle as it stands, single-threaded, on a bounded sample."""
    upd, dt = oracle_sample(wl, rp, cl, M, samples, 7)
    return {"value": upd / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"exact h-degrees and Def. 4.1 estimates at h=2 of {samples} seeded sample "
                      f"nodes of the same graph ({dt:.1f} s, single thread)"}


def run_reference(args):
    rank, world, local = dist_env()
    if rank != 0:
        return
    wl = Workload(args.workload if args.workload in ("rmat", "chung_lu") else "rmat")
    import oracle as O
    rp, cl = wl.make_graph()
    n = rp.size - 1
    M = O.budget_M(n, EPS, DELTA)
    per_step = 400
    for i in range(args.warmup):
        oracle_sample(wl, rp, cl, M, 50, 100 + i)
    t = 0.0
    upd = 0
    for i in range(args.steps):
        u, dt = oracle_sample(wl, rp, cl, M, per_step, 1000 + i)
        t += dt
        upd += u
    value = upd / t
    line = {
        "impl": "reference", "metric": wl.metric, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int32",
        "data": "synthetic (seeded generator; no dataset)", "config": wl.config(rp, cl, M),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": f"per step: exact h-degrees and Def. 4.1 estimates at h=2 of "
                                   f"{per_step} seeded sample nodes (single-threaded CPU oracle)"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def run_op(args):
    """One operation on the headline workload's graph, once (a target for ncu)."""
    import torch
    from paper_2112_06154_gb300 import khcore as K
    K.load(build_if_missing=True)
    wl = Workload(args.workload if args.workload in ("rmat", "chung_lu") else "rmat")
    if wl.key == "rmat" and args.rmat_scale != 22:
        from paper_2112_06154_gb300 import graphgen as gg
        rp, cl = gg.rmat(args.rmat_scale, 16, 0.57, 0.19, 0.19, wl.graph_seed)
    else:
        rp, cl = wl.make_graph()
    ctx = K.kh_ctx_create(0)
    G = K.kh_graph_load_csr(ctx, rp, cl)
    K.kh_set_sampling(G, seed=RANK_SEED, M=0, eps=EPS, delta=DELTA)
    apply_union(K, G, args)
    op, h = args.op[:-1], int(args.op[-1])
    K.kh_set_h(G, h)
    if args.variant:
        f = args.variant.split(",")
        if f[0] == "cta":
            K.kh_set_variant(G, K.KH_VAR_CTA)
        else:
            var = K.KH_VAR_SLICED_SMALL if f[0] == "small" else K.KH_VAR_SLICED
            K.kh_set_variant(G, var, int(f[1]), int(f[2]))
    if args.sweep == "off":
        K.kh_set_variant(G, K.KH_SWEEP_OFF, op=K.KH_OP_HDEG2_SWEEP)
    elif args.sweep is not None:
        K.kh_set_variant(G, K.KH_SWEEP_FROM, int(args.sweep), 0, op=K.KH_OP_HDEG2_SWEEP)
    if op in ("hdeg", "counts") and h == 2:
        K.kh_get_variant(G)  # the tuner (if it runs) stays out of the timed call
    if args.prof:
        K.kh_prof_enable(G, True)
    t0 = time.perf_counter()
    fn = {"hdeg": K.kh_hdegree_exact, "counts": lambda g: K.kh_sampled_counts(g, J_LO, J_HI),
          "est": K.kh_estimate, "sampled": K.kh_core_sampled, "exact": K.kh_core_exact}[op]
    fn(G)
    K.kh_sync(G)
    secs = time.perf_counter() - t0
    info = {"op": args.op, "seconds": secs, "launches": K.kh_launch_count(G), "n": int(rp.size - 1)}
    if args.prof:
        info["classes"] = {}
        for kind in range(K.KH_PROF_KINDS):
            ms, nl, byts = K.kh_prof_read(G, kind)
            if nl:
                info["classes"][K.PROF_NAMES[kind]] = {
                    "ms": ms, "launches": nl, "alg_bytes": byts,
                    "per_launch_ms": K.kh_prof_trace(G, kind).tolist()[:8]}
    if op in ("hdeg", "counts") and h == 2:
        info["variant"] = K.kh_get_variant(G)
        info["sweep"] = K.kh_get_variant(G, op=K.KH_OP_HDEG2_SWEEP)[:2]
    print(json.dumps(info), flush=True)
    G.close()
    ctx.close()


def run_ops(args):
    """Single operations on one graph, each timed once after a warm-up call:
    rmat_ops: R-MAT scale 22: exact h-degrees at h=2, adaptive estimates and
              sampled (k,h)-cores at h=2,3,4;
    c2_ops:   Chung-Lu n=200k: exact h-degrees, fixed-level counts and estimates
              at h=2,3, sampled cores at h=2,3,4 and exact cores at h=2,3."""
    import torch
    from paper_2112_06154_gb300 import graphgen as gg
    from paper_2112_06154_gb300 import khcore as K
    K.load()
    rmat = args.workload == "rmat_ops"
    t0 = time.perf_counter()
    rowptr, col = (gg.rmat(22, 16, 0.57, 0.19, 0.19, 1003) if rmat
                   else Workload("chung_lu").make_graph())
    stats = gg.graph_stats(rowptr, col)
    gen_s = time.perf_counter() - t0
    ctx = K.kh_ctx_create(0)
    G = K.kh_graph_load_csr(ctx, rowptr, col)
    K.kh_set_sampling(G, seed=1)
    apply_union(K, G, args)
    out = {"workload": "rmat_scale22_ops" if rmat else "chung_lu_n200k_ops", "impl": "ours",
           "union": args.union, "graph": stats, "M": K.kh_get_M(G), "gen_s": gen_s, "unit": "s",
           "higher_is_better": False}

    def timed(fn, warm=False):
        if warm:
            fn()
        torch.cuda.synchronize()
        t = time.perf_counter()
        r = fn()
        torch.cuda.synchronize()
        return r, time.perf_counter() - t

    K.kh_set_h(G, 2)
    out["hdeg_h2_variant"] = K.kh_get_variant(G)  # tunes first
    K.kh_prof_enable(G, True)
    _, out["hdeg_h2_s"] = timed(lambda: K.kh_hdegree_exact(G))
    ms, _, b = K.kh_prof_read(G, K.KH_PROF_BFS)
    K.kh_prof_enable(G, False)
    out["hdeg_h2_alg_GBps"] = b / 1e6 / ms if ms > 0 else None
    if not rmat:
        K.kh_set_h(G, 3)
        _, out["hdeg_h3_s"] = timed(lambda: K.kh_hdegree_exact(G), True)
        for h in (2, 3):
            K.kh_set_h(G, h)
            _, out[f"counts_h{h}_s"] = timed(lambda: K.kh_sampled_counts(G, J_LO, J_HI), True)
    for h in (2, 3, 4):
        K.kh_set_h(G, h)
        _, out[f"estimate_h{h}_s"] = timed(lambda: K.kh_estimate(G), not rmat)
    for h in (2, 3, 4):
        K.kh_set_h(G, h)
        core, secs = timed(lambda: K.kh_core_sampled(G), not rmat)
        _, rounds, updates = K.kh_peel_info(G, False)
        out[f"core_sampled_h{h}"] = {"s": secs, "rounds": rounds, "updates": updates,
                                     "max_core": int(core.max())}
    if not rmat:
        for h in (2, 3):
            K.kh_set_h(G, h)
            core, secs = timed(lambda: K.kh_core_exact(G), h == 2)
            _, rounds, updates = K.kh_peel_info(G, False)
            out[f"core_exact_h{h}"] = {"s": secs, "rounds": rounds, "updates": updates,
                                       "max_core": int(core.max()), "us_per_round": 1e6 * secs / rounds}
    free, total = torch.cuda.mem_get_info()
    out["device_gib_used"] = (total - free) / 2**30
    print(json.dumps(out), flush=True)
    G.close()
    ctx.close()


def run_dense(args):
    """EstDense (Alg. 7) on the Chung-Lu n=200k graph: the removal order of a
    sampled (k,h)-core (rank seed 1) replayed with fresh ranks (seed 2), h = 2
    and 3, and the exact form along the exact (k,2)-core.  Each call is timed
    once after a warm-up call."""
    import torch
    from paper_2112_06154_gb300 import khcore as K
    K.load()
    rowptr, col = Workload("chung_lu").make_graph()
    ctx = K.kh_ctx_create(0)
    G = K.kh_graph_load_csr(ctx, rowptr, col)
    out = {"workload": "estdense_chung_lu_n200k", "impl": "ours", "unit": "s",
           "higher_is_better": False}

    def timed(fn):
        fn()
        torch.cuda.synchronize()
        t = time.perf_counter()
        r = fn()
        torch.cuda.synchronize()
        return r, time.perf_counter() - t

    for h, exact in ((2, False), (3, False), (2, True)):
        K.kh_set_h(G, h)
        K.kh_set_sampling(G, seed=1)
        (_, secs_core) = timed(lambda: K.kh_core_exact(G) if exact else K.kh_core_sampled(G))
        order, rounds, _ = K.kh_peel_info(G, True)
        if not exact:
            K.kh_set_sampling(G, seed=2)
        (total, size, best), secs = timed(lambda: K.kh_dense(G, exact, order, rounds))
        _, _, updates = K.kh_peel_info(G, False)
        key = f"{'exact' if exact else 'sampled'}_h{h}"
        out[key] = {"dense_s": secs, "core_s": secs_core, "rounds": rounds, "updates": updates,
                    "best_round": best, "best_size": int(size[best]),
                    "best_density": float(total[best]) / (2.0 * float(size[best]))}
    print(json.dumps(out), flush=True)
    G.close()
    ctx.close()


def run_sweep(args):
    """Analogues of Fig. 1 and Fig. 2 (Sec. 8.2, 8.3), on seeded synthetic graphs.
    (1) eps sweep: M from Eq. (buffer); the sampled (k,h)-core's time and its
    relative error |c'(v) - c(v)| / c(v) against the exact core (maximum, the
    paper's measure, and mean) on the Chung-Lu n=200k graph (h=2), and, as Fig. 1
    does at h = 3 and 4, on a collaboration-shaped Chung-Lu graph (n = 18k, mean
    degree 21) and a co-purchase-shaped one (n = 100k, mean degree 5.5, exponent
    2.8); eps goes down to 0.12, where M reaches 12000, the largest hash set a
    CTA's shared memory holds.  (2) hierarchical SBM, n = 10k..100k, h = 2, 3, 4
    at eps = 0.5: the sampled core's time against the number of edges."""
    import torch
    from paper_2112_06154_gb300 import graphgen as gg
    from paper_2112_06154_gb300 import khcore as K
    K.load()
    ctx = K.kh_ctx_create(0)

    def timed(fn):
        torch.cuda.synchronize()
        t = time.perf_counter()
        r = fn()
        torch.cuda.synchronize()
        return r, time.perf_counter() - t

    out = {"workload": "eps_sweep_and_sbm", "impl": "ours", "unit": "s", "higher_is_better": False,
           "eps_sweep": [], "sbm": []}
    collab = gg.chung_lu(18000, 21, 2.5, 1000, 1102)
    copurchase = gg.chung_lu(100000, 5.5, 2.8, 300, 1103)
    cases = [("chung_lu_n200k", Workload("chung_lu").make_graph(), 2, (0.5, 0.35, 0.25)),
             ("collab_n18k", collab, 3, (0.5, 0.4, 0.3, 0.2, 0.15, 0.12)),
             ("collab_n18k", collab, 4, (0.5, 0.4, 0.3, 0.2, 0.15, 0.12)),
             ("copurchase_n100k", copurchase, 3, (0.5, 0.4, 0.3, 0.2, 0.15)),
             ("copurchase_n100k", copurchase, 4, (0.5, 0.4, 0.3, 0.2))]
    for name, (rowptr, col), h, eps_list in cases:
        G = K.kh_graph_load_csr(ctx, rowptr, col)
        K.kh_set_h(G, h)
        K.kh_core_exact(G)  # warm-up
        exact, t_exact = timed(lambda: K.kh_core_exact(G))
        exact = exact.astype(np.float64)
        pos = exact > 0
        for eps in eps_list:
            K.kh_set_sampling(G, seed=1, M=0, eps=eps, delta=0.05)
            sampled, secs = timed(lambda: K.kh_core_sampled(G))
            rel = np.abs(sampled.astype(np.float64)[pos] - exact[pos]) / exact[pos]
            out["eps_sweep"].append({
                "graph": name, "h": h, "eps": eps, "M": K.kh_get_M(G), "sampled_core_s": secs,
                "exact_core_s": t_exact, "max_rel_err": float(rel.max()) if rel.size else 0.0,
                "mean_rel_err": float(rel.mean()) if rel.size else 0.0,
                "frac_above_eps": float((rel > eps).mean()) if rel.size else 0.0,
                "zero_core_mismatches": int((sampled[~pos] != 0).sum())})
        G.close()
    for n in (10000, 25000, 50000, 100000):
        rowptr, col = gg.sbm_hierarchical(n, 1007)
        G = K.kh_graph_load_csr(ctx, rowptr, col)
        K.kh_set_sampling(G, seed=1)
        row = {"n": n, "m": int(col.size // 2), "M": K.kh_get_M(G)}
        for h in (2, 3, 4):
            K.kh_set_h(G, h)
            K.kh_core_sampled(G)  # warm-up
            _, secs = timed(lambda: K.kh_core_sampled(G))
            row[f"h{h}_s"] = secs
        out["sbm"].append(row)
        G.close()
    print(json.dumps(out), flush=True)
    ctx.close()


def run_batch(args):
    """Batched workload: many preferential-attachment graphs (n log-uniform in
    [100, 20000], m uniform in {3..8}, h uniform in {2,3,4}, per-graph M).

    The plain form loads and peels one graph per call; the batched form peels
    all graphs from one packed CSR, each graph with its own h, M and core value
    (kh_graph_load_batch).  Both are timed in full on every graph, and the
    batched results must equal the per-graph ones bit for bit.
      sampled: Core (Alg. 4) on all graphs at their own h;
      exact:   ExactCore at h = 2 on the first --exact-graphs graphs (exact
               peels at h = 3, 4 of these graphs are the O(n^2 m) regime the
               paper's sampling exists to avoid)."""
    import torch
    from paper_2112_06154_gb300 import graphgen as gg
    from paper_2112_06154_gb300 import khcore as K
    K.load(build_if_missing=True)
    G = args.batch_graphs
    t0 = time.perf_counter()
    vtx_off, rp, cl, hs = gg.ba_batch_workload(G)
    gen_s = time.perf_counter() - t0
    n = int(vtx_off[-1])
    ctx = K.kh_ctx_create(0)

    def sub(q):
        a, b = int(vtx_off[q]), int(vtx_off[q + 1])
        return rp[a:b + 1] - rp[a], cl[rp[a]:rp[b]] - a

    def batched(vo, rpb, clb, hpg, fn, force_h=None):
        B = K.kh_graph_load_batch(ctx, vo, rpb, clb, hpg)
        if force_h:
            K.kh_set_h(B, force_h)
        fn(B)  # warm-up: allocation and graph capture
        torch.cuda.synchronize()
        t = time.perf_counter()
        out = fn(B)
        dt = time.perf_counter() - t
        _, rounds, upd = K.kh_peel_info(B, False)
        B.close()
        return out, dt, rounds, upd

    def alone(qs, fn, force_h=None):
        outs = []
        t = time.perf_counter()
        for q in qs:
            Gq = K.kh_graph_load_csr(ctx, *sub(q))
            K.kh_set_h(Gq, int(force_h or hs[q]))
            K.kh_set_sampling(Gq, seed=1, M=0, eps=EPS, delta=DELTA)
            outs.append(fn(Gq))
            Gq.close()
        return outs, time.perf_counter() - t

    # sampled, every graph at its own h
    cs, t_bs, r_bs, u_bs = batched(vtx_off, rp, cl, hs, K.kh_core_sampled)
    outs, t_as = alone(range(G), K.kh_core_sampled)
    same_s = all((o == cs[vtx_off[q]:vtx_off[q + 1]]).all() for q, o in enumerate(outs))
    # exact at h = 2 on a sub-batch
    GE = min(args.exact_graphs, G)
    vo_e = vtx_off[:GE + 1]
    rp_e = rp[:int(vo_e[-1]) + 1]
    cl_e = cl[:int(rp_e[-1])]
    ce, t_be, r_be, u_be = batched(vo_e, rp_e, cl_e, hs[:GE], K.kh_core_exact, force_h=2)
    oute, t_ae = alone(range(GE), K.kh_core_exact, force_h=2)
    same_e = all((o == ce[vtx_off[q]:vtx_off[q + 1]]).all() for q, o in enumerate(oute))
    line = {
        "workload": f"batch_ba{G}", "impl": "ours",
        "metric": "(k,h)-core decompositions of a batch of graphs: batched vs one graph per call",
        "unit": "s", "higher_is_better": False,
        "graphs": G, "n": n, "m": int(cl.size // 2), "h_counts": np.bincount(hs, minlength=5)[2:].tolist(),
        "generation_s": round(gen_s, 1),
        "sampled": {"batched_s": t_bs, "one_graph_per_call_s": t_as, "speedup": t_as / t_bs,
                    "rounds": r_bs, "updates": u_bs, "identical": bool(same_s)},
        "exact_h2": {"graphs": GE, "batched_s": t_be, "one_graph_per_call_s": t_ae,
                     "speedup": t_ae / t_be, "rounds": r_be, "updates": u_be,
                     "identical": bool(same_e)},
        "timing": "wall clock around the call (host outputs); one-graph-per-call includes each "
                  "graph's load, as a caller without batching pays it",
    }
    print(json.dumps(line), flush=True)
    ctx.close()


def serve_pool(count, n_max, seed):
    """Request graphs: half Chung-Lu (n log-uniform in [1000, n_max], mean degree
    uniform in [4, 32], exponent uniform in [2.1, 3.0], maximum expected degree
    sqrt(n * mean degree)), half 2-D grids with 1% shortcut edges (side chosen
    so that n is log-uniform in the same range)."""
    from paper_2112_06154_gb300 import graphgen as gg
    rng = np.random.default_rng(seed)
    pool = []
    for i in range(count):
        n = int(np.exp(rng.uniform(np.log(1000), np.log(n_max))))
        if i % 2 == 0:
            avg = rng.uniform(4, 32)
            gam = rng.uniform(2.1, 3.0)
            pool.append(gg.chung_lu(n, avg, gam, int(np.sqrt(n * avg)), seed + i))
        else:
            a = int(np.sqrt(n))
            pool.append(gg.grid(a, max(n // a, 2), 0.01, seed + i))
    return pool


def run_serve(args):
    """Poisson request stream (rate req/s) of sampled (k,h)-core decompositions,
    h uniform in {2, 3, 4}, through the continuous-batching server with
    --slots concurrent requests, against the same stream with one slot."""
    from paper_2112_06154_gb300 import serve as S
    pool = serve_pool(args.pool, args.n_max, 1005)
    rng = np.random.default_rng(1006)
    gaps = rng.exponential(1.0 / args.rate, args.requests)
    picks = rng.integers(0, len(pool), args.requests)
    hs_r = rng.integers(2, 5, args.requests)
    out = {}
    for slots in sorted({args.slots, 1}, reverse=True):
        srv = S.KhServer(S.gpu_runner(0), slots=slots, mem_budget=96 << 30)
        rp0, cl0 = pool[0]
        srv.submit(rp0, cl0, 2).result()  # warm-up: library load, first allocations
        srv.done.clear()
        t0 = time.perf_counter()
        futs = []
        due = t0
        for i in range(args.requests):
            due += gaps[i]
            now = time.perf_counter()
            if due > now:
                time.sleep(due - now)
            rp, cl = pool[picks[i]]
            futs.append(srv.submit(rp, cl, int(hs_r[i]), arrival=due))
        for f in futs:
            f.result()
        srv.close()
        out[f"slots{slots}"] = srv.latency_stats()
    line = {
        "workload": "serve_poisson", "impl": "ours",
        "metric": "sampled (k,h)-core serving: p50/p99 latency and throughput",
        "requests": args.requests, "rate_rps": args.rate, "pool_graphs": len(pool),
        "n_range": [1000, args.n_max],
        "pool_nodes_mean": float(np.mean([p[0].size - 1 for p in pool])),
        "results": out,
        "throughput_gain": (out[f"slots{args.slots}"]["throughput_rps"] /
                            out["slots1"]["throughput_rps"]) if args.slots != 1 else 1.0,
        "unit": "s", "higher_is_better": False,
    }
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    if args.op:
        run_op(args)
    elif args.workload == "serve" and args.impl == "ours":
        run_serve(args)
    elif args.workload == "batch" and args.impl == "ours":
        run_batch(args)
    elif args.workload in ("rmat_ops", "c2_ops") and args.impl == "ours":
        run_ops(args)
    elif args.workload == "dense" and args.impl == "ours":
        run_dense(args)
    elif args.workload == "sweep" and args.impl == "ours":
        run_sweep(args)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
