"""Benchmark of the batched distance-reporting hot path on GB300.

One step = the whole path over one batch of the mixed-1e7 workload (n = 10^7 points, half
uniform and half in 1,000 Gaussian clusters; m = 10^6 queries at data points with
log-uniform expected counts in [1, 2000]): build the Z-order index from points resident in
HBM (keys + onesweep sort + decode), fit the learned bounds when they are enabled, then
answer the m queries (ranges, bounds, count, scan, write).  value = queries answered per
second of step time.  After the timed steps the same run measures, outside the headline:
the learned-vs-binary query phase, the Hilbert curve, and reports per-step times.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
Under torchrun (N > 1) every rank answers its own independent problem instance (weak
scaling, no data-path collective); rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import workloads  # noqa: E402

METRIC = "queries/s & reported pts/s (learned vs binary search), build pts/s, %HBM peak"
UNIT = "queries/s"
WORKLOAD = "mixed-1e7"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--scale", type=float, default=1.0, help="shrink the workload (tests only)")
    ap.add_argument("--bounds", choices=["learned", "binary"], default=None)
    ap.add_argument("--workload", choices=["mixed-1e7", "mixed-1e8", "uniform-1e5", "normal-1e7",
                                           "paper-uniform", "paper-normal", "paper-skewed", "mixed3d-1e7"],
                    default="mixed-1e7",
                    help="the headline is mixed-1e7; the others are supplementary measurements")
    ap.add_argument("--reorder", type=int, choices=[0, 1, 2], default=None,
                    help="query processing order (0 input, 1 curve, 2 automatic)")
    ap.add_argument("--leaves", type=int, default=None, help="leaf segments of the learned model")
    ap.add_argument("--occupancy", type=int, default=0,
                    help="early-termination quadtree depth (0 = off; the paper uses 12)")
    ap.add_argument("--rel-side", type=float, default=1e-3,
                    help="normal-1e7: disc diameter; paper-*: square window side; relative to the domain side")
    ap.add_argument("--n", type=float, default=1e7, help="paper-*: points")
    ap.add_argument("--m", type=float, default=1e6, help="paper-*: queries (uniformly placed)")
    ap.add_argument("--cover", type=int, choices=[-1, 0, 1, 2], default=-1,
                    help="cover of each query's ball: 0 cells(Q), 1/2 levels finer, -1 autotuned")
    ap.add_argument("--no-extras", action="store_true", help="skip the untimed extra measurements")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def instance_seed(rank: int) -> int:
    """Each rank answers its own instance; rank 0 is the canonical seed of the workload."""
    return 2 + 7919 * rank


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


# --------------------------------------------------------------------------------------
# clocks during the timed region
# --------------------------------------------------------------------------------------

class ClockSampler:
    """nvidia-smi clock and throttle-reason samples (every 50 ms, time-stamped).  Started
    before the warm-up so that the tool's own start-up does not fall inside the timed region;
    only the samples taken between begin() and end() are reported (the nearest ones when the
    region is shorter than the sampling period)."""
    FIELDS = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None
        self.t0 = self.t1 = None

    def start(self):
        fd, self.path = tempfile.mkstemp(prefix="clocks", suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "50"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
            return
        deadline = time.time() + 5.0   # wait for the first sample
        while time.time() < deadline and os.path.getsize(self.path) == 0:
            time.sleep(0.02)

    def begin(self):
        self.t0 = time.time()

    def end(self):
        self.t1 = time.time()

    @staticmethod
    def _stamp(text):
        import datetime
        try:
            return datetime.datetime.strptime(text.strip(), "%Y/%m/%d %H:%M:%S.%f").timestamp()
        except ValueError:
            return None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.1)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 10:
                    rows.append((self._stamp(parts[0]), parts[1:]))
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        t0, t1 = self.t0 or 0.0, self.t1 or float("inf")
        inside = [r for t, r in rows if t is not None and t0 <= t <= t1]
        if len(inside) < 2:   # region shorter than the period: the samples nearest to it
            mid = 0.5 * (t0 + t1)
            stamped = sorted((abs(t - mid), i) for i, (t, r) in enumerate(rows) if t is not None)
            inside = [rows[i][1] for _, i in stamped[:2]] or [r for _, r in rows]
        sm = [float(r[1]) for r in inside if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in inside if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in inside for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons, "samples": len(inside)}


# --------------------------------------------------------------------------------------
# our arm
# --------------------------------------------------------------------------------------

def run_ours(args, rank, world, local):
    import torch
    import paper_2508_19891_gb300 as sfc

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    pg = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
        pg = dist

    wl = make_workload(args, rank)
    n, m = wl.n, wl.m
    dim = wl.meta.get("dim", 2)
    if dim == 3:   # 3-D indexes search with binary bounds only
        bounds = "binary"
    else:
        bounds = args.bounds or ("learned" if learned_available(sfc) else "binary")
    pts = torch.from_numpy(wl.points).to(dev)
    q = torch.from_numpy(wl.queries).to(dev)
    d = torch.from_numpy(wl.delta).to(dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)   # > L2 (129 MB)
    opts = dict(bounds=bounds, profile=1)
    if args.reorder is not None:
        opts["reorder_queries"] = args.reorder
    if args.cover is not None:
        opts["cover_refine"] = args.cover
    if args.leaves is not None:
        opts["leaves"] = args.leaves
    if args.occupancy:
        opts["occupancy_depth"] = args.occupancy
    norm = wl.meta.get("norm", "disc")
    opts["query_norm"] = norm
    if dim == 3:   # 3-D: binary bounds, disc windows; the cover may be cells(Q) or one level finer
        opts = {"profile": 1, "cover_refine": args.cover if args.cover is not None and args.cover < 2 else -1}

    # size the output once (the total is the same for every step) and let the autotuner pick
    # the cover, the scan's chunk size and work-queue batches for this shape
    ix = sfc.sfc_build3(pts, **opts) if dim == 3 else sfc.sfc_build(pts, "z", **opts)
    tuned = sfc.sfc_autotune(ix, q, d)
    off, ids = sfc.query(ix, q, d)
    total = int(off[-1].item())
    ids = torch.empty(max(total, 1), dtype=torch.int32, device=dev)
    off = torch.empty(m + 1, dtype=torch.int64, device=dev)

    def step():
        # the whole build on the same index object (its buffers are reused, so steps allocate
        # nothing): keys, sort, decode (+ model fit), then the query batch
        sfc.sfc_rebuild(ix, pts)
        sfc.sfc_query_batch(ix, q, d, off, ids, capacity=total)

    clocks = ClockSampler(local)
    clocks.start()
    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()

    if pg:
        pg.barrier()
    torch.cuda.synchronize()
    sfc.sfc_profile_read(ix, reset=True)      # drop the warm-up records
    clocks.begin()
    launches0 = sfc.sfc_launch_count()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    for i in range(args.steps):
        flush.fill_(i & 255)                      # evict L2 between timed steps
        ev[i][0].record()
        step()
        ev[i][1].record()
    torch.cuda.synchronize()
    clocks.end()
    launches = sfc.sfc_launch_count() - launches0
    clk = clocks.stop()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    local_ms = sum(step_ms)
    total_ms = max_over_ranks(local_ms, pg, dev)
    # per-step device times of the library's steps (events on the launching stream)
    agg = sfc.sfc_profile_read(ix, reset=True)
    stats = sfc.sfc_query_stats(ix)
    cell_stats = sfc.sfc_query_cell_stats(ix)
    status, bits = sfc.sfc_device_status(ix)
    ix.close()
    if status != 0:
        raise RuntimeError(f"device status {status} bits {bits:#x}")

    ms_per_step = total_ms / args.steps
    value = job_throughput(m, world, ms_per_step)
    hbm_peak, peak_kind = peaks()
    S = stats["scanned"]
    H = stats["hits"]
    dominant, others = query_rooflines(agg, S, H, dim, hbm_peak, peak_kind)
    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "int64", "data": "synthetic",
        "config": {"workload": args.workload, "n": n, "m": m, "dim": dim, "curve": "z", "bounds": bounds,
                   "window": norm,
                   **({"rel_side": args.rel_side} if args.workload.startswith("paper-") or
                      args.workload == "normal-1e7" else {}),
                   "reorder_queries": opts.get("reorder_queries", 2), "autotuned": tuned,
                   "seed": instance_seed(rank), "l2": "flushed between timed steps (256 MB write)",
                   "step": "rebuild of the index (keys+sort+decode) + learned-model fit if enabled + query batch"},
        "roofline": dominant,
        "roofline_other": others,
        "gpu_launches": int(launches),
        "clocks": clk,
        "breakdown": {
            "step_ms": step_ms,
            "phase_ms_per_step": {k: v[1] / args.steps for k, v in agg.items()},
            "build_pts_per_s": n / (agg.get("sort", (1, float("nan")))[1] / args.steps / 1e3),
            "reported_pts_per_s": world * stats["hits"] / (ms_per_step / 1e3),
            "hits_per_step": stats["hits"], "scanned_per_step": S, "chunks": stats["chunks"],
            "scan_amplification": S / max(stats["hits"], 1),
            "cover_cells": cell_stats["cells"], "cells_found_empty": cell_stats["empty"],
        },
    }
    if rank == 0 and not args.no_extras and dim == 2:
        bopts = {"cover_refine": tuned["cover"], "occupancy_depth": args.occupancy, "query_norm": norm}
        if args.leaves is not None:
            bopts["leaves"] = args.leaves
        out["breakdown"].update(extras(sfc, torch, pts, q, d, total, n, m, flush, bopts))
        out["e2e"] = e2e(sfc, torch, wl, total, bounds, args, tuned["cover"])
    elif rank == 0:
        out["e2e"] = e2e(sfc, torch, wl, total, bounds, args, tuned["cover"])
    if rank == 0 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(wl, budget_s=20.0)
    if rank == 0:
        print(json.dumps(out), flush=True)
    if pg:
        pg.barrier()
        pg.destroy_process_group()


def max_over_ranks(local_ms: float, pg=None, device=None) -> float:
    """Timed-region length of the slowest rank (the only cross-rank exchange: timing, not
    data).  With no process group it is the local time."""
    if pg is None:
        return local_ms
    import torch
    t = torch.tensor([local_ms], dtype=torch.float64, device=device if device is not None else "cpu")
    pg.all_reduce(t, op=pg.ReduceOp.MAX)
    pg.barrier()
    return float(t.item())


def job_throughput(m_per_rank: int, world: int, ms_per_step: float) -> float:
    """Queries answered per second by the whole job: every rank answers its own m queries per
    step (weak scaling), and the step time is the slowest rank's."""
    return world * m_per_rank / (ms_per_step / 1e3)


def make_workload(args, rank):
    if args.workload == "mixed-1e8":
        return workloads.mixed_1e8(scale=args.scale, seed=4 + 7919 * rank)
    if args.workload == "uniform-1e5":
        return workloads.uniform_1e5(scale=args.scale, seed=1 + 7919 * rank)
    if args.workload == "mixed3d-1e7":
        return workloads.mixed3d(scale=args.scale, seed=8 + 7919 * rank)
    if args.workload.startswith("paper-"):
        return workloads.paper_static(args.workload[6:], int(args.n), int(args.m), args.rel_side,
                                      seed=7 + 7919 * rank, scale=args.scale)
    if args.workload == "normal-1e7":
        return workloads.normal_uniform_queries(max(2, int(10_000_000 * args.scale)),
                                                max(1, int(1_000_000 * args.scale)), args.rel_side,
                                                seed=6 + 7919 * rank)
    return workloads.mixed_1e7(scale=args.scale, seed=instance_seed(rank))


def learned_available(sfc) -> bool:
    try:
        import torch
        p = torch.zeros((64, 2), dtype=torch.int32, device="cuda")
        p[:, 0] = torch.arange(64, device="cuda")
        ix = sfc.sfc_build(p, "z", bounds="learned")
        ix.close()
        return True
    except Exception:
        return False


def query_rooflines(agg, scanned: int, hits: int, dim: int, hbm_peak: float, peak_kind: str):
    """Roofline objects of the two query kernels (one launch each per step; the small queries
    run inside them), the one with the longer live time first.  count reads the coordinates
    (x, y[, z] as int32) and writes one mask bit per scanned point; write reads the mask bit of
    each scanned point and each hit's id, and writes the id.  agg maps a phase name to
    (launches, total ms) from the CUDA events of the timed steps."""
    kern = []
    for name, phase, alg in (("count_kernel", "count", 4 * dim * scanned + scanned // 8),
                             ("write_kernel", "write", 8 * hits + scanned // 8)):
        runs, ms = agg.get(phase, (0, float("nan")))
        avg = ms / max(runs, 1)
        ach = alg / (avg / 1e3) / 1e9
        kern.append({"kernel": name, "bound": "hbm", "achieved": ach, "peak": hbm_peak, "unit": "GB/s",
                     "frac": ach / hbm_peak,
                     "peak_kind": f"{peak_kind} copy bandwidth (MEASURED_PEAKS.json hbm_gbs)",
                     "traffic": committed_traffic(name, alg), "algorithmic_bytes": alg, "avg_launch_ms": avg})
    kern.sort(key=lambda k: -k["avg_launch_ms"])
    return kern[0], kern[1:]


def committed_traffic(kernel: str, alg_bytes: int):
    """DRAM bytes per launch from the committed ncu summary, if it was taken on the current
    source of the kernel (else null)."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as f:
            t = json.load(f)
        e = t[kernel]
        src = os.path.join(ROOT, "paper_2508_19891_gb300", "csrc", e["source"])
        import hashlib
        h = hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]
        if h != e["source_sha"]:
            return None
        return float(e["dram_bytes_per_launch"])
    except Exception:
        return None


def timed(fn, torch, flush, reps=3):
    best = float("inf")
    for i in range(reps):
        flush.fill_(i)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        fn()
        b.record()
        torch.cuda.synchronize()
        best = min(best, a.elapsed_time(b))
    return best


def extras(sfc, torch, pts, q, d, total, n, m, flush, bopts):
    """Untimed-for-the-headline measurements: query phase with binary vs learned bounds,
    Hilbert build and query, and the learned model's window statistics (indexes built with
    the step's cover and model options, tuned settings applied)."""
    out = {}
    off = torch.empty(m + 1, dtype=torch.int64, device=pts.device)
    ids = torch.empty(max(total, 1), dtype=torch.int32, device=pts.device)
    for curve in ("z", "h"):
        build_ms = timed(lambda: sfc.sfc_build(pts, curve, **bopts).close(), torch, flush)
        ix = sfc.sfc_build(pts, curve, **bopts)
        sfc.sfc_autotune(ix, q, d)
        res = {"build_ms": build_ms, "build_pts_per_s": n / (build_ms / 1e3),
               "cover": sfc.sfc_cover_refine(ix)}
        modes = ["binary"]
        try:
            sfc.sfc_train_model(ix)
            modes.append("learned")
            tr = timed(lambda: sfc.sfc_train_model(ix), torch, flush)
            res["train_ms"] = tr
        except Exception:
            pass
        ref_ids = None
        for mode in modes:
            sfc.sfc_set_bounds_mode(ix, mode)
            qms = timed(lambda: sfc.sfc_query_batch(ix, q, d, off, ids, capacity=total), torch, flush)
            res[f"query_ms_{mode}"] = qms
            res[f"queries_per_s_{mode}"] = m / (qms / 1e3)
            res[f"reported_pts_per_s_{mode}"] = total / (qms / 1e3)
            cur = ids.clone()
            if ref_ids is None:
                ref_ids = cur
            else:
                res["learned_equals_binary"] = bool(torch.equal(cur, ref_ids))
            if mode == "learned":
                res["learned_stats"] = sfc.sfc_model_stats(ix)
        st = sfc.sfc_device_status(ix)
        res["device_status"] = st[0]
        ix.close()
        out[curve] = res
    out["update"] = update_round(sfc, torch, pts, flush)
    return out


def update_round(sfc, torch, pts, flush):
    """One dynamic round shaped like the dynamic workload (delete 5% of the live ids, insert
    10% new points from the same distribution), on the learned Z index: batch sort, merge,
    and the model refit."""
    n = pts.shape[0]
    k_del, k_ins = n // 20, n // 10
    rng = np.random.default_rng(99)
    dels = torch.from_numpy(rng.choice(n, k_del, replace=False).astype(np.int32)).to(pts.device)
    ins = pts[torch.from_numpy(rng.integers(0, n, k_ins)).to(pts.device)].contiguous()
    times = []
    for rep in range(3):
        ix = sfc.sfc_build(pts, "z", bounds="learned")
        torch.cuda.synchronize()
        flush.fill_(rep)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        sfc.sfc_update(ix, ins, dels)
        b.record()
        torch.cuda.synchronize()
        times.append(a.elapsed_time(b))
        ix.close()
    ms = min(times)
    return {"deletes": k_del, "inserts": k_ins, "ms": ms,
            "updated_pts_per_s": (k_del + k_ins) / (ms / 1e3),
            "note": "includes the host validation sync and the learned-model refit"}


def e2e(sfc, torch, wl, total, bounds, args, cover):
    """The same step through the C ABI with host buffers: sfc_build_host + (model fit) +
    sfc_query_batch_host, host->device and device->host copies inside the timed region,
    inputs in pinned host memory."""
    n, m = wl.n, wl.m
    dim = wl.meta.get("dim", 2)
    hp = torch.empty((n, dim), dtype=torch.int32, pin_memory=True).numpy()
    hp[:] = wl.points
    hq = torch.empty((m, dim), dtype=torch.int32, pin_memory=True).numpy()
    hq[:] = wl.queries
    hd = torch.empty(m, dtype=torch.int32, pin_memory=True).numpy()
    hd[:] = wl.delta
    hoff = torch.empty(m + 1, dtype=torch.int64, pin_memory=True).numpy().view(np.uint64)
    hids = torch.empty(max(total, 1), dtype=torch.int32, pin_memory=True).numpy().view(np.uint32)
    times = []
    for i in range(args.warmup + args.steps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        if dim == 3:
            ix = sfc.sfc_build3_host(hp)
        else:
            ix = sfc.sfc_build_host(hp, "z", bounds=bounds, cover_refine=cover, query_norm=wl.meta.get("norm", "disc"))
        sfc.sfc_query_batch_host(ix, hq, hd, total, out_offsets=hoff, out_ids=hids)
        ix.close()
        torch.cuda.synchronize()
        if i >= args.warmup:
            times.append(time.perf_counter() - t0)
    t = sum(times) / len(times)
    return {"value": m / t, "unit": UNIT, "h2d_bytes_per_step": n * 4 * dim + m * 4 * (dim + 1),
            "d2h_bytes_per_step": (m + 1) * 8 + int(hoff[m]) * 4, "ms_per_step": t * 1e3}


# --------------------------------------------------------------------------------------
# the oracle on the host cores (cpu_baseline and the reference arm)
# --------------------------------------------------------------------------------------

def oracle_sample(wl, budget_s: float, threads: int):
    """Oracle build on the whole point set, then as many queries as fit in the remaining
    budget (at least 1000); returns (queries/s for the whole workload, details)."""
    import oracle

    t0 = time.perf_counter()
    dim = wl.meta.get("dim", 2)
    idx = oracle.build3(wl.points) if dim == 3 else oracle.build(wl.points, 30, "z")
    norm = wl.meta.get("norm", "disc")
    tb = time.perf_counter() - t0
    left = max(budget_s - tb, 1.0)
    k = 2000
    done = 0
    tq = 0.0
    while True:
        k = min(k, wl.m - done)
        if k <= 0:
            break
        t1 = time.perf_counter()
        if dim == 3:   # the 3-D oracle runs on one thread
            oracle.query3(idx, wl.queries[done:done + k], wl.delta[done:done + k])
        else:
            oracle.query(idx, wl.queries[done:done + k], wl.delta[done:done + k], threads=threads, norm=norm)
        tq += time.perf_counter() - t1
        done += k
        if tq > left:
            break
        k *= 2
    per_q = tq / done
    t_full = tb + per_q * wl.m
    return wl.m / t_full, {"build_s": tb, "queries_timed": done, "query_s": tq,
                           "extrapolated_step_s": t_full}


def cpu_baseline(wl, budget_s: float):
    threads = os.cpu_count() or 1
    v, det = oracle_sample(wl, budget_s, threads)
    if wl.meta.get("dim", 2) == 3:
        threads = 1
    return {"value": v, "unit": UNIT, "cores": threads, "kind": "oracle",
            "sample": (f"oracle build (qsort, 1 thread) of all {wl.n} points + the first "
                       f"{det['queries_timed']} of {wl.m} queries on {threads} threads; "
                       f"queries/s of a whole step extrapolated from that sample"),
            "detail": det}


def run_reference(args, rank, world):
    if rank != 0:
        return
    wl = make_workload(args, 0)
    threads = 1 if wl.meta.get("dim", 2) == 3 else (os.cpu_count() or 1)
    vals = []
    det = None
    for i in range(args.warmup + args.steps):
        v, det = oracle_sample(wl, budget_s=6.0, threads=threads)
        if i >= args.warmup:
            vals.append(v)
    v = statistics.median(vals)
    t = wl.m / v
    out = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": world,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": t * 1e3,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int64",
           "data": "synthetic", "config": {"workload": args.workload, "n": wl.n, "m": wl.m, "curve": "z",
                                           "window": wl.meta.get("norm", "disc"),
                                           "bounds": "binary (std lower_bound)"},
           "cpu_baseline": {"value": v, "unit": UNIT, "cores": threads, "kind": "oracle",
                            "sample": (f"per step: oracle build of all {wl.n} points + the first "
                                       f"{det['queries_timed']} queries, extrapolated to {wl.m}")},
           "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def main():
    args = parse()
    rank, world, local = dist_env()
    if args.gpus != world and world == 1 and args.gpus > 1:
        print(json.dumps({"error": "run N>1 under torchrun"}), flush=True)
        sys.exit(2)
    if args.impl == "reference":
        run_reference(args, rank, world)
    else:
        run_ours(args, rank, world, local)


if __name__ == "__main__":
    main()
