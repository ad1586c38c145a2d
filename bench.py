"""Benchmark of the batched distance-reporting hot path on GB300.

Default workload: mixed-1e8, the learned-bounds configuration (n = 10^8 points, half uniform
and half in 1,000 Gaussian clusters, Z order, a 4,096-leaf learned model; m = 10^7 queries
at data points with log-uniform expected counts in [1, 2000]).  One step = the whole path
over one batch: build the index from points resident in HBM (keys + onesweep sort + decode),
fit the learned model, then answer the m queries (ranges, bounds, count, scan, write).
value = queries answered per second of step time.

After the timed steps the same run measures, from the same index: the query phase with
learned bounds, with binary search and with an untrained model, in interleaved repeats
(median, min, max; outputs compared bit for bit); build and reported points per second; the
host link rates; the end-to-end rate through the host-buffer C calls; and the oracle on the
host cores (one thread and all cores).

Other workloads (--workload): mixed-1e7, roads-3e7 (Hilbert order, build + query captured as
one CUDA graph), dynamic-5e7 (a step is one round of deletes, inserts, refit and queries;
the timed steps are the rounds), uniform-1e5, normal-1e7, paper-{uniform,normal,skewed},
mixed3d-1e7.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
Under torchrun (N > 1) every rank answers its own independent problem instance (weak
scaling, no data-path collective); rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import hashlib
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
WORKLOAD = "mixed-1e8"
WORKLOADS = ["mixed-1e8", "mixed-1e7", "roads-3e7", "dynamic-5e7", "uniform-1e5", "normal-1e7",
             "paper-uniform", "paper-normal", "paper-skewed", "mixed3d-1e7"]
# canonical seed of each workload (rank r answers seed + 7919 r)
SEEDS = {"mixed-1e8": 4, "mixed-1e7": 2, "roads-3e7": 3, "dynamic-5e7": 5, "uniform-1e5": 1,
         "normal-1e7": 6, "paper-uniform": 7, "paper-normal": 7, "paper-skewed": 7, "mixed3d-1e7": 8}
NOMINAL_HBM_GBS = 8000.0   # the ~8 TB/s nominal HBM3e figure
WARP_SCHEDULERS_PER_SM = 4  # each issues one warp instruction per cycle


def parse(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--scale", type=float, default=1.0, help="shrink the workload (tests only)")
    ap.add_argument("--bounds", choices=["learned", "binary"], default=None)
    ap.add_argument("--workload", choices=WORKLOADS, default=WORKLOAD,
                    help="the headline is mixed-1e8; the others are supplementary measurements")
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
    ap.add_argument("--tuning", default=None, metavar="CHUNK,BATCH,QBATCH",
                    help="set the scan settings instead of autotuning them (with --cover 0/1/2): "
                         "replays a plain run's choice under a profiler, whose overhead would "
                         "change the autotuner's timings")
    ap.add_argument("--repeats", type=int, default=10,
                    help="interleaved repeats of the learned / binary / untrained query-phase comparison")
    ap.add_argument("--no-extras", action="store_true", help="skip the untimed extra measurements")
    ap.add_argument("--no-e2e", action="store_true", help="skip the end-to-end measurement")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    args = ap.parse_args(argv)
    pinned_tuning(args)   # refuse a malformed --tuning before any work
    return args


def pinned_tuning(args):
    """The scan settings given with --tuning as (chunk, batch, qbatch), else None.  They replace
    the autotuner's timed choice, which also picks the cover, so they need an explicit --cover;
    the dynamic workload tunes its own index and takes none."""
    if not args.tuning:
        return None
    if args.workload == "dynamic-5e7":
        raise SystemExit("--tuning applies to the static workloads")
    if args.cover < 0:
        raise SystemExit("--tuning needs --cover 0, 1 or 2")
    parts = args.tuning.split(",")
    if len(parts) != 3 or not all(p.strip().isdigit() for p in parts):
        raise SystemExit("--tuning takes CHUNK,BATCH,QBATCH (three integers)")
    return tuple(int(p) for p in parts)


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def instance_seed(rank: int, workload: str = WORKLOAD) -> int:
    """Each rank answers its own instance; rank 0 is the canonical seed of the workload."""
    return SEEDS[workload] + 7919 * rank


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
# roofline of the two query kernels
# --------------------------------------------------------------------------------------

# Warp instructions that the method itself needs per 32 scanned points in the count pass:
# one 8-byte load per lane, dx and dy, the two squares as 32x32 -> 64-bit multiply(-add)s,
# the 64-bit compare against delta^2 (two instructions) and the ballot.
COUNT_MIN_WARP_INST_PER_32 = 8


def committed_traffic(kernel: str, workload: str):
    """ncu record of a query kernel at a workload from profiles/traffic.json (DRAM bytes per
    launch and, for the count kernel, warp instructions per scanned point), if it was taken
    on the current source of the kernel (the sha256 of its source files, concatenated in the
    listed order); else None."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as f:
            t = json.load(f)
        e = t[kernel]
        srcs = e["source"] if isinstance(e["source"], list) else [e["source"]]
        hs = hashlib.sha256()
        for name in srcs:
            hs.update(open(os.path.join(ROOT, "paper_2508_19891_gb300", "csrc", name), "rb").read())
        if hs.hexdigest()[:16] != e["source_sha"]:
            return None
        return e["workloads"][workload]
    except Exception:
        return None


def query_rooflines(agg, scanned: int, hits: int, dim: int, hbm_peak: float, peak_kind: str,
                    workload: str = WORKLOAD, sm_count: int = 152, sm_mhz: float = 2070.0):
    """Roofline objects of the two query passes (the small queries run inside them), the one
    with the longer time first.  The count pass is one count_kernel launch; the write pass is
    write_kernel, preceded by write_big_kernel for the chunks of queries split over warps
    (its time and DRAM bytes are the two launches together).

    write_kernel, bound by HBM: the method must read every reported id and write it, 8 B per
    hit (the hit mask is the two-pass implementation's own traffic and is not counted).
    count_kernel, bound by instruction issue (the coordinates mostly come from L2, so the HBM
    roof does not bind): the method needs COUNT_MIN_WARP_INST_PER_32 warp instructions per 32
    scanned points, against an issue peak of 4 warp instructions per SM and cycle.  Both carry
    the DRAM traffic of a committed ncu capture of the same kernel source and workload, as a
    fraction of the measured copy peak (dram_frac) and of the nominal 8 TB/s.
    agg maps a phase name to (launches, total ms) from the CUDA events of the timed steps."""
    out = []
    for name, phase in (("count_kernel", "count"), ("write_kernel", "write")):
        runs, ms = agg.get(phase, (0, float("nan")))
        avg = ms / max(runs, 1)
        rec = committed_traffic(name, workload) or {}
        traffic = rec.get("dram_bytes_per_launch")
        o = {"kernel": name, "avg_launch_ms": avg, "traffic": traffic,
             "traffic_source": rec.get("command") if traffic is not None else None}
        if name == "write_kernel":
            o["launches"] = "write_big_kernel + write_kernel"
        if traffic is not None:
            gbs = traffic / (avg / 1e3) / 1e9
            o.update({"dram_gbs": gbs, "dram_frac": gbs / hbm_peak, "dram_frac_nominal": gbs / NOMINAL_HBM_GBS})
        else:
            o.update({"dram_gbs": None, "dram_frac": None, "dram_frac_nominal": None})
        if name == "write_kernel":
            alg = 8 * hits
            ach = alg / (avg / 1e3) / 1e9
            o.update({"bound": "hbm", "achieved": ach, "peak": hbm_peak, "unit": "GB/s", "frac": ach / hbm_peak,
                      "peak_kind": f"{peak_kind} copy bandwidth (MEASURED_PEAKS.json hbm_gbs)",
                      "algorithmic_bytes": alg, "algorithmic": "8 B per reported id (read + write)"})
        else:
            inst = COUNT_MIN_WARP_INST_PER_32 * scanned / 32.0
            ach = inst / (avg / 1e3) / 1e9
            peak = sm_count * WARP_SCHEDULERS_PER_SM * sm_mhz * 1e6 / 1e9
            o.update({"bound": "alu", "achieved": ach, "peak": peak, "unit": "G warp-inst/s", "frac": ach / peak,
                      "peak_kind": f"issue rate: {sm_count} SMs x {WARP_SCHEDULERS_PER_SM} warp instructions per "
                                   f"cycle at {sm_mhz:.0f} MHz",
                      "algorithmic_inst": inst,
                      "algorithmic": f"{COUNT_MIN_WARP_INST_PER_32} warp instructions per 32 scanned points",
                      "executed_inst_per_32_points": (32 * rec["inst_per_scanned_point"]
                                                      if rec.get("inst_per_scanned_point") else None),
                      "effective_gbs": 4 * dim * scanned / (avg / 1e3) / 1e9})
        out.append(o)
    out.sort(key=lambda k: -k["avg_launch_ms"])
    return out[0], out[1:]


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
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)   # > L2 (129 MB)
    if args.workload == "dynamic-5e7":
        bench = DynamicBench(args, rank, sfc, torch, dev)
    else:
        bench = StaticBench(args, rank, sfc, torch, dev)

    clocks = ClockSampler(local)
    clocks.start()
    for i in range(args.warmup):
        bench.step(i)
    torch.cuda.synchronize()
    if pg:
        pg.barrier()
    torch.cuda.synchronize()
    bench.reset_profile()
    clocks.begin()
    launches0 = sfc.sfc_launch_count()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    for i in range(args.steps):
        flush.fill_(i & 255)                      # evict L2 between timed steps
        ev[i][0].record()
        bench.step(args.warmup + i)
        ev[i][1].record()
    torch.cuda.synchronize()
    clocks.end()
    launches = sfc.sfc_launch_count() - launches0
    clk = clocks.stop()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    total_ms = max_over_ranks(sum(step_ms), pg, dev)
    ms_per_step = total_ms / args.steps
    out = bench.report(step_ms, ms_per_step, world, clk, int(launches))
    if rank == 0 and not args.no_extras:
        out["breakdown"].update(bench.extras(flush))
    if rank == 0 and not args.no_e2e:
        out["e2e"] = bench.e2e()
    bench.close()
    if rank == 0 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(bench.wl, args.workload)
    if rank == 0:
        print(json.dumps(out), flush=True)
    if pg:
        pg.barrier()
        pg.destroy_process_group()


def base_line(args, world, ms_per_step, m_per_step, step_ms, clk, launches, config):
    return {
        "metric": METRIC, "value": job_throughput(m_per_step, world, ms_per_step), "unit": UNIT,
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_per_step,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int64",
        "data": "synthetic", "config": config, "gpu_launches": launches, "clocks": clk,
        "breakdown": {"step_ms": step_ms}}


class StaticBench:
    """Static workloads: a step rebuilds the index over the resident points (keys, sort,
    decode, model fit) and answers the query batch; roads-3e7 replays both as one CUDA graph."""

    def __init__(self, args, rank, sfc, torch, dev):
        self.args, self.sfc, self.torch, self.dev = args, sfc, torch, dev
        self.wl = wl = make_workload(args, rank)
        self.seed = instance_seed(rank, args.workload)
        self.dim = wl.meta.get("dim", 2)
        self.curve = "h" if args.workload == "roads-3e7" else "z"
        self.graph = args.workload == "roads-3e7"
        if self.dim == 3:   # 3-D indexes search with binary bounds only
            self.bounds = "binary"
        else:
            self.bounds = args.bounds or "learned"
        self.pts = torch.from_numpy(wl.points).to(dev)
        self.q = torch.from_numpy(wl.queries).to(dev)
        self.d = torch.from_numpy(wl.delta).to(dev)
        self.norm = wl.meta.get("norm", "disc")
        opts = {"bounds": self.bounds, "profile": 1, "cover_refine": args.cover, "query_norm": self.norm}
        if args.reorder is not None:
            opts["reorder_queries"] = args.reorder
        if args.leaves is not None:
            opts["leaves"] = args.leaves
        if args.occupancy:
            opts["occupancy_depth"] = args.occupancy
        if self.dim == 3:   # binary bounds, disc windows; cover cells(Q) or one level finer
            opts = {"profile": 1, "cover_refine": args.cover if args.cover < 2 else -1}
        self.opts = opts
        # size the output once (the total is the same for every step) and let the autotuner
        # pick the cover, the scan's chunk size and work-queue batches for this shape
        self.ix = sfc.sfc_build3(self.pts, **opts) if self.dim == 3 else sfc.sfc_build(self.pts, self.curve, **opts)
        pinned = pinned_tuning(args)
        if pinned:
            chunk, batch, qbatch = pinned
            sfc.sfc_set_tuning(self.ix, chunk, batch, qbatch)
            self.tuned = {"chunk": chunk, "batch": batch, "qbatch": qbatch, "cover": sfc.sfc_cover_refine(self.ix),
                          "pinned": True}
        else:
            self.tuned = sfc.sfc_autotune(self.ix, self.q, self.d)
        off, ids = sfc.query(self.ix, self.q, self.d)
        self.total = int(off[-1].item())
        del off, ids
        self.ids = torch.empty(max(self.total, 1), dtype=torch.int32, device=dev)
        self.off = torch.empty(wl.m + 1, dtype=torch.int64, device=dev)
        self.g = None
        if self.graph:
            self.g = sfc.sfc_graph_capture(self.ix, self.pts, self.q, self.d, self.off, self.ids, self.total)

    def same_tuning(self, ix):
        """Gives another index of the same shape the scan settings of the timed one: the
        pinned ones under --tuning, else the autotuner's cached choice."""
        if self.tuned.get("pinned"):
            self.sfc.sfc_set_tuning(ix, self.tuned["chunk"], self.tuned["batch"], self.tuned["qbatch"])
        else:
            self.sfc.sfc_autotune(ix, self.q, self.d)

    def step(self, i):
        sfc = self.sfc
        if self.g is not None:
            self.g.launch()
            return
        # the whole build on the same index object (its buffers are reused, so steps allocate
        # nothing): keys, sort, decode (+ model fit), then the query batch
        sfc.sfc_rebuild(self.ix, self.pts)
        sfc.sfc_query_batch(self.ix, self.q, self.d, self.off, self.ids, capacity=self.total)

    def reset_profile(self):
        self.sfc.sfc_profile_read(self.ix, reset=True)

    def report(self, step_ms, ms_per_step, world, clk, launches):
        sfc, torch, wl, args = self.sfc, self.torch, self.wl, self.args
        if self.g is not None:
            # graph replays record no per-step events: one eager step, outside the timed
            # region, gives the phase breakdown
            sfc.sfc_profile_read(self.ix, reset=True)
            sfc.sfc_rebuild(self.ix, self.pts)
            sfc.sfc_query_batch(self.ix, self.q, self.d, self.off, self.ids, capacity=self.total)
            agg = sfc.sfc_profile_read(self.ix, reset=True)
            runs = 1
        else:
            agg = sfc.sfc_profile_read(self.ix, reset=True)
            runs = args.steps
        stats = sfc.sfc_query_stats(self.ix)
        cell_stats = sfc.sfc_query_cell_stats(self.ix)
        status, bits = sfc.sfc_device_status(self.ix)
        if status != 0:
            raise RuntimeError(f"device status {status} bits {bits:#x}")
        hbm_peak, peak_kind = peaks()
        sm_count = torch.cuda.get_device_properties(self.dev).multi_processor_count
        sm_mhz = clk.get("sm_mhz") or 2070.0
        S, H = stats["scanned"], stats["hits"]
        per = {k: (v[0] / runs, v[1] / runs) for k, v in agg.items()}   # per step
        dominant, others = query_rooflines({k: (v[0], v[1]) for k, v in per.items()}, S, H, self.dim,
                                           hbm_peak, peak_kind, args.workload, sm_count, sm_mhz)
        phase = {k: v[1] for k, v in per.items()}
        build_ms = phase.get("sort", float("nan"))
        fit_ms = phase.get("train", 0.0)
        query_ms = sum(v for k, v in phase.items() if k not in ("sort", "train", "occupancy"))
        config = {"workload": args.workload, "n": wl.n, "m": wl.m, "dim": self.dim, "curve": self.curve,
                  "bounds": self.bounds, "window": self.norm,
                  **({"rel_side": args.rel_side} if args.workload.startswith("paper-") or
                     args.workload == "normal-1e7" else {}),
                  **({"leaves": args.leaves or 4096} if self.bounds == "learned" else {}),
                  "reorder_queries": self.opts.get("reorder_queries", 2), "autotuned": self.tuned,
                  "seed": self.seed, "l2": "flushed between timed steps (256 MB write)",
                  "step": ("one CUDA graph replay: " if self.graph else "") +
                          "rebuild of the index (keys+sort+decode) + learned-model fit if enabled + query batch"}
        out = base_line(args, world, ms_per_step, wl.m, step_ms, clk, launches, config)
        out["roofline"] = dominant
        out["roofline_other"] = others
        out["breakdown"].update({
            "phase_ms_per_step": phase,
            "build_ms": build_ms, "fit_ms": fit_ms, "query_phase_ms": query_ms,
            "build_pts_per_s": wl.n / (build_ms / 1e3),
            "build_and_fit_pts_per_s": wl.n / ((build_ms + fit_ms) / 1e3),
            "queries_per_s_query_phase": wl.m / (query_ms / 1e3),
            "reported_pts_per_s": world * H / (ms_per_step / 1e3),
            "reported_pts_per_s_query_phase": H / (query_ms / 1e3),
            "hits_per_step": H, "scanned_per_step": S, "chunks": stats["chunks"],
            "scan_amplification": S / max(H, 1),
            # coordinates of every scanned point plus the read and write of every reported id,
            # over the query phase; above the DRAM rate where overlapping queries share L2
            "algorithmic_gbs_query_phase": (4 * self.dim * S + 8 * H) / (query_ms / 1e3) / 1e9,
            "cover_cells": cell_stats["cells"], "cells_found_empty": cell_stats["empty"],
        })
        return out

    def extras(self, flush):
        out = {}
        if self.dim == 2:
            out["bounds_comparison"] = self.bounds_comparison(flush)
            if not self.graph:
                out["hilbert"] = self.other_curve(flush)
            out["update"] = update_round(self.sfc, self.torch, self.pts, flush)
        out["link"] = link_rates(self.torch, self.dev)
        return out

    def bounds_comparison(self, flush):
        """Query phase (plan + scans + count + write) with learned bounds, binary search and an
        untrained model (the root left at its start, 0 Adam steps), on indexes over the same
        points with the same settings, in `repeats` interleaved rounds (the order rotates every
        round, L2 flushed before each batch).  The outputs of all three are compared bit for
        bit with the binary-search output."""
        sfc, torch = self.sfc, self.torch
        reps = max(1, self.args.repeats)
        if self.bounds != "learned":
            sfc.sfc_train_model(self.ix)
        ix0 = sfc.sfc_build(self.pts, self.curve, **{**self.opts, "bounds": "learned", "train_steps": 0})
        self.same_tuning(ix0)
        sfc.sfc_set_cover(ix0, sfc.sfc_cover_refine(self.ix))
        modes = [("learned", self.ix, "learned"), ("binary", self.ix, "binary"),
                 ("learned_untrained", ix0, "learned")]
        res = {name: {"query_ms": [], "plan_ms": []} for name, _, _ in modes}
        stats = {}
        for r in range(reps):
            for k in range(len(modes)):
                name, index, mode = modes[(k + r) % len(modes)]
                sfc.sfc_set_bounds_mode(index, mode)
                sfc.sfc_profile_read(index, reset=True)
                flush.fill_(r & 255)
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record()
                sfc.sfc_query_batch(index, self.q, self.d, self.off, self.ids, capacity=self.total)
                b.record()
                torch.cuda.synchronize()
                res[name]["query_ms"].append(a.elapsed_time(b))
                agg = sfc.sfc_profile_read(index, reset=True)
                res[name]["plan_ms"].append(agg.get("plan", (0, float("nan")))[1])
                if mode == "learned" and name not in stats:
                    stats[name] = sfc.sfc_model_stats(index)
        # bit-exact outputs
        same = {}
        sfc.sfc_set_bounds_mode(self.ix, "binary")
        sfc.sfc_query_batch(self.ix, self.q, self.d, self.off, self.ids, capacity=self.total)
        ref_off, ref_ids = self.off.clone(), self.ids.clone()
        for name, index, mode in modes:
            if name == "binary":
                continue
            sfc.sfc_set_bounds_mode(index, mode)
            sfc.sfc_query_batch(index, self.q, self.d, self.off, self.ids, capacity=self.total)
            same[name] = bool(torch.equal(self.off, ref_off) and torch.equal(self.ids, ref_ids))
        del ref_off, ref_ids
        sfc.sfc_set_bounds_mode(self.ix, self.bounds)
        st0, _ = sfc.sfc_device_status(ix0)
        ix0.close()
        m = self.wl.m
        out = {"repeats": reps, "order": "interleaved, rotating", "outputs_equal_binary": same,
               "device_status_untrained": st0}
        for name, v in res.items():
            q, p = v["query_ms"], v["plan_ms"]
            out[name] = {"query_ms": {"median": statistics.median(q), "min": min(q), "max": max(q)},
                         "plan_ms": {"median": statistics.median(p), "min": min(p), "max": max(p)},
                         "queries_per_s": m / (statistics.median(q) / 1e3),
                         "reported_pts_per_s": self.total / (statistics.median(q) / 1e3),
                         "samples_query_ms": q}
            if name in stats:
                st = stats[name]
                out[name]["window_mean"] = st["window_sum"] / max(st["endpoints"], 1)
                out[name]["window_misses"] = st["misses"]
                out[name]["endpoints"] = st["endpoints"]
        lq, bq = res["learned"]["query_ms"], res["binary"]["query_ms"]
        out["learned_over_binary_qps"] = statistics.median(bq) / statistics.median(lq)
        out["learned_over_binary_plan"] = (statistics.median(res["binary"]["plan_ms"]) /
                                           statistics.median(res["learned"]["plan_ms"]))
        out["learned_beats_binary_beyond_spread"] = max(lq) < min(bq)
        out["trained_over_untrained_qps"] = statistics.median(res["learned_untrained"]["query_ms"]) / statistics.median(lq)
        return out

    def other_curve(self, flush):
        """Build and query timing on the Hilbert curve (same points and queries)."""
        sfc, torch = self.sfc, self.torch
        opts = {**self.opts, "profile": 0}
        build_ms = timed(lambda: sfc.sfc_build(self.pts, "h", **{**opts, "bounds": "binary"}).close(), torch, flush)
        ix = sfc.sfc_build(self.pts, "h", **opts)
        self.same_tuning(ix)
        res = {"build_ms": build_ms, "build_pts_per_s": self.wl.n / (build_ms / 1e3),
               "cover": sfc.sfc_cover_refine(ix)}
        for mode in (["binary", "learned"] if self.bounds == "learned" else ["binary"]):
            sfc.sfc_set_bounds_mode(ix, mode)
            qms = timed(lambda: sfc.sfc_query_batch(ix, self.q, self.d, self.off, self.ids, capacity=self.total),
                        torch, flush)
            res[f"query_ms_{mode}"] = qms
            res[f"queries_per_s_{mode}"] = self.wl.m / (qms / 1e3)
        res["device_status"] = sfc.sfc_device_status(ix)[0]
        ix.close()
        return res

    def e2e(self):
        """The same step through the C ABI with host buffers: sfc_rebuild_host (points copied in,
        keys, sort, model fit) of one index and sfc_query_batch_host, host->device and
        device->host copies inside the timed region, inputs and outputs in page-locked host
        memory.  The index is made once, before the timed steps, by sfc_build_host."""
        sfc, torch, wl, args = self.sfc, self.torch, self.wl, self.args
        n, m, dim = wl.n, wl.m, self.dim
        hp = torch.empty((n, dim), dtype=torch.int32, pin_memory=True).numpy()
        hp[:] = wl.points
        hq = torch.empty((m, dim), dtype=torch.int32, pin_memory=True).numpy()
        hq[:] = wl.queries
        hd = torch.empty(m, dtype=torch.int32, pin_memory=True).numpy()
        hd[:] = wl.delta
        hoff = torch.empty(m + 1, dtype=torch.int64, pin_memory=True).numpy().view(np.uint64)
        hids = torch.empty(max(self.total, 1), dtype=torch.int32, pin_memory=True).numpy().view(np.uint32)
        cover = self.tuned["cover"]
        if dim == 3:
            ix = sfc.sfc_build3_host(hp, cover_refine=cover)
        else:
            ix = sfc.sfc_build_host(hp, self.curve, bounds=self.bounds, cover_refine=cover, query_norm=self.norm)
        times = []
        for i in range(args.warmup + args.steps):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            sfc.sfc_rebuild_host(ix, hp)
            sfc.sfc_query_batch_host(ix, hq, hd, self.total, out_offsets=hoff, out_ids=hids)
            torch.cuda.synchronize()
            if i >= args.warmup:
                times.append(time.perf_counter() - t0)
        ix.close()
        t = sum(times) / len(times)
        return {"value": m / t, "unit": UNIT, "h2d_bytes_per_step": n * 4 * dim + m * 4 * (dim + 1),
                "d2h_bytes_per_step": (m + 1) * 8 + int(hoff[m]) * 4, "ms_per_step": t * 1e3,
                "ms_min": min(times) * 1e3, "ms_max": max(times) * 1e3}

    def close(self):
        if self.g is not None:
            self.g.close()
        self.ix.close()
        del self.ids


class DynamicBench:
    """dynamic-5e7: base 5*10^7 clustered points; a step is one round (delete 5*10^5 live ids,
    insert 10^6 new points, refit the learned model, answer 10^6 queries at live points).  The
    rounds are precomputed on the host (deletes as ids, queries and radii), so the timed steps
    run the library calls only; the timed steps are consecutive rounds, and with the default
    20 timed steps their sum is the 20-round total."""

    def __init__(self, args, rank, sfc, torch, dev):
        self.args, self.sfc, self.torch, self.dev = args, sfc, torch, dev
        R = args.warmup + args.steps
        self.seed = instance_seed(rank, args.workload)
        dwl = workloads.dynamic_5e7(scale=args.scale, seed=self.seed, rounds=R)
        self.dwl = dwl
        self.bounds = args.bounds or "learned"
        xy_by_id = dwl.base
        alive = np.ones(dwl.base.shape[0], bool)
        cluster = dwl.meta["base_cluster"]
        next_id = dwl.base.shape[0]
        self.rounds = []
        xy_parts, alive_parts, cl_parts = [xy_by_id], [alive], [cluster]
        for r, rd in enumerate(dwl.rounds):
            alive_all = np.concatenate(alive_parts) if len(alive_parts) > 1 else alive_parts[0]
            live = np.nonzero(alive_all)[0]
            dels = live[rd["delete_rank"]].astype(np.uint32)
            alive_all[dels] = False
            k = rd["inserts"].shape[0]
            xy_parts = [np.concatenate(xy_parts + [rd["inserts"]])]
            alive_parts = [np.concatenate([alive_all, np.ones(k, bool)])]
            cl_parts = [np.concatenate(cl_parts + [rd["insert_cluster"]])]
            next_id += k
            livef = np.nonzero(alive_parts[0])[0]
            qs, d = workloads.dynamic_round_queries(dwl, r, xy_parts[0][livef], cl_parts[0][livef])
            self.rounds.append({"ins": torch.from_numpy(rd["inserts"]).to(dev),
                                "dels": torch.from_numpy(dels.view(np.int32)).to(dev),
                                "q": torch.from_numpy(qs).to(dev), "d": torch.from_numpy(d).to(dev),
                                "h_ins": rd["inserts"], "h_dels": dels, "h_q": qs, "h_d": d})
        self.m = dwl.rounds[0]["m"]
        self.wl = workloads.Workload("dynamic-5e7", dwl.base, self.rounds[0]["h_q"], self.rounds[0]["h_d"],
                                     {"seed": self.seed})
        self.base = torch.from_numpy(dwl.base).to(dev)
        self.opts = {"bounds": self.bounds, "profile": 1, "cover_refine": args.cover}
        self.ix = sfc.sfc_build(self.base, "z", **self.opts)
        self.tuned = sfc.sfc_autotune(self.ix, self.rounds[0]["q"], self.rounds[0]["d"])
        self.ix.close()
        self.ix = sfc.sfc_build(self.base, "z", **self.opts)   # fresh index, tuned settings cached
        sfc.sfc_autotune(self.ix, self.rounds[0]["q"], self.rounds[0]["d"])
        self.totals = [0] * len(self.rounds)

    def step(self, i):
        sfc = self.sfc
        r = self.rounds[i]
        sfc.sfc_update(self.ix, r["ins"], r["dels"])
        off, ids = sfc.query(self.ix, r["q"], r["d"])
        self.totals[i] = int(ids.numel())

    def reset_profile(self):
        self.sfc.sfc_profile_read(self.ix, reset=True)

    def report(self, step_ms, ms_per_step, world, clk, launches):
        sfc, args = self.sfc, self.args
        agg = sfc.sfc_profile_read(self.ix, reset=True)
        status, bits = sfc.sfc_device_status(self.ix)
        if status != 0:
            raise RuntimeError(f"device status {status} bits {bits:#x}")
        stats = sfc.sfc_query_stats(self.ix)
        config = {"workload": "dynamic-5e7", "n_base": int(self.dwl.base.shape[0]), "rounds_timed": args.steps,
                  "rounds_warmup": args.warmup, "inserts_per_round": int(self.rounds[0]["h_ins"].shape[0]),
                  "deletes_per_round": int(self.rounds[0]["h_dels"].shape[0]), "m_per_round": self.m,
                  "curve": "z", "bounds": self.bounds, "autotuned": self.tuned, "seed": self.seed,
                  "l2": "flushed between timed steps (256 MB write)",
                  "step": "one round: sfc_update (deletes, inserts, merge, model refit) + query batch"}
        out = base_line(args, world, ms_per_step, self.m, step_ms, clk, launches, config)
        per = {k: v[1] / args.steps for k, v in agg.items()}
        hbm_peak, peak_kind = peaks()
        dom, others = query_rooflines({k: (v[0] / args.steps, v[1] / args.steps) for k, v in agg.items()},
                                      stats["scanned"], stats["hits"], 2, hbm_peak, peak_kind, args.workload)
        out["roofline"] = dom
        out["roofline_other"] = others
        out["breakdown"].update({"phase_ms_per_step": per, "rounds_total_ms": sum(step_ms),
                                 "updates_per_s": (int(self.rounds[0]["h_ins"].shape[0]) +
                                                   int(self.rounds[0]["h_dels"].shape[0])) / (ms_per_step / 1e3),
                                 "last_round_hits": stats["hits"], "last_round_scanned": stats["scanned"]})
        return out

    def extras(self, flush):
        return {"link": link_rates(self.torch, self.dev)}

    def e2e(self):
        """Rounds through the public API with host buffers: the round's inserts and delete ids
        copied in from page-locked memory, sfc_update, then sfc_query_batch_host (queries in,
        offsets and ids out), on a fresh index over the same base."""
        sfc, torch, args = self.sfc, self.torch, self.args
        ix = sfc.sfc_build(self.base, "z", **{**self.opts, "profile": 0})
        sfc.sfc_set_cover(ix, self.tuned["cover"])
        cap = max(max(self.totals), 1)   # the same rounds on the same base give the same totals
        pinned = []
        for r in self.rounds:
            hi = torch.empty(r["h_ins"].shape, dtype=torch.int32, pin_memory=True)
            hi.numpy()[:] = r["h_ins"]
            hd = torch.empty(r["h_dels"].shape[0], dtype=torch.int32, pin_memory=True)
            hd.numpy()[:] = r["h_dels"].view(np.int32)
            pinned.append((hi, hd))
        hoff = torch.empty(self.m + 1, dtype=torch.int64, pin_memory=True).numpy().view(np.uint64)
        hids = torch.empty(cap, dtype=torch.int32, pin_memory=True).numpy().view(np.uint32)
        times, d2h = [], []
        for i, r in enumerate(self.rounds):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            di = pinned[i][0].to(self.dev, non_blocking=True)
            dd = pinned[i][1].to(self.dev, non_blocking=True)
            sfc.sfc_update(ix, di, dd)
            sfc.sfc_query_batch_host(ix, r["h_q"], r["h_d"], cap, out_offsets=hoff, out_ids=hids)
            torch.cuda.synchronize()
            if i >= args.warmup:
                times.append(time.perf_counter() - t0)
                d2h.append((self.m + 1) * 8 + int(hoff[self.m]) * 4)
        ix.close()
        t = sum(times) / len(times)
        r0 = self.rounds[0]
        return {"value": self.m / t, "unit": UNIT,
                "h2d_bytes_per_step": int(r0["h_ins"].nbytes + r0["h_dels"].nbytes + r0["h_q"].nbytes + r0["h_d"].nbytes),
                "d2h_bytes_per_step": int(sum(d2h) / len(d2h)), "ms_per_step": t * 1e3}

    def close(self):
        self.ix.close()


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
    seed = instance_seed(rank, args.workload)
    if args.workload == "mixed-1e8":
        return workloads.mixed_1e8(scale=args.scale, seed=seed)
    if args.workload == "mixed-1e7":
        return workloads.mixed_1e7(scale=args.scale, seed=seed)
    if args.workload == "roads-3e7":
        return workloads.roads_3e7(scale=args.scale, seed=seed)
    if args.workload == "uniform-1e5":
        return workloads.uniform_1e5(scale=args.scale, seed=seed)
    if args.workload == "mixed3d-1e7":
        return workloads.mixed3d(scale=args.scale, seed=seed)
    if args.workload.startswith("paper-"):
        return workloads.paper_static(args.workload[6:], int(args.n), int(args.m), args.rel_side,
                                      seed=seed, scale=args.scale)
    if args.workload == "normal-1e7":
        return workloads.normal_uniform_queries(max(2, int(10_000_000 * args.scale)),
                                                max(1, int(1_000_000 * args.scale)), args.rel_side, seed=seed)
    raise ValueError(args.workload)


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


def update_round(sfc, torch, pts, flush):
    """One batched update on the learned Z index (delete 5% of the live ids, insert 10% new
    points from the same distribution): batch sort, merge, and the model refit."""
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


def link_rates(torch, dev, nbytes: int = 2 << 30):
    """Host link: one cudaMemcpyAsync of 2 GiB between device memory and page-locked host
    memory in each direction, timed with CUDA events (best of 3), and where the host buffer
    lives."""
    d = torch.empty(nbytes, dtype=torch.uint8, device=dev)
    h = torch.empty(nbytes, dtype=torch.uint8, pin_memory=True)
    d.fill_(1)
    h.fill_(2)
    out = {"bytes": nbytes}
    for name, fn in (("d2h", lambda: h.copy_(d, non_blocking=True)), ("h2d", lambda: d.copy_(h, non_blocking=True))):
        best = float("inf")
        for _ in range(3):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            fn()
            b.record()
            torch.cuda.synchronize()
            best = min(best, a.elapsed_time(b))
        out[f"{name}_gbs"] = nbytes / (best / 1e3) / 1e9
    try:
        nodes = sorted(x for x in os.listdir("/sys/devices/system/node") if x.startswith("node") and x[4:].isdigit())
        out["host_numa_nodes"] = len(nodes)
    except Exception:
        out["host_numa_nodes"] = None
    del d, h
    return out


# --------------------------------------------------------------------------------------
# the oracle on the host cores (cpu_baseline and the reference arm)
# --------------------------------------------------------------------------------------

def cpu_model() -> str:
    try:
        r = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10)
        for line in r.stdout.splitlines():
            if line.strip().startswith("Model name:"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.lower().startswith(("model name", "cpu model")):
                    return line.split(":", 1)[1].strip()
    except Exception:
        pass
    return "unknown"


class OracleSample:
    """The oracle (plain C: qsort of (key, id), lower_bound, scalar scan) on the host cores:
    its build of the whole point set, timed once on one thread, and query samples (the first
    k queries of the batch, k grown until one sample takes about `target_s`), timed best of 3
    on one thread and on all cores; queries/s of a whole step (build + m queries) is
    extrapolated from the per-query time of the sample."""

    def __init__(self, wl):
        import oracle
        self.oracle = oracle
        self.wl = wl
        self.dim = wl.meta.get("dim", 2)
        self.norm = wl.meta.get("norm", "disc")
        t0 = time.perf_counter()
        self.idx = oracle.build3(wl.points) if self.dim == 3 else oracle.build(wl.points, 30, "z")
        self.build_s = time.perf_counter() - t0

    def run(self, k: int, threads: int) -> float:
        wl = self.wl
        t1 = time.perf_counter()
        if self.dim == 3:   # the 3-D oracle runs on one thread
            self.oracle.query3(self.idx, wl.queries[:k], wl.delta[:k])
        else:
            self.oracle.query(self.idx, wl.queries[:k], wl.delta[:k], threads=threads, norm=self.norm)
        return time.perf_counter() - t1

    def size_sample(self, threads: int, target_s: float) -> int:
        k = min(1000, self.wl.m)
        while True:
            t = self.run(k, threads)
            if t >= target_s / 4 or k >= self.wl.m:
                return min(self.wl.m, max(k, int(k * target_s / max(t, 1e-6))))
            k = min(self.wl.m, 4 * k)

    def per_query(self, threads: int, target_s: float, reps: int = 3):
        k = self.size_sample(threads, target_s)
        best = min(self.run(k, threads) for _ in range(reps))
        return best / k, k


def cpu_baseline(wl, workload: str):
    cores = os.cpu_count() or 1
    s = OracleSample(wl)
    threads_all = 1 if s.dim == 3 else cores
    pq1, k1 = s.per_query(1, 1.5)
    pqa, ka = s.per_query(threads_all, 1.5)
    m = wl.m
    step_all = s.build_s + pqa * m
    step_1 = s.build_s + pq1 * m
    per = "round (rebuild from scratch + " if workload == "dynamic-5e7" else "step (build + "
    return {"value": m / step_all, "unit": UNIT, "cores": threads_all, "kind": "oracle",
            "cpu_model": cpu_model(), "nproc": cores,
            "sample": (f"oracle build (qsort, 1 thread) of all {wl.n} points timed once ({s.build_s:.2f} s); "
                       f"the first {ka} of {m} queries on {threads_all} threads and the first {k1} on 1 thread, "
                       f"best of 3 each; queries/s of a whole {per}{m} queries) extrapolated from the sample"),
            "one_thread": {"value": m / step_1, "query_s_per_query": pq1, "queries_timed": k1,
                           "queries_per_s_query_only": 1.0 / pq1},
            "all_cores": {"value": m / step_all, "threads": threads_all, "query_s_per_query": pqa,
                          "queries_timed": ka, "queries_per_s_query_only": 1.0 / pqa},
            "build_s": s.build_s}


def run_reference(args, rank, world):
    """The reference arm: the oracle as it stands on the host cores (no GPU).  Its build of
    the whole point set is timed once; each step times a bounded query sample on all cores,
    and the step's queries/s is m / (build + m x the sample's per-query time)."""
    if rank != 0:
        return
    if args.workload == "dynamic-5e7":
        dwl = workloads.dynamic_5e7(scale=args.scale, seed=instance_seed(0, args.workload), rounds=1)
        live = dwl.base
        qs, d = workloads.dynamic_round_queries(dwl, 0, live, dwl.meta["base_cluster"])
        wl = workloads.Workload("dynamic-5e7", live, qs, d, {})
    else:
        wl = make_workload(args, 0)
    s = OracleSample(wl)
    threads = 1 if s.dim == 3 else (os.cpu_count() or 1)
    k = s.size_sample(threads, 1.0)
    vals = []
    for i in range(args.warmup + args.steps):
        t = s.run(k, threads)
        if i >= args.warmup:
            vals.append(wl.m / (s.build_s + t / k * wl.m))
    v = statistics.median(vals)
    t = wl.m / v
    out = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": world,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": t * 1e3,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int64",
           "data": "synthetic", "config": {"workload": args.workload, "n": wl.n, "m": wl.m, "curve": "z",
                                           "window": wl.meta.get("norm", "disc"),
                                           "bounds": "binary (lower_bound)"},
           "cpu_baseline": {"value": v, "unit": UNIT, "cores": threads, "kind": "oracle", "cpu_model": cpu_model(),
                            "sample": (f"oracle build (qsort, 1 thread) of all {wl.n} points timed once "
                                       f"({s.build_s:.2f} s); per step the first {k} queries on {threads} "
                                       f"threads, extrapolated to {wl.m} queries")},
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
