#!/usr/bin/env python3
"""Benchmark of the Mixture Graph hot path on GB300.

One step = one pass of the served hot path over one batch of synthetic input:
  A4  propagate one RGBA fp32 transfer function through the whole graph,
  A6-A8  answer one batch of box-histogram queries (exact u32 histograms,
      persistent batched launch),
  A5  look up one 1920x1080 frame of ray samples in the propagated palette.
The queries run on the main stream and, concurrently on a second stream (no
shared data), the propagation followed by the lookup; a step ends when both
have finished.  Per-kernel rooflines use each kernel timed alone.
The graph build (A1-A3, the paper's offline encoder) runs once per volume
before the timed region and is reported as build_ms.

value = box-histogram queries per second over whole steps (all ranks).
e2e   = the same through the public API with host buffers: boxes, TF and
        samples copied host->device and histograms and looked-up colours
        copied back inside the timed region.
--impl reference times the CPU oracle (brute-force counting) on bounded
samples of the same workload on the host cores.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2009_02702_gb300 import synth  # noqa: E402

METRIC = "box-histogram queries/s & TF propagations/s (HBM GB/s vs peak); p99 latency"
NOMINAL_HBM_GBS = 7900.0   # vendor HBM3e figure; the measured copy peak is the roofline denominator
UNIT = "queries/s"


def parse(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--config", type=int, default=3)
    ap.add_argument("--secondary", type=int, default=2, help="second workload measured the same way (0: none)")
    ap.add_argument("--storage", default="", choices=["", "f32", "f16", "bf16"],
                    help="node value storage of the step's propagation (default: f16 for config 3, else f32)")
    ap.add_argument("--cpu-boxes", type=int, default=1000, help="boxes of the CPU oracle's timed sample")
    ap.add_argument("--dims", default="", help="nx,ny,nz: the config's recipe on a volume of these dims "
                                               "(profiling cases; not a bench workload)")
    ap.add_argument("--queries", type=int, default=0)
    ap.add_argument("--schedule", default="batched", choices=["batched", "plain"])
    ap.add_argument("--chunk", type=int, default=0)
    ap.add_argument("--threads", type=int, default=0)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-plan", action="store_true", help="time direct calls instead of the captured plan")
    ap.add_argument("--no-forms", action="store_true", help="skip the plain/naive/16-bit extra measurements")
    ap.add_argument("--no-serve", action="store_true", help="skip the request-loop (serving mix) measurement")
    ap.add_argument("--no-large", action="store_true", help="skip the cylinder graph measurements")
    ap.add_argument("--no-ext", action="store_true",
                    help="skip ray marching, bitstream, greedy factorisation and error-table measurements")
    ap.add_argument("--serve-requests", type=int, default=0)
    ap.add_argument("--serve-rate", type=float, default=0.0)
    return ap.parse_args(argv)


def workload_config(cfg_index, Q, args, storage="f32"):
    cfg = synth.CONFIGS[cfg_index]
    nx, ny, nz = cfg["dims"]
    return {"workload": "%s (synthetic, seeded; stands in for the paper's volume)" % cfg["name"],
            "volume": "%dx%dx%d uint16" % (nx, ny, nz), "segments": cfg["S"],
            "queries_per_step": Q, "box_sides": "%s 1..%d" % (cfg["box"], cfg["box_max"]),
            "hist": "exact u32, dense Q x S", "schedule": args.schedule,
            "tf": "RGBA fp32 in, node values stored as %s" % storage, "samples_per_step": 1920 * 1080,
            "l2": "flushed between steps (write of a 512 MiB buffer)"}


# --------------------------------------------------------------------------
# clocks during the timed region
# --------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.lines = []
        self.proc = None
        self.th = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return
        self.th = threading.Thread(target=self._read, daemon=True)
        self.th.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        if self.th:
            self.th.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# --------------------------------------------------------------------------
# algorithmic bytes of a query batch (footprint assembly, counted on the host)
# --------------------------------------------------------------------------
def _runs(i, di, dim):
    r = []
    di = min(i + di, dim) - i
    while di > 0:
        a = di.bit_length() - 1
        b = (i & -i).bit_length() - 1 if i else 63
        l = min(a, b)
        r.append(l)
        di -= 1 << l
        i += 1 << l
    return np.array(r, np.int64)


def cube_levels(boxes, dims):
    """Number of footprint-assembly cubes per mip level over all boxes."""
    out = np.zeros(40, np.int64)
    for b in boxes:
        lx = _runs(int(b[0]), int(b[3]), dims[0])
        ly = _runs(int(b[1]), int(b[4]), dims[1])
        lz = _runs(int(b[2]), int(b[5]), dims[2])
        L3 = lx[None, None, :] + ly[None, :, None] + lz[:, None, None]
        lmin = np.minimum(np.minimum(lx[None, None, :], ly[None, :, None]), lz[:, None, None])
        cnt = np.left_shift(1, L3 - 3 * lmin)
        out += np.bincount(lmin.ravel(), weights=cnt.ravel(), minlength=40).astype(np.int64)[:40]
    return out


def measured_traffic(kernel, cfg_i, Q):
    """DRAM bytes per launch from the committed ncu records (profiles/
    traffic.json: one record per kernel and workload), only while the kernel's
    source is the one the counters were taken on (else None)."""
    import hashlib
    try:
        with open(os.path.join(ROOT, "profiles", "traffic.json")) as f:
            recs = json.load(f)["records"]
    except (OSError, KeyError, ValueError):
        return None
    for rec in recs:
        if rec.get("kernel") != kernel or rec.get("config") != cfg_i or rec.get("queries") != Q:
            continue
        try:
            with open(os.path.join(ROOT, rec["source"]), "rb") as f:
                sha = hashlib.sha256(f.read()).hexdigest()[:16]
        except (OSError, KeyError):
            return None
        return rec["dram_bytes_per_launch"] if sha == rec["sha256_16"] else None
    return None


# --------------------------------------------------------------------------
# multi-rank plumbing (one replica per GPU, weak scaling, no data-path exchange)
# --------------------------------------------------------------------------
def rank_env():
    """(world, rank, local_rank) from the torchrun environment (1, 0, 0 alone)."""
    return (int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")),
            int(os.environ.get("LOCAL_RANK", "0")))


def rank_boxes(cfg_i, Q, rank):
    """This rank's own batch of boxes: same recipe, an independent stream per rank."""
    return synth.make_boxes(cfg_i, Q=Q, stream_offset=rank)


def max_over_ranks(x, world, device):
    """The largest x over all ranks (the slowest rank times the job)."""
    if world <= 1:
        return float(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(world, units_per_rank, ms_per_step):
    """Units all ranks processed per second, timed by the slowest rank."""
    return world * units_per_rank / (ms_per_step / 1e3)


# --------------------------------------------------------------------------
# our arm
# --------------------------------------------------------------------------
def load_peak():
    """(HBM GB/s, source) from the driver-written measurement, else the fallback."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def query_kernel_name(S, threads, hist="u32"):
    """The histogram kernel the library launches for S segments and a CTA size
    (a private histogram per warp when it fits, else one per CTA)."""
    per_warp = S * 4 * (2 if hist == "f32" else 1) + 64 * 8 + 16   # histogram and push queue
    warp_mode = S <= 2048 and threads <= 256 and per_warp * (threads // 32) <= 96 * 1024
    return "query_warp_kernel" if warp_mode else "query_batched_kernel"


def query_bytes(boxes_h, dims, S):
    """Algorithmic bytes of one query launch: the box, every footprint cube's
    node ID (uint16 at level 0, uint32 above) and the dense u32 row out."""
    lv = cube_levels(boxes_h, dims)
    id0 = 2 if S <= 65536 else 4
    Q = len(boxes_h)
    return 24 * Q + id0 * int(lv[0]) + 4 * int(lv[1:].sum()) + 4 * Q * S, int(lv.sum()), lv


def build_graph(mg, cfg_i, dev, dims=None):
    """The config's volume (GPU generator for Voronoi volumes, host for the
    cylinders), optionally at other dims, and its graph; returns (graph,
    seconds of volume generation)."""
    import torch
    c = synth.CONFIGS[cfg_i]
    t0 = time.perf_counter()
    if c["kind"] == "voronoi":
        vol = synth.make_volume(cfg_i, device=dev, dims=dims)
    else:
        vol = torch.from_numpy(synth.make_volume(cfg_i, dims=dims)).to(dev)
    torch.cuda.synchronize()
    gen_s = time.perf_counter() - t0
    g = mg.mg_build(vol, c["S"])
    del vol
    return g, gen_s


STORAGE = {"f32": ("torch.float32", 4), "f16": ("torch.float16", 2), "bf16": ("torch.bfloat16", 2)}


def measure_step(mg, g, cfg_i, boxes_h, storage, args, dev, flush, stream, world, peak, peak_src,
                 clocks_index=None, e2e=True):
    """Time whole steps of one workload: the box queries on the main stream
    and, concurrently on a side stream, the TF propagation followed by the
    lookup of one 1920x1080 frame.  Returns the workload's measurements."""
    import torch
    from paper_2009_02702_gb300 import mg as _mg
    cfg = synth.CONFIGS[cfg_i]
    S = cfg["S"]
    dims = tuple(g.info["dims"][0])
    Q = len(boxes_h)
    info = g.info
    dt = _mg._DTYPES[storage][1]
    esz = STORAGE[storage][1]
    tf_h = synth.make_tf(cfg_i, S, 4)
    smp_h = synth.make_samples(cfg_i, dims=dims)
    P = smp_h.shape[0]
    boxes = torch.from_numpy(boxes_h).to(dev)
    tf = torch.from_numpy(tf_h).to(dev)
    smp = torch.from_numpy(smp_h).to(dev)
    vals = torch.empty((g.N, 4), dtype=dt, device=dev)
    hist = torch.empty((Q, S), dtype=torch.uint32, device=dev)
    look = torch.empty((P, 4), dtype=dt, device=dev)
    tune = None
    if args.schedule == "batched" and not args.chunk and not args.threads:
        tune = mg.mg_query_autotune(g, boxes, cache=os.environ.get("MG_AUTOTUNE_CACHE"),
                                    key="%s-Q%d" % (cfg["name"], Q))
    threads = args.threads or (tune or {}).get("block_threads") or 256
    qkw = dict(schedule=args.schedule, chunk_cubes=args.chunk, block_threads=args.threads)
    use_plan = args.schedule == "batched" and not args.no_plan
    plan = mg.QueryPlan(g, max_Q=Q, chunk_cubes=args.chunk, block_threads=args.threads) if use_plan else None

    def query(bx, out, st, pl):
        if pl is not None:
            pl.run(bx, out=out, stream=st)
        else:
            mg.mg_query_boxes(g, bx, out=out, stream=st, **qkw)

    side = torch.cuda.Stream(dev)

    def step(e):
        e[0].record(stream)
        side.wait_event(e[0])
        mg.mg_propagate_tf(g, tf, storage=storage, out=vals, stream=side)
        e[1].record(side)
        mg.mg_render_lookup(g, vals, smp, out=look, stream=side)
        e[2].record(side)
        query(boxes, hist, stream, plan)
        e[3].record(stream)
        stream.wait_event(e[2])
        e[4].record(stream)

    warm = [torch.cuda.Event(enable_timing=True) for _ in range(5)]
    for _ in range(max(args.warmup, 3)):
        step(warm)
    mg.mg_sync_status(g)
    torch.cuda.synchronize()

    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(5)] for _ in range(args.steps)]
    clocks = ClockSampler(clocks_index) if clocks_index is not None else None
    if clocks:
        clocks.start()
        time.sleep(0.3)
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    torch.cuda.synchronize()
    t_wall = time.perf_counter()
    for k in range(args.steps):
        flush.zero_()
        step(ev[k])
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    wall = time.perf_counter() - t_wall
    clk = clocks.stop() if clocks else None
    mg.mg_sync_status(g)
    # stage split of the query from CUDA events the library records: a plan
    # with timing events in its graph (plan stage, main kernel), else the
    # direct call's (plan, main kernel, output); same launch shape, L2 flushed
    qmain = []
    if use_plan:
        plan_t = mg.QueryPlan(g, max_Q=Q, chunk_cubes=args.chunk, block_threads=args.threads, timing=True)
        for k in range(args.steps):
            flush.zero_()
            plan_t.run(boxes, out=hist, stream=stream)
            pm, mm = plan_t.timing()
            qmain.append((pm, mm, None))
        plan_t.close()
    else:
        for k in range(args.steps):
            flush.zero_()
            mg.mg_query_boxes(g, boxes, out=hist, timing=True, **qkw)
            qmain.append(mg.mg_query_timing(g))
    torch.cuda.synchronize()
    step_ms = np.array([e[0].elapsed_time(e[4]) for e in ev])
    prop_ms = np.array([e[0].elapsed_time(e[1]) for e in ev])
    look_ms = np.array([e[1].elapsed_time(e[2]) for e in ev])
    query_ms = np.array([e[0].elapsed_time(e[3]) for e in ev])
    main_ms = np.array([t[1] for t in qmain])
    # propagation and lookup each timed alone (L2 flushed) for their rooflines
    prop_alone = _time(lambda: mg.mg_propagate_tf(g, tf, storage=storage, out=vals), 10, flush, stream)
    tf_pin = torch.from_numpy(tf_h).pin_memory()
    tf_up = torch.empty_like(tf)

    def prop_upload():
        tf_up.copy_(tf_pin, non_blocking=True)
        mg.mg_propagate_tf(g, tf_up, storage=storage, out=vals)
    prop_with_upload = _time(prop_upload, 10, flush, stream)
    look_alone = _time(lambda: mg.mg_render_lookup(g, vals, smp, out=look), 10, flush, stream)
    tot_ms = max_over_ranks(float(step_ms.sum()), world, dev)
    ms_per_step = tot_ms / args.steps
    value = whole_job_rate(world, Q, ms_per_step)

    q_bytes, cubes, _ = query_bytes(boxes_h, dims, S)
    kernel = query_kernel_name(S, threads) if args.schedule == "batched" else "query_plain_kernel"
    achieved = q_bytes / (float(np.mean(main_ms)) / 1e3) / 1e9
    traffic = measured_traffic(kernel, cfg_i, Q)
    n_int = info["num_nodes"] - S
    # edges 8 + weight (4 or 2) + value row out per internal node; TF row in and value row out per source
    prop_bytes = n_int * (8 + (4 if storage == "f32" else 2) + 4 * esz) + S * (16 + 4 * esz)
    prop_gbs = prop_bytes / (prop_alone / 1e3) / 1e9
    look_bytes = P * (16 + 4 + 8 * esz)
    look_gbs = look_bytes / (look_alone / 1e3) / 1e9

    e2e_rec = None
    if e2e:
        e2e_rec = end_to_end(mg, g, boxes_h, tf_h, smp_h, storage, Q, S, P, esz, args, dev, stream, flush, world,
                             use_plan, qkw)
    res = {
        "workload": cfg["name"], "value": value, "ms_per_step": ms_per_step, "queries_per_step": Q,
        "storage": storage,
        "tf_propagations_per_s": 1e3 / prop_alone, "samples_per_s": P / (look_alone / 1e3),
        "latency_ms": {"step_p50": float(np.percentile(step_ms, 50)), "step_p99": float(np.percentile(step_ms, 99)),
                       "query_batch_p50": float(np.percentile(query_ms, 50)),
                       "query_batch_p99": float(np.percentile(query_ms, 99)),
                       "propagate_p50": float(np.percentile(prop_ms, 50)),
                       "propagate_p99": float(np.percentile(prop_ms, 99)),
                       "lookup_p50": float(np.percentile(look_ms, 50))},
        "stages_ms": {"propagate": float(np.mean(prop_ms)), "query": float(np.mean(query_ms)),
                      "query_plan": float(np.mean([t[0] for t in qmain])), "query_main": float(np.mean(main_ms)),
                      "query_rest": float(np.mean(query_ms) - np.mean([t[0] for t in qmain]) - np.mean(main_ms)),
                      "lookup": float(np.mean(look_ms)),
                      "propagate_alone": prop_alone, "propagate_with_tf_upload": prop_with_upload,
                      "lookup_alone": look_alone,
                      "note": "propagate/lookup run concurrently with the query; *_alone timed by themselves; "
                              "query_plan = tile reset + fused plan kernel, query_main = histogram kernel (events "
                              "in a timed copy of the plan's graph), query_rest = the rest of a batch (batch size "
                              "and io slots, launch gaps)" if use_plan else
                              "propagate/lookup run concurrently with the query; *_alone timed by themselves; "
                              "query_rest includes the output stage"},
        "roofline_nominal": {"peak": NOMINAL_HBM_GBS, "unit": "GB/s", "frac": achieved / NOMINAL_HBM_GBS,
                             "propagate_frac": prop_gbs / NOMINAL_HBM_GBS, "lookup_frac": look_gbs / NOMINAL_HBM_GBS},
        "roofline": {"bound": "hbm", "kernel": kernel, "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "peak_source": peak_src + " hbm_gbs (copy, burst)",
                     "traffic": traffic, "algorithmic_bytes_per_launch": q_bytes, "cubes_per_launch": cubes,
                     "kernel_ms": float(np.mean(main_ms))},
        "other_kernels": {"propagate_gbs": prop_gbs, "propagate_frac": prop_gbs / peak, "propagate_bytes": prop_bytes,
                          "propagate_storage": storage,
                          "lookup_gbs": look_gbs, "lookup_frac": look_gbs / peak, "lookup_bytes": look_bytes},
        "graph": {"nodes": info["num_nodes"], "depth": info["depth"], "levels": info["levels"],
                  "build_ms": info["build_ms"], "device_bytes": info["device_bytes"],
                  "max_list": info["max_list"], "pairs": info["pairs"], "lut_entries": info["lut_entries"]},
        "e2e": e2e_rec,
        "autotune": tune,
        "query_path": "captured plan (one CUDA graph launch per batch)" if use_plan else "direct calls",
        "clocks": clk,
        "wall_s_timed": wall,
    }
    # one persistent propagation launch (depth within the single pass), the lookup, and the query:
    # batch size and io slots, tile reset, fused plan kernel, main kernel (plans)
    launches_prop = 1 if info["depth"] + 1 <= 64 else 1 + sum(
        1 for d in range(1, info["depth"] + 1) if info["bucket"][d + 1] > info["bucket"][d])
    if args.schedule == "batched" and use_plan:
        launches_query = 4
    elif args.schedule == "batched":
        nscan = 1 if Q <= 2048 else 3
        launches_query = 1 + (1 if Q <= (1 << 18) else 2 * nscan + 1) + 1 + 1
    else:
        launches_query = Q
    res["gpu_launches"] = args.steps * (launches_prop + launches_query + 1)
    if plan is not None:
        plan.close()
    return res


def end_to_end(mg, g, boxes_h, tf_h, smp_h, storage, Q, S, P, esz, args, dev, stream, flush, world, use_plan,
               qkw):
    """The step through the public API with host buffers: every step copies its
    boxes, TF and samples in from pinned memory and its histograms and colours
    out.  Pipelined: a copy-in stream, a query stream (the steps' query
    batches in step order, so no two share the GPU), a frame stream beside it
    (propagation and lookup, as in `value`) and a copy-out stream, over two
    slots of device buffers, ordered by events, so a step's copies overlap
    its neighbours' kernels.
    Serial: one slot, each step on its own with the L2 flushed before it (the
    footing of `value`)."""
    import torch
    from paper_2009_02702_gb300 import mg as _mg
    dt = _mg._DTYPES[storage][1]
    boxes_p = torch.from_numpy(boxes_h).pin_memory()
    tf_p = torch.from_numpy(tf_h).pin_memory()
    smp_p = torch.from_numpy(smp_h).pin_memory()
    cin, cq, cf, cout = (torch.cuda.Stream(dev) for _ in range(4))

    class Slot:
        """Device buffers of one step in flight (and its own query plan, whose
        buffers a run owns until it ends), with pinned host results."""

        def __init__(self):
            self.boxes = torch.empty((Q, 6), dtype=torch.int32, device=dev)
            self.tf = torch.empty((S, 4), dtype=torch.float32, device=dev)
            self.smp = torch.empty((P, 4), dtype=torch.float32, device=dev)
            self.vals = torch.empty((g.N, 4), dtype=dt, device=dev)
            self.look = torch.empty((P, 4), dtype=dt, device=dev)
            self.hist = torch.empty((Q, S), dtype=torch.uint32, device=dev)
            self.hist_p = torch.empty((Q, S), dtype=torch.uint32).pin_memory()
            self.look_p = torch.empty((P, 4), dtype=dt).pin_memory()
            self.plan = mg.QueryPlan(g, max_Q=Q, chunk_cubes=args.chunk,
                                     block_threads=args.threads) if use_plan else None
            self.ev_in, self.ev_q, self.ev_f, self.ev_out = (torch.cuda.Event() for _ in range(4))
            self.used = False

        def step(self):
            # inputs: once this slot's previous kernels have read them
            if self.used:
                cin.wait_event(self.ev_q)
                cin.wait_event(self.ev_f)
            with torch.cuda.stream(cin):
                self.boxes.copy_(boxes_p, non_blocking=True)
                self.tf.copy_(tf_p, non_blocking=True)
                self.smp.copy_(smp_p, non_blocking=True)
            self.ev_in.record(cin)
            # kernels: after the inputs, and once the previous results are out
            for st_ in (cq, cf):
                st_.wait_event(self.ev_in)
                if self.used:
                    st_.wait_event(self.ev_out)
            if self.plan is not None:
                self.plan.run(self.boxes, out=self.hist, stream=cq)
            else:
                mg.mg_query_boxes(g, self.boxes, out=self.hist, stream=cq, **qkw)
            self.ev_q.record(cq)
            mg.mg_propagate_tf(g, self.tf, storage=storage, out=self.vals, stream=cf)
            mg.mg_render_lookup(g, self.vals, self.smp, out=self.look, stream=cf)
            self.ev_f.record(cf)
            # results out
            cout.wait_event(self.ev_q)
            cout.wait_event(self.ev_f)
            with torch.cuda.stream(cout):
                self.hist_p.copy_(self.hist, non_blocking=True)
                self.look_p.copy_(self.look, non_blocking=True)
            self.ev_out.record(cout)
            self.used = True

        def close(self):
            if self.plan is not None:
                self.plan.close()

    def window(slots, steps, flushed):
        e_start, e_end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e_start.record(stream)
        for st_ in (cin, cq, cf, cout):
            st_.wait_event(e_start)
        ms = 0.0
        for k in range(steps):
            sl = slots[k % len(slots)]
            if flushed:
                # each step alone: flush the L2, then time from its first copy to its last
                flush.zero_()
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(stream)
                for st_ in (cin, cq, cf, cout):
                    st_.wait_event(a)
            sl.step()
            if flushed:
                stream.wait_event(sl.ev_out)
                b.record(stream)
                torch.cuda.synchronize()
                ms += a.elapsed_time(b)
        for st_ in (cin, cq, cf, cout):
            ev_ = torch.cuda.Event()
            ev_.record(st_)
            stream.wait_event(ev_)
        e_end.record(stream)
        torch.cuda.synchronize()
        return ms if flushed else float(e_start.elapsed_time(e_end))

    slots = [Slot() for _ in range(2)]
    for k in range(4):
        slots[k % 2].step()
    torch.cuda.synchronize()
    e_ms = max_over_ranks(window(slots, args.steps, False), world, dev)
    s_ms = max_over_ranks(window(slots[:1], args.steps, True), world, dev)
    for sl in slots:
        sl.close()
    return {"value": whole_job_rate(world, Q, e_ms / args.steps), "unit": UNIT,
            "h2d_bytes_per_step": int(boxes_h.nbytes + tf_h.nbytes + smp_h.nbytes),
            "d2h_bytes_per_step": int(Q * S * 4 + P * 4 * esz), "ms_per_step": e_ms / args.steps,
            "timing": "one window over all steps: copy-in stream, query stream (batches in step order), frame "
                      "stream beside it, copy-out stream, two slots of buffers ordered by events; a step's copies "
                      "overlap its neighbours' kernels",
            "l2": "not flushed in the pipelined window (a step reads far more distinct IDs than the 129 MB L2)",
            "serial_flushed": {"value": whole_job_rate(world, Q, s_ms / args.steps), "unit": UNIT,
                               "ms_per_step": s_ms / args.steps,
                               "timing": "one slot, each step alone: L2 flushed, copies in, kernels, copies out"}}


def run_ours(args):
    import torch
    import torch.distributed as dist
    from paper_2009_02702_gb300 import mg

    world, rank, local = rank_env()
    if world > 1:
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    peak, peak_src = load_peak()
    flush = torch.empty(512 << 20, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev)
    cfg_i = args.config
    cfg = synth.CONFIGS[cfg_i]
    S = cfg["S"]
    Q = args.queries or cfg["queries"]
    dims = cfg["dims"]
    storage = args.storage or ("f16" if cfg_i == 3 else "f32")
    if args.dims:
        dims = tuple(int(v) for v in args.dims.split(","))

    g, gen_s = build_graph(mg, cfg_i, dev, dims=dims if args.dims else None)
    boxes_h = synth.make_boxes(cfg_i, Q=Q, dims=dims, stream_offset=rank) if args.dims else rank_boxes(cfg_i, Q, rank)
    head = measure_step(mg, g, cfg_i, boxes_h, storage, args, dev, flush, stream, world, peak, peak_src,
                        clocks_index=local, e2e=not args.no_e2e)
    head["graph"]["volume_generation_s"] = gen_s
    boxes = torch.from_numpy(boxes_h).to(dev)

    cpu, ref = None, {}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(cfg_i, boxes_h, args.cpu_boxes, keep=ref)

    forms = None
    if not args.no_forms:
        forms = other_forms(mg, g, boxes, boxes_h, Q, S, dims, cfg_i, flush, stream, peak, ref=ref)
        forms["storage_types"] = storage_forms(mg, g, cfg_i, flush, stream, peak)
        if not args.no_ext:
            forms["raymarch"] = raymarch_forms(mg, g, cfg_i, dev, flush, stream)
            forms["bitstream"] = bitstream_forms(mg, g, cfg_i, dev, flush, stream)

    secondary = None
    graphs = {cfg_i: g}
    if args.secondary and rank == 0 and args.secondary != cfg_i:
        c2 = args.secondary
        g2, gen2 = build_graph(mg, c2, dev)
        graphs[c2] = g2
        b2 = synth.make_boxes(c2)
        secondary = measure_step(mg, g2, c2, b2, "f32", args, dev, flush, stream, 1, peak, peak_src,
                                 e2e=not args.no_e2e)
        secondary["graph"]["volume_generation_s"] = gen2
        if not args.no_cpu_baseline:
            secondary["cpu_baseline"] = cpu_baseline(c2, b2, args.cpu_boxes, tf=synth.make_tf(c2, synth.CONFIGS[c2]["S"], 4))

    ext = None
    if not args.no_ext and rank == 0:
        ext = {}
        if secondary is not None:
            ext["error_table_" + synth.CONFIGS[args.secondary]["name"]] = \
                error_table_forms(mg, graphs[args.secondary], args.secondary, dev, flush, stream)
            ext["bitstream_" + synth.CONFIGS[args.secondary]["name"]] = \
                bitstream_forms(mg, graphs[args.secondary], args.secondary, dev, flush, stream)
        ext["greedy"] = greedy_forms(mg, dev, cpu=world == 1 and not args.no_cpu_baseline)

    served = None
    if not args.no_serve and rank == 0:
        served = serving(mg, graphs, args, dev)

    large = None
    if not args.no_large and rank == 0:
        large = cylinder_workload(mg, dev, flush, stream, peak, march=not args.no_ext)

    line = {
        "metric": METRIC, "value": head["value"], "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": max(args.warmup, 3), "ms_per_step": head["ms_per_step"], "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": "u32 counts / %s colours (f32 math)" % storage, "data": "synthetic",
        "config": workload_config(cfg_i, Q, args, storage),
    }
    if args.dims:
        line["config"]["volume"] = "%dx%dx%d uint16 (the recipe at other dims: a profiling case)" % dims
    for k in ("tf_propagations_per_s", "samples_per_s", "latency_ms", "stages_ms", "roofline_nominal", "roofline",
              "other_kernels", "graph", "e2e", "autotune", "query_path", "gpu_launches", "clocks", "wall_s_timed"):
        line[k] = head[k]
    line["forms"] = forms
    line["secondary"] = secondary
    line["serving"] = served
    line["cylinders"] = large
    line["extensions"] = ext
    if cpu is not None:
        line["cpu_baseline"] = cpu
    if rank == 0:
        print(json.dumps(line))
    for c, gg in graphs.items():
        gg.close()
    if world > 1:
        dist.destroy_process_group()


# --------------------------------------------------------------------------
# the other forms the workload is reported in
# --------------------------------------------------------------------------
def _time(fn, reps, flush, stream):
    import torch
    fn()
    torch.cuda.synchronize()
    ts = []
    for _ in range(reps):
        flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        fn()
        b.record(stream)
        torch.cuda.synchronize()
        ts.append(a.elapsed_time(b))
    return float(np.median(ts))


def storage_errors(mg, g, tf, vol_h, dims, S, nsample=1500, seed=5, block=None, max_level=5):
    """Max / mean |colour - fp64 direct sum| of node values stored in fp32,
    fp16 and bf16, over sampled interior voxels of levels 1..max_level (their
    mixture is the count of level-0 IDs in the voxel's footprint).  The
    voxels come from the host volume, or from block(origin, side) (host
    generator) when the volume is not held on the host."""
    import torch
    rng = np.random.default_rng(seed)
    tf64 = tf.detach().cpu().numpy().astype(np.float64)
    vals = {dt: mg.mg_propagate_tf(g, tf, storage=dt).float().cpu().numpy() for dt in ("f32", "f16", "bf16")}
    mips = {}
    errs = {dt: [] for dt in vals}
    for _ in range(nsample):
        l = int(rng.integers(1, max_level + 1))
        e = 1 << l
        X, Y, Z = [int(rng.integers(0, d // e)) for d in dims]
        if block is None:
            sub = vol_h[Z * e:(Z + 1) * e, Y * e:(Y + 1) * e, X * e:(X + 1) * e].ravel()
        else:
            sub = block((X * e, Y * e, Z * e), (e, e, e)).ravel()
        ref = np.bincount(sub, minlength=S).astype(np.float64) @ tf64 / sub.size
        if l not in mips:
            mips[l] = mg.mg_graph_copy_mip(g, l)
        node = mips[l][Z, Y, X]
        for dt, v in vals.items():
            errs[dt].append(np.abs(v[node] - ref).max())
    return {dt: {"max_abs": float(np.max(v)), "mean_abs": float(np.mean(v))} for dt, v in errs.items()}


def error_sample(boxes_h, dims, n, seed):
    """n boxes of the batch spread over its size range: equal numbers from each
    decile of clipped volume (seeded)."""
    d = np.array(dims, np.int64)
    side = np.minimum(boxes_h[:, :3].astype(np.int64) + boxes_h[:, 3:], d) - boxes_h[:, :3]
    vol = side.prod(axis=1)
    order = np.argsort(vol, kind="stable")
    rng = np.random.default_rng(seed)
    parts = np.array_split(order, 10)
    pick = np.concatenate([rng.choice(p, size=min(len(p), n // 10), replace=False) for p in parts])
    return np.sort(pick), vol


def exact_vs_oracle(hist_u32, ref):
    """The GPU's exact histograms (host copy) of the CPU baseline's sampled
    boxes against the oracle's counts of the same boxes (ref: the dict
    cpu_baseline fills)."""
    if not ref:
        return None
    got = hist_u32[ref["pick"]].astype(np.int64)
    return {"boxes": int(len(ref["pick"])), "equal": bool(np.array_equal(got, ref["counts"].astype(np.int64)))}


def other_forms(mg, g, boxes, boxes_h, Q, S, dims, cfg_i, flush, stream, peak, n_err=5000, ref=None):
    """The batch in the other forms: direct calls (u32, f32, f32 with 16-bit
    weights), the f32 forms with their relative l1 error against the exact
    counts on n_err boxes across the size range, the plain one-launch-per-box
    form and the naive level-0 count.  The exact counts themselves are
    checked against the oracle on the CPU baseline's sample (ref)."""
    import torch
    out = {}
    hist = torch.empty((Q, S), dtype=torch.uint32, device=boxes.device)
    histf = torch.empty((Q, S), dtype=torch.float32, device=boxes.device)
    ms = _time(lambda: mg.mg_query_boxes(g, boxes, out=hist), 5, flush, stream)
    hist_h = hist.cpu().numpy()
    out["batched_direct_u32"] = {"queries_per_s": Q / (ms / 1e3), "ms": ms,
                                 "exact_vs_oracle": exact_vs_oracle(hist_h, ref)}
    pick, vol = error_sample(boxes_h, dims, n_err, 21)
    exact = hist_h[pick].astype(np.float64)
    del hist_h
    for name, alpha in (("batched_direct_f32", "f32"), ("batched_direct_f32_alpha_f16", "f16"),
                        ("batched_direct_f32_alpha_bf16", "bf16")):
        ms = _time(lambda: mg.mg_query_boxes(g, boxes, out=histf, hist="f32", alpha=alpha), 5, flush, stream)
        h = histf.cpu().numpy()[pick].astype(np.float64)
        rel = np.abs(h - exact).sum(axis=1) / vol[pick]
        out[name] = {"queries_per_s": Q / (ms / 1e3), "ms": ms,
                     "rel_l1_error_vs_exact": {"max": float(rel.max()), "mean": float(rel.mean()),
                                               "boxes": int(len(pick)),
                                               "box_voxels": [int(vol[pick].min()), int(vol[pick].max())]}}
    n = min(Q, 1000)
    sub = boxes[:n].contiguous()
    hs = torch.empty((n, S), dtype=torch.float32, device=boxes.device)
    ms = _time(lambda: mg.mg_query_boxes(g, sub, out=hs, hist="f32", schedule="plain"), 3, flush, stream)
    out["plain_one_launch_per_box_f32"] = {"queries_per_s": n / (ms / 1e3), "ms": ms, "boxes": n}
    hn = torch.empty((n, S), dtype=torch.uint32, device=boxes.device)
    ms = _time(lambda: mg.mg_query_boxes(g, sub, out=hn, schedule="naive"), 3, flush, stream)
    nv = int(vol[:n].sum())
    out["naive_gpu_level0_u32"] = {"queries_per_s": n / (ms / 1e3), "ms": ms, "boxes": n,
                                   "gbs": 2 * nv / (ms / 1e3) / 1e9, "frac": 2 * nv / (ms / 1e3) / 1e9 / peak}
    return out


def storage_forms(mg, g, cfg_i, flush, stream, peak, nsample=400):
    """Propagation and lookup for each node-value storage type against the HBM
    peak, with the error of each against fp64 on sampled voxels (host volume)."""
    import torch
    c = synth.CONFIGS[cfg_i]
    S = c["S"]
    dev = torch.device("cuda", torch.cuda.current_device())
    info = g.info
    tf_h = synth.make_attribute_tf(cfg_i, S) if cfg_i == 4 else synth.make_tf(cfg_i, S, 4)
    tf = torch.from_numpy(tf_h).to(dev)
    smp = torch.from_numpy(synth.make_samples(cfg_i)).to(dev)
    P = smp.shape[0]
    NI = info["num_nodes"] - S
    r = {}
    for st, dt, esz in (("f32", torch.float32, 4), ("f16", torch.float16, 2), ("bf16", torch.bfloat16, 2)):
        vals = torch.empty((g.N, 4), dtype=dt, device=dev)
        look = torch.empty((P, 4), dtype=dt, device=dev)
        ms_p = _time(lambda: mg.mg_propagate_tf(g, tf, storage=st, out=vals), 10, flush, stream)
        ms_l = _time(lambda: mg.mg_render_lookup(g, vals, smp, out=look), 10, flush, stream)
        pb = NI * (8 + (4 if st == "f32" else 2) + 4 * esz) + S * (16 + 4 * esz)
        lb = P * (16 + 4 + 8 * esz)
        r["propagate_" + st] = {"ms": ms_p, "gbs": pb / ms_p / 1e6, "frac": pb / ms_p / 1e6 / peak, "bytes": pb}
        r["lookup_" + st] = {"ms": ms_l, "samples_per_s": P / (ms_l / 1e3), "gbs": lb / ms_l / 1e6,
                             "frac": lb / ms_l / 1e6 / peak}
    # k transfer functions in one pass (one read of the node table, k*C
    # values written per node) against k single passes
    k = 8
    tfs_h = np.stack([synth.make_attribute_tf(cfg_i, S, frame=j) if cfg_i == 4 else synth.make_tf(cfg_i, S, 4, frame=j)
                      for j in range(k)])
    tfs = torch.from_numpy(tfs_h).to(dev)
    for st, dt, esz in (("f32", torch.float32, 4), ("f16", torch.float16, 2)):
        vk = torch.empty((g.N, k * 4), dtype=dt, device=dev)
        ms = _time(lambda: mg.mg_propagate_tf_multi(g, tfs, storage=st, out=vk), 10, flush, stream)
        pb = NI * (8 + (4 if st == "f32" else 2) + k * 4 * esz) + S * k * (16 + 4 * esz)
        r["propagate_multi_k8_" + st] = {"ms": ms, "ms_per_tf": ms / k, "tfs": k, "gbs": pb / ms / 1e6,
                                         "frac": pb / ms / 1e6 / peak, "bytes": pb,
                                         "speedup_vs_k_single": k * r["propagate_" + st]["ms"] / ms}
        del vk
    vol_h = synth.make_volume(cfg_i)
    r["storage_error_vs_fp64"] = storage_errors(mg, g, tf, vol_h, c["dims"], S, nsample=nsample, seed=11,
                                                max_level=4)
    return r


# --------------------------------------------------------------------------
# ray marching, the bitstream, greedy factorisation and error bars
# --------------------------------------------------------------------------
def selection_tf(cfg_i, S, frac=0.02, seed=31):
    """The config's RGBA TF with all but a seeded fraction of the segments
    made fully transparent (a selection of a few segments, as a user
    highlighting them would set it)."""
    tf = synth.make_tf(cfg_i, S, 4).copy()
    keep = np.random.default_rng(seed).random(S) < frac
    tf[~keep, 3] = 0.0
    return tf


def raymarch_forms(mg, g, cfg_i, dev, flush, stream, reps=3):
    """1920x1080 frames ray-marched through the propagated node values
    (Sec. 4: LOD steps, opacity correction, early termination at 0.99),
    with and without empty-space skipping through the propagated opacity;
    frame time, composited samples per second, and that skipping leaves
    the image bit for bit unchanged."""
    import torch
    c = synth.CONFIGS[cfg_i]
    S = c["S"]
    cam = synth.orbit_camera(cfg_i)
    W, H = cam["width"], cam["height"]
    tfs = {"attribute_tf": synth.make_attribute_tf(cfg_i, S)} if cfg_i == 4 else \
        {"uniform_tf": synth.make_tf(cfg_i, S, 4), "selection_tf_2pct": selection_tf(cfg_i, S)}
    out = {"image": "%dx%d RGBA fp32" % (W, H),
           "camera": "seeded orbit frame 0, 45 deg vertical fov, lattice step 0.5 voxel, lod bias 0, "
                     "early termination at opacity 0.99"}
    img = torch.empty((H, W, 4), dtype=torch.float32, device=dev)
    for name, tf_h in tfs.items():
        vals = mg.mg_propagate_tf(g, torch.from_numpy(tf_h).to(dev))
        opac = vals[:, 3].contiguous()
        row, ref = {}, None
        for ess in (False, True):
            op = opac if ess else None
            ms = _time(lambda: mg.mg_raymarch(g, vals, cam, opacity=op, image=img), reps, flush, stream)
            im, st = mg.mg_raymarch(g, vals, cam, opacity=op, steps=True)
            n = int(st.sum().item())
            row["skip" if ess else "plain"] = {"frame_ms": ms, "frames_per_s": 1e3 / ms, "composited_samples": n,
                                               "samples_per_s": n / (ms / 1e3),
                                               "rays_hit": int((st > 0).sum().item())}
            if ref is None:
                ref = im
            else:
                row["skip_image_identical"] = bool(torch.equal(ref, im))
        mg.mg_sync_status(g)
        row["skip_speedup"] = row["plain"]["frame_ms"] / row["skip"]["frame_ms"]
        row["transparent_segments"] = int((tf_h[:, 3] == 0).sum())
        out[name] = row
        del vals, opac, ref, im, st
    return out


def bitstream_forms(mg, g, cfg_i, dev, flush, stream, reps=5):
    """The graph's bitstream (Sec. 3.3, Table 1): bytes and bits per level-0
    voxel against the raw 16-bit volume and the in-memory graph, GPU encode
    and node-table decode time, and the palette lookup reading node IDs from
    the stream by bit address against the plain lookup (same colours)."""
    import torch
    c = synth.CONFIGS[cfg_i]
    S = c["S"]
    bs = mg.mg_bitstream_write(g)
    n = bs.data.numel()
    vox = int(np.prod(c["dims"]))
    lib = mg.lib()
    enc = _time(lambda: mg._check(lib.mg_bitstream_write(g.handle, bs.data.data_ptr(), n, mg._stream(stream))),
                reps, flush, stream)
    dec = _time(lambda: bs.decode_nodes(stream=stream), reps, flush, stream)
    tf = torch.from_numpy(synth.make_tf(cfg_i, S, 4)).to(dev)
    vals = mg.mg_propagate_tf(g, tf)
    smp = torch.from_numpy(synth.make_samples(cfg_i)).to(dev)
    P = smp.shape[0]
    look = torch.empty((P, 4), dtype=torch.float32, device=dev)
    ms_plain = _time(lambda: mg.mg_render_lookup(g, vals, smp, out=look), reps, flush, stream)
    ms_bs = _time(lambda: bs.lookup(vals, smp, stream=stream), reps, flush, stream)
    same = bool(torch.equal(look, bs.lookup(vals, smp)))
    mg.mg_sync_status(g)
    out = {"bytes": n, "bits_per_voxel": 8.0 * n / vox, "raw_u16_volume_bytes": 2 * vox,
           "ratio_vs_raw_u16": 2.0 * vox / n, "graph_device_bytes": g.info["device_bytes"],
           "encode_ms": enc, "encode_gbs": n / enc / 1e6, "decode_nodes_ms": dec,
           "lookup_plain_ms": ms_plain, "lookup_bitstream_ms": ms_bs,
           "lookup_bitstream_samples_per_s": P / (ms_bs / 1e3), "lookup_same_colours": same, "samples": P}
    del bs, vals, smp, look
    return out


def _hist_rel_l1(h, exact, vox):
    rel = np.abs(h - exact).sum(axis=1) / np.maximum(vox, 1)
    return {"max": float(rel.max()), "mean": float(rel.mean())}


def greedy_forms(mg, dev, cpu=True):
    """Greedy factorisation on the GPU (Sec. 3.3, Sec. 3.7) on the 64^3
    Voronoi config: nodes N and depth D of phi_1 and phi_2 at b = 0 (exact)
    and b = 5, 7, 9 bits against the pairwise graph; the quantised graphs'
    box histograms (fp32 push) against the exact counts; their table-summed
    histograms with Eq. 17 error bars against the realised error; GPU time
    against the oracle's on the host cores (cpu).  Then the same for phi_2,
    b = 9 on the 512x512x384 config (GPU only)."""
    import torch
    out = {}
    for ci, bits, strategies in ((1, (0, 5, 7, 9), ("occurrence", "reduction")), (2, (9,), ("reduction",))):
        c = synth.CONFIGS[ci]
        S = c["S"]
        vol = synth.make_volume(ci, device=dev)
        torch.cuda.synchronize()
        g = mg.mg_build(vol, S)
        info = g.info
        boxes_h = synth.make_boxes(ci)[:1000]
        boxes = torch.from_numpy(boxes_h).to(dev)
        exact = mg.mg_query_boxes(g, boxes).cpu().numpy().astype(np.float64)
        d = np.array(c["dims"], np.int64)
        vox = (np.minimum(boxes_h[:, :3].astype(np.int64) + boxes_h[:, 3:], d) - boxes_h[:, :3]).prod(axis=1)
        res = {"pairwise": {"nodes": info["num_nodes"], "depth": info["depth"], "build_ms": info["build_ms"]},
               "boxes": int(len(boxes_h))}
        for strategy in strategies:
            for b in bits:
                key = "%s_b%d" % ("phi1" if strategy == "occurrence" else "phi2", b)
                try:
                    t0 = time.perf_counter()
                    r = mg.mg_factor_greedy(vol, S, strategy=strategy, tau=3, bitrate=b, graph=b > 0)
                    wall = time.perf_counter() - t0
                except mg.MGError as e:
                    res[key] = {"error": str(e)}
                    continue
                row = {"nodes": r["N"], "depth": r["D"], "nodes_vs_pairwise": r["N"] / info["num_nodes"],
                       "stage1_picks": int(len(r["picks"])), "stage2_waves": r["waves"], "gpu_ms": r["ms"],
                       "wall_s": wall}
                if b > 0:
                    gq = r["graph"]
                    hf = mg.mg_query_boxes(gq, boxes, hist="f32").cpu().numpy().astype(np.float64)
                    row["box_rel_l1_error_fp32_push"] = _hist_rel_l1(hf, exact, vox)
                    hl, el = mg.mg_query_lut(gq, boxes)
                    hl, el = hl.cpu().numpy(), el.cpu().numpy()
                    dev_ = np.abs(hl - exact)
                    row["box_rel_l1_error_table"] = _hist_rel_l1(hl, exact, vox)
                    nz = el > 0
                    row["error_bars"] = {"mean_bar_over_box_voxels": float((el.sum(axis=1) / vox).mean()),
                                         "realised_within_1_bar": float((dev_ <= el + 1e-9).mean()),
                                         "realised_within_2_bars": float((dev_ <= 2 * el + 1e-9).mean()),
                                         "bins_with_bar": float(nz.mean())}
                    mg.mg_sync_status(gq)
                    gq.close()
                res[key] = row
        if ci == 1 and cpu:
            res["cpu_baseline"] = greedy_cpu_baseline(ci)
        out[c["name"]] = res
        g.close()
        del vol
    return out


def error_table_forms(mg, g, cfg_i, dev, flush, stream, reps=5):
    """The mixture table of an exact graph (Sec. 3.5-3.6): entries, GPU
    build time, and the table-summed fp64 box query against the exact u32
    query on the config's boxes."""
    import torch
    c = synth.CONFIGS[cfg_i]
    S = c["S"]
    t0 = time.perf_counter()
    off, src, mu, dmu = mg.mg_error_table(g)
    build_s = time.perf_counter() - t0
    boxes_h = synth.make_boxes(cfg_i)
    boxes = torch.from_numpy(boxes_h).to(dev)
    Q = boxes_h.shape[0]
    ms_lut = _time(lambda: mg.mg_query_lut(g, boxes, errors=False, stream=stream), reps, flush, stream)
    hist = torch.empty((Q, S), dtype=torch.uint32, device=dev)
    ms_u32 = _time(lambda: mg.mg_query_boxes(g, boxes, out=hist), reps, flush, stream)
    hl, _ = mg.mg_query_lut(g, boxes, errors=False)
    diff = float(np.abs(hl.cpu().numpy() - hist.cpu().numpy().astype(np.float64)).max())
    mg.mg_sync_status(g)
    return {"entries": int(off[-1]), "entries_per_node": float(off[-1]) / g.N, "build_and_copy_s": build_s,
            "query_table_f64_ms": ms_lut, "query_table_queries_per_s": Q / (ms_lut / 1e3),
            "query_u32_ms": ms_u32, "table_max_abs_diff_vs_exact": diff, "boxes": Q}


# --------------------------------------------------------------------------
# the cylinder graph: many segments, attribute TF, bf16 frames
# --------------------------------------------------------------------------
def cylinder_workload(mg, dev, flush, stream, peak, march=True):
    """The cylinder graph (15,917 segments, 8.9 M nodes): propagation and
    lookup per storage type against the HBM peak, errors against fp64 on
    sampled voxels, and a 10,000-box batch through the CTA-shared histogram
    kernel, with its own roofline."""
    import torch
    cfg_i = 4
    c = synth.CONFIGS[cfg_i]
    S = c["S"]
    g, gen_s = build_graph(mg, cfg_i, dev)
    info = g.info
    r = {"workload": c["name"], "nodes": info["num_nodes"], "depth": info["depth"], "levels": info["levels"],
         "build_ms": info["build_ms"], "device_bytes": info["device_bytes"], "lut_entries": info["lut_entries"],
         "volume_generation_s": gen_s, "tf": "attribute RGBA (opacity x |axis.view|)"}
    r.update(storage_forms(mg, g, cfg_i, flush, stream, peak))
    boxes_h = synth.make_boxes(cfg_i)
    boxes = torch.from_numpy(boxes_h).to(dev)
    Q = boxes_h.shape[0]
    tune = mg.mg_query_autotune(g, boxes)
    plan = mg.QueryPlan(g, max_Q=Q)
    res = torch.empty((Q, S), dtype=torch.uint32, device=dev)
    ms = _time(lambda: plan.run(boxes, out=res), 5, flush, stream)
    mg.mg_sync_status(g)
    plan.close()
    plan_t = mg.QueryPlan(g, max_Q=Q, timing=True)
    mains = []
    for _ in range(5):
        flush.zero_()
        plan_t.run(boxes, out=res, stream=stream)
        mains.append(plan_t.timing()[1])
    plan_t.close()
    qb, cubes, _ = query_bytes(boxes_h, c["dims"], S)
    main_ms = float(np.median(mains))
    kernel = query_kernel_name(S, tune.get("block_threads") or 256)
    r["queries"] = {"boxes": Q, "u32": {"ms": ms, "queries_per_s": Q / (ms / 1e3)}, "autotune": tune,
                    "roofline": {"bound": "hbm", "kernel": kernel, "kernel_ms": main_ms,
                                 "achieved": qb / main_ms / 1e6, "peak": peak, "unit": "GB/s",
                                 "frac": qb / main_ms / 1e6 / peak, "algorithmic_bytes_per_launch": qb,
                                 "cubes_per_launch": cubes, "traffic": measured_traffic(kernel, cfg_i, Q)}}
    if march:
        r["raymarch"] = raymarch_forms(mg, g, cfg_i, dev, flush, stream)
    g.close()
    return r


# --------------------------------------------------------------------------
# the request loop under the serving mix (volumes of configs 1-3 resident)
# --------------------------------------------------------------------------
def _pct(x, q):
    return float(np.percentile(x, q)) * 1e3 if len(x) else None


def serving(mg, have, args, dev):
    """Replay the Poisson mix through the continuously batched server and
    through the plain one-launch-per-box server (both fp32 histograms, so at
    equal accuracy), at the offered rate and as one saturating burst."""
    import torch
    c5 = synth.CONFIGS[5]
    n = args.serve_requests or c5["requests"]
    rate = args.serve_rate or c5["rate"]
    t0 = time.perf_counter()
    graphs, meta = [], []
    for ci in c5["volumes"]:
        cfg = synth.CONFIGS[ci]
        if ci in have:
            g = have[ci]
        else:
            vol = synth.make_volume(ci, device=dev)
            torch.cuda.synchronize()
            g = mg.mg_build(vol, cfg["S"])
            del vol
        graphs.append(g)
        meta.append(dict(cfg=ci, S=cfg["S"], dims=cfg["dims"], bmax=cfg["box_max"]))
    build_s = time.perf_counter() - t0
    arr, kind, vidx, boxes = synth.make_request_mix(n, rate, [m["dims"] for m in meta], [m["bmax"] for m in meta],
                                                    c5["tf_frac"])
    side = int(math.isqrt(c5["frame_samples"]))
    frames = {v: [(synth.make_tf(5, m["S"], 4, frame=f),
                   synth.make_samples(m["cfg"], width=side, height=side, frame=f)) for f in range(8)]
              for v, m in enumerate(meta)}
    reqs = []
    for i in range(n):
        v = int(vidx[i])
        if kind[i] == 0:
            reqs.append(dict(kind="box", volume=v, box=boxes[i], arrival=float(arr[i])))
        else:
            tf, smp = frames[v][i % 8]
            reqs.append(dict(kind="tf", volume=v, tf=tf, samples=smp, arrival=float(arr[i])))
    burst = [dict(r, arrival=0.0) for r in reqs]
    is_box = np.array([r["kind"] == "box" for r in reqs])
    out = {"workload": c5["name"], "requests": n, "offered_rate_hz": rate, "tf_fraction": c5["tf_frac"],
           "frame_samples": side * side, "volumes": [synth.CONFIGS[m["cfg"]]["name"] for m in meta],
           "hist": "f32 (both forms)", "volume_build_s": build_s}
    # the same requests at other offered rates (arrival times scaled) and as
    # one burst; the sweep shows where each form saturates
    sweep = [("offered", reqs)]
    for r in (200000.0, 2000000.0):
        if r > rate:
            sweep.append(("rate_%d" % int(r), [dict(q, arrival=q["arrival"] * rate / r) for q in reqs]))
    sweep.append(("burst", burst))
    for form, plain in (("batched", False), ("plain", True)):
        srv = mg.Server(slots=4, max_batch=1024, hist="f32", storage="f32", max_samples=side * side, plain=plain)
        for g in graphs:
            srv.add_volume(g, 4)
        srv.start()
        res = {}
        for mode, stream in sweep:
            before = srv.stats()
            results, lat, wall = srv.replay(stream)
            after = srv.stats()
            launches = after["box_launches"] - before["box_launches"]
            tfl = after["tf_launches"] - before["tf_launches"]
            nb = int(is_box.sum())
            offered = None if mode == "burst" else n / max(stream[-1]["arrival"], 1e-9)
            res[mode] = {"offered_requests_per_s": offered, "wall_s": wall, "queries_per_s": nb / wall,
                         "requests_per_s": n / wall, "tf_frames_per_s": (n - nb) / wall,
                         "p50_ms": _pct(lat, 50), "p99_ms": _pct(lat, 99),
                         "box_p50_ms": _pct(lat[is_box], 50), "box_p99_ms": _pct(lat[is_box], 99),
                         "tf_p50_ms": _pct(lat[~is_box], 50), "tf_p99_ms": _pct(lat[~is_box], 99),
                         "mean_batch": nb / max(launches, 1), "box_launches": launches,
                         "tf_launches": tfl, "tf_frames_per_launch": (n - nb) / max(tfl, 1),
                         "failed": after["failed"] - before["failed"]}
            if form == "batched" and mode == "offered":
                # served results against the same boxes queried alone (fp32 tolerance)
                rng = np.random.default_rng(7)
                pick = rng.choice(np.flatnonzero(is_box), size=min(200, int(is_box.sum())), replace=False)
                ok = True
                for i in pick:
                    g = graphs[reqs[i]["volume"]]
                    b = torch.from_numpy(np.asarray(reqs[i]["box"], np.int32).reshape(1, 6)).to(dev)
                    ref = mg.mg_query_boxes(g, b, hist="f32").cpu().numpy()[0].astype(np.float64)
                    got = results[i].astype(np.float64)
                    ok &= bool(np.all(np.abs(got - ref) <= np.maximum(1e-5 * np.abs(ref), 1e-7)))
                res[mode]["sampled_alone_match"] = {"boxes": int(len(pick)), "ok": ok}
            del results
        res["memory_admitted_bytes"] = srv.stats()["memory_admitted"]
        srv.close()
        out[form] = res
    out["batched_over_plain_queries_per_s"] = {m: out["batched"][m]["queries_per_s"] / out["plain"][m]["queries_per_s"]
                                               for m, _ in sweep}
    for g in graphs:
        if all(g is not h for h in have.values()):
            g.close()
    return out


# --------------------------------------------------------------------------
# CPU oracle (reported baseline and the reference arm)
# --------------------------------------------------------------------------
def _host_volume(cfg_i):
    return synth.make_volume(cfg_i, device="cpu")


def cpu_model():
    """The host CPU's model name (lscpu, else /proc/cpuinfo, else platform)."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.split(":")[0].strip().lower() == "model name":
                    return line.split(":", 1)[1].strip()
    except OSError:
        pass
    import platform
    return platform.processor() or platform.machine()


def cpu_baseline(cfg_i, boxes, n_boxes, vol=None, tf=None, keep=None):
    """The oracle's brute-force counting timed on the host cores on a seeded
    sample of the step's boxes (n_boxes of them on all cores, a tenth on one
    core); with tf, also the oracle's TF propagation as the direct per-voxel
    sum over levels 1-3 (the paper's 'revisiting every voxel').  keep (a
    dict) receives the sample's indices and counts, against which the GPU's
    histograms of the same boxes are checked."""
    import oracle
    cfg = synth.CONFIGS[cfg_i]
    if vol is None:
        vol = _host_volume(cfg_i)
    all_threads = oracle.set_threads(0)
    rng = np.random.default_rng(1000 + cfg_i)
    n = min(n_boxes, len(boxes))
    pick = np.sort(rng.choice(len(boxes), size=n, replace=False))
    smp = boxes[pick]
    t0 = time.perf_counter()
    counts = oracle.box_hist(vol, cfg["S"], smp)
    t_all = time.perf_counter() - t0
    oracle.set_threads(1)
    n1 = max(1, n // 10)
    t0 = time.perf_counter()
    oracle.box_hist(vol, cfg["S"], smp[:n1])
    t_one = time.perf_counter() - t0
    oracle.set_threads(all_threads)
    res = {"value": n / t_all, "unit": UNIT, "cores": all_threads, "kind": "oracle",
           "sample": "seeded %d-box subset of the step's %d boxes, brute-force level-0 counting "
                     "(OpenMP over boxes), %.1f s" % (n, len(boxes), t_all),
           "single_thread": {"value": n1 / t_one, "unit": UNIT, "boxes": n1, "seconds": t_one},
           "cpu_model": cpu_model()}
    if keep is not None:
        keep["pick"], keep["counts"] = pick, counts
    if tf is not None:
        dims = oracle.level_dims(*cfg["dims"])
        vox_all = int(np.prod(dims[1:], axis=1).sum())
        n_vox, t_vox = 0, 0.0
        for l in (1, 2, 3):
            t0 = time.perf_counter()
            oracle.direct_colors(vol, l, tf)
            t_vox += time.perf_counter() - t0
            n_vox += int(np.prod(dims[l]))
        res["propagation"] = {"voxels_per_s": n_vox / t_vox, "sample": "levels 1-3 (%d voxels), %.1f s"
                              % (n_vox, t_vox), "full_mip_estimate_s": vox_all / (n_vox / t_vox)}
    return res


def greedy_cpu_baseline(cfg_i, reps=20):
    """The oracle's greedy factorisation (phi_2, tau 3, b = 9) of the config's
    volume timed on the host cores (single-threaded C), reps repetitions."""
    import oracle
    c = synth.CONFIGS[cfg_i]
    vol = _host_volume(cfg_i)
    t0 = time.perf_counter()
    for _ in range(reps):
        og, _, _, _ = oracle.greedy(vol, c["S"], "reduction", tau=3, bitrate=9)
    dt = (time.perf_counter() - t0) / reps
    return {"value": 1.0 / dt, "unit": "factorisations/s", "seconds": dt, "cores": 1, "kind": "oracle",
            "sample": "%d repetitions of the whole %s volume" % (reps, c["name"]), "nodes": og.N}


def run_reference(args):
    _, rank, _ = rank_env()
    if rank != 0:
        return None
    cfg_i = args.config
    cfg = synth.CONFIGS[cfg_i]
    Q = args.queries or cfg["queries"]
    import oracle
    vol = _host_volume(cfg_i)
    boxes = synth.make_boxes(cfg_i, Q=Q)
    # size one step to ~4 s of host work (calibrated on 200 boxes: sizes vary widely)
    t0 = time.perf_counter()
    oracle.box_hist(vol, cfg["S"], boxes[:200])
    dt = time.perf_counter() - t0
    n = int(min(Q, max(200, 200 * 4.0 / max(dt, 1e-6))))
    times = []
    for k in range(max(args.warmup, 3) + args.steps):
        sl = boxes[(k * n) % Q:][:n]
        if len(sl) < n:
            sl = boxes[:n]
        t0 = time.perf_counter()
        oracle.box_hist(vol, cfg["S"], sl)
        if k >= max(args.warmup, 3):
            times.append(time.perf_counter() - t0)
    ms = 1e3 * float(np.mean(times))
    value = n / (ms / 1e3)
    cores = oracle.set_threads(0)
    sample = "%d of the %d boxes per step, brute-force level-0 counting (OpenMP over boxes)" % (n, Q)
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
            "warmup": max(args.warmup, 3), "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "u32 counts", "data": "synthetic", "impl": "reference",
            "config": workload_config(cfg_i, Q, args, args.storage or ("f16" if cfg_i == 3 else "f32")),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
