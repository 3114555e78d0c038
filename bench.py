#!/usr/bin/env python
"""Benchmark of the GB300 tiled point rasterizer.

Metric: splatted points/s for one forward + backward pass (the whole hot
path: projection, split radix sort, duplication, tile ranges, blend, replay
backward, per-point reduction) on the training-shape workload: 4,194,304
clustered points (64 anisotropic Gaussian clusters + 10% uniform background),
opacity ~ Beta(2, 2), 4 FP32 features, one 1280x832 view, bilinear splats,
upstream gradients ~ N(0, 1). Inputs are seeded and synthetic.

    python bench.py [--gpus N --steps K --warmup W] [--impl reference]

With torchrun (N > 1) every rank renders its own independent frame (weak
scaling, no collective on the data path); the time is the max over ranks.
Prints one JSON line on rank 0.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

UNIT = "points/s"


def metric_label(scene):
    """The headline metric for this workload: splatted points/s of the pass it
    runs, at its image size (several views: their count and size range)."""
    pas = "fwd+bwd" if scene.backward else "fwd"
    sizes = sorted({(v.camera.width, v.camera.height) for v in scene.views}, key=lambda s: s[0] * s[1])
    if len(scene.views) == 1:
        where = f"at {sizes[0][0]}x{sizes[0][1]}"
    else:
        where = (f"over {len(scene.views)} views of {sizes[0][0]}x{sizes[0][1]} to "
                 f"{sizes[-1][0]}x{sizes[-1][1]}")
    mode = "" if scene.mode == "bilinear" else ", Gaussian splats"
    return f"splatted points/s ({pas}{mode}) {where}"
L2_FLUSH_BYTES = 256 << 20  # > 129 MB L2


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--config", type=int, default=2, help="workload id (2: 4M points, 1280x832)")
    ap.add_argument("--scale-points", type=float, default=1.0, help="shrink the point count (tests)")
    ap.add_argument("--tile", type=int, default=0, help="tile edge: 16, 8, or 0 = autotuned with the blend depth")
    ap.add_argument("--blend-depth", type=int, default=0, help="records per blend batch (0 = tile^2)")
    ap.add_argument("--record-copy", type=int, default=-1,
                    help="training steps: 1 = the forward keeps the tile-ordered record copy for the backward, "
                         "0 = not, -1 = autotuned with the split (on when --tile fixes the split)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-bg", action="store_true", help="skip the background-model measurement")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-accuracy", action="store_true",
                    help="skip the per-output error measurement against the FP64 oracle")
    ap.add_argument("--cpu-budget-s", type=float, default=20.0)
    ap.add_argument("--graph", type=int, default=-1,
                    help="time CUDA-graph replays of the step: 1/-1 (default) = on, 0 = eager calls")
    ap.add_argument("--batch-compare", type=int, default=-1,
                    help="also time the 8-view BF16 batch (config 5) as one graph replay against the same "
                         "views as sequential FP32 calls: 1 = on, 0 = off, -1 (default) = on for the "
                         "default workload on one GPU")
    return ap.parse_args()


# ----------------------------------------------------------------------------- helpers

def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, ValueError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def measured_peak_hbm():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


# ----------------------------------------------------------------------------- algorithmic bytes

# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) per launch from one
# ncu capture of the kernel as it is built now, keyed by (kernel, workload id,
# tile edge, blend depth, record copy). Random 32-byte record gathers and
# gradient-row scatters move 64-byte DRAM bursts, hence traffic above the
# algorithmic bytes (profiles/ncu_blend_traffic_all_workloads.md).
MEASURED_TRAFFIC = {
    ("blend_fwd", 2, 8, 64, 0): 324530432,
    ("blend_bwd", 2, 8, 64, 0): 707129600,
    ("blend_fwd", 2, 8, 64, 1): 528297216,
    ("blend_bwd", 2, 8, 64, 1): 412425216,
    ("blend_fwd", 3, 16, 256, 0): 2890925056,
    ("blend_fwd", 4, 16, 256, 0): 380597760,
    ("blend_bwd", 4, 16, 256, 0): 1149237248,
    ("blend_fwd", 5, 8, 64, 1): 9635505408,
    ("blend_bwd", 5, 8, 64, 1): 9302492928,
}

def kernel_bytes(name, w):
    """Algorithmic DRAM bytes of ONE launch of kernel `name` on workload counts w."""
    N, D, Dn, Db, HW, C, P = w["N"], w["D"], w["needed"], w["needed_bwd"], w["HW"], w["C"], w["P"]
    rec, fb, npart = w["rec_bytes"], w["feat_bytes"], w["partial_floats"]
    gauss = w.get("gauss", False)
    rb = 8 if gauss else 4  # tile rect per point: 8 bytes (Gaussian), packed 4 bytes (bilinear)
    if name == "project":
        # read xyz, opacity, features (and the Gaussian scale); write the record's
        # used words, depth key, rect (+ copy count for Gaussians) and depth bits
        used = 4 * ((8 if gauss else 4) + -(-C * fb // 4))
        return N * (12 + 4 + C * fb + (4 if gauss else 0)) + N * (used + 4 + rb + (4 if gauss else 0) + 4)
    if name.endswith(".hist"):      # one read of the keys counts every pass's digits
        return 4 * (N if name.startswith("depth") else D)
    if name.endswith(".sweep"):     # per pass: read key+value, write key+value
        if name.startswith("depth"):  # the first pass makes the point indices itself
            passes = max(w.get("depth_passes", 1), 1)
            return (16 * passes - 4) * N / passes
        return 16 * D
    if name == "dup.count":   # sorted point indices, gathered rects, rects in depth order
        return N * (4 + rb + rb)
    if name == "dup.write":
        return N * (rb + 4) + D * 8
    if name == "ranges":
        return D * 4 + P * 8
    if name == "blend_fwd":
        return Dn * (rec + 4) + P * 8 + HW * (4 * C + 16)
    if name == "point_scan.count":
        return N * 4
    if name == "point_scan.apply":
        return N * 8
    if name == "blend_bwd":   # replayed records + indices, one gradient row per copy, pixel state
        return Db * (rec + 4 + 4 * npart) + P * 16 + HW * (4 * C + 16)
    if name == "reduce_grads":
        # rect, depth bits, slot base; the rows; dL/df and dL/do; Gaussians also
        # read the position and scale and write dL/dxyz and dL/ds
        return N * (rb + 4 + 4) + Db * 4 * npart + N * (4 * C + 4) + (N * (12 + 4 + 12 + 4) if gauss else 0)
    return 0


# ----------------------------------------------------------------------------- our arm

def make_views(scene, dev, bf16):
    """Device tensors and C-ABI view structs for every view of a scene."""
    import torch

    from paper_2508_19140_gb300 import rast

    gauss = scene.mode == "gaussian"
    tens, cviews = [], []
    for v in scene.views:
        t = {}
        t["xyz"] = torch.from_numpy(v.xyz).to(dev)
        t["op"] = torch.from_numpy(v.opacity).to(dev)
        t["feat"] = torch.from_numpy(v.feat).to(dev, torch.bfloat16 if bf16 else torch.float32)
        t["scale"] = torch.from_numpy(v.scale).to(dev) if (gauss and v.scale is not None) else None
        H, W, C = v.camera.height, v.camera.width, v.feat.shape[1]
        n = v.xyz.shape[0]
        t["F"] = torch.empty((H, W, C), device=dev)
        t["A"] = torch.empty((H, W), device=dev)
        t["D"] = torch.empty((H, W), device=dev)
        t["gF"] = torch.from_numpy(v.g_feat).to(dev)
        t["gA"] = torch.from_numpy(v.g_alpha).to(dev)
        t["gD"] = torch.from_numpy(v.g_depth).to(dev)
        t["d_feat"] = torch.empty((n, C), device=dev)
        t["d_op"] = torch.empty((n,), device=dev)
        t["d_xyz"] = torch.empty((n, 3), device=dev) if gauss else None
        t["d_scale"] = torch.empty((n,), device=dev) if t["scale"] is not None else None
        cv = rast.View()
        cv.pts = rast.make_points(t["xyz"], t["op"], t["feat"], t["scale"])
        cv.cam = rast.make_camera(v.camera)
        cv.out = rast.make_images(t["F"], t["A"], t["D"])
        cv.grad = rast.make_grads(t["gF"], t["gA"], t["gD"], t["d_feat"], t["d_op"], t["d_xyz"],
                                  t["d_scale"])
        tens.append(t)
        cviews.append(cv)
    return tens, cviews


def sequential_f32_ms(scene, dev, opts, reps, flush):
    """The same views as separate single-view FP32 rasterize_fwd + rasterize_bwd
    calls (no batching, no graph): the baseline the batched BF16 graph path is
    compared with."""
    import torch

    from paper_2508_19140_gb300 import rast

    tens, cviews = make_views(scene, dev, bf16=False)
    nbytes = max(rast.rasterize_workspace_size([cv], opts) for cv in cviews)
    ws = torch.empty(nbytes, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev)

    def run():
        for cv in cviews:
            rast.rasterize_fwd(cv.pts, cv.cam, opts, ws, cv.out, stream)
            if scene.backward:
                rast.rasterize_bwd(cv.pts, cv.cam, opts, ws, cv.grad, stream)

    for _ in range(2):
        run()
    torch.cuda.synchronize()
    tot = 0.0
    for _ in range(reps):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        run()
        e1.record(stream)
        torch.cuda.synchronize()
        tot += e0.elapsed_time(e1)
    del tens, ws
    return tot / reps


def run_ours(args, ws_, rank, local):
    import torch

    from paper_2508_19140_gb300 import build as build_mod
    from paper_2508_19140_gb300 import rast, scenes

    build_mod.build()
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    dist = None
    if ws_ > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)

    from paper_2508_19140_gb300.shard import rank_seed
    scene = scenes.make_scene(args.config, seed=rank_seed(args.config, rank),
                              scale_points=args.scale_points)
    bf16 = scene.feat_dtype == "bf16"
    gauss = scene.mode == "gaussian"
    # Training workloads keep the forward's tile-ordered record copy for the
    # backward (RAST_FLAG_SAVE_FOR_BWD); inference workloads do not need it.
    flags = rast.FLAG_SAVE_FOR_BWD if scene.backward and args.record_copy != 0 else 0
    opts = rast.make_opts(mode=scene.mode, tile=args.tile or 16, blend_depth=args.blend_depth, flags=flags)
    tens, cviews = make_views(scene, dev, bf16)
    tune = None
    if args.tile == 0:
        # Work split (tile edge, blend depth) measured on this workload before
        # any timed step; the choice is cached per workload class.
        from paper_2508_19140_gb300 import autotune
        tr = autotune.autotune(cviews, opts, rast.PASS_FWD | (rast.PASS_BWD if scene.backward else 0),
                               torch.cuda.current_stream(dev))
        opts = autotune.with_split(opts, tr.tile, tr.blend_depth,
                                   tr.save_copy if args.record_copy < 0 else None)
        tune = {"tile": tr.tile, "blend_depth": tr.blend_depth, "record_copy": tr.save_copy,
                "from_cache": tr.from_cache,
                "timings_ms": {autotune._label(c): (round(ms, 4) if ms is not None else None)
                               for c, ms in tr.timings_ms.items()}}
    ws_bytes = rast.rasterize_workspace_size(cviews, opts)
    wsp = torch.empty(ws_bytes, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev)
    n_points = sum(v.xyz.shape[0] for v in scene.views)
    do_bwd = scene.backward
    # The step is one rasterize_batch call (no host synchronisation inside), so
    # it is captured once and replayed: the replay spares the per-kernel
    # launch gaps (measured: 0.845 -> 0.807 ms on the 4 M-point frame).
    use_graph = args.graph != 0

    def step():
        rast.rasterize_batch(cviews, rast.PASS_FWD | (rast.PASS_BWD if do_bwd else 0), opts, wsp, stream)

    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    for _ in range(max(args.warmup, 0)):
        step()
    torch.cuda.synchronize()
    graph = None
    if use_graph:
        # One replayable graph of the whole fwd+bwd step (no host sync inside).
        graph = torch.cuda.CUDAGraph()
        cap = torch.cuda.Stream(dev)
        cap.wait_stream(stream)
        with torch.cuda.graph(graph, stream=cap):
            rast.rasterize_batch(cviews, rast.PASS_FWD | (rast.PASS_BWD if do_bwd else 0), opts, wsp,
                                 torch.cuda.current_stream(dev))
        stream.wait_stream(cap)
        for _ in range(2):
            graph.replay()
        torch.cuda.synchronize()
    st, stats = rast.rasterize_get_status(wsp, stream)
    if st != rast.RAST_OK:
        raise RuntimeError(f"rasterizer status {st}: {stats}")
    if dist:
        dist.barrier()
    torch.cuda.synchronize()

    sampler = ClockSampler(local) if rank == 0 else None
    if sampler:
        sampler.start()
        time.sleep(0.3)
    # The timed region runs the bare product call (no per-kernel events);
    # per-kernel times come from a separate pass right after it.
    rast.rasterize_profile_enable(False)
    evs = []
    for _ in range(args.steps):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        if graph is not None:
            graph.replay()
        else:
            step()
        e1.record(stream)
        evs.append((e0, e1))
    torch.cuda.synchronize()
    st, stats = rast.rasterize_get_status(wsp, stream)  # counters of the last fwd+bwd step
    total_ms = sum(a.elapsed_time(b) for a, b in evs)
    if dist:
        t = torch.tensor([total_ms], device=dev, dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = float(t.item())
        dist.barrier()
    torch.cuda.synchronize()
    clocks = sampler.stop() if sampler else None

    # Per-kernel times: CUDA events on the launch stream around every kernel,
    # in non-graph steps run right after the timed region (L2 flushed before
    # each step as in the timed region).
    prof_steps = max(3, args.steps // 2)
    rast.rasterize_profile_enable(True)
    for _ in range(prof_steps):
        flush.zero_()
        step()
    torch.cuda.synchronize()
    prof = rast.rasterize_profile_read()
    rast.rasterize_profile_enable(False)
    prof_src = ("CUDA events around each kernel on the launch stream, in non-graph steps right after "
                "the timed region (the timed region itself records no per-kernel events)")

    seq = None
    if len(scene.views) > 1 and bf16 and rank == 0:
        seq_ms = sequential_f32_ms(scene, dev, rast.make_opts(mode=scene.mode, flags=flags),
                                   max(3, args.steps // 4), flush)
        seq = {"sequential_f32_ms": round(seq_ms, 4),
               "batched_bf16_graph_ms": round(total_ms / max(args.steps, 1), 4),
               "speedup": round(seq_ms / (total_ms / max(args.steps, 1)), 3),
               "what": "same views: one batched BF16 graph replay vs per-view FP32 rasterize_fwd+rasterize_bwd calls without a graph"}

    # Forward-only timing (reported beside the headline).
    fwd_ms = None
    if do_bwd:
        evf = []
        for _ in range(max(3, args.steps // 2)):
            flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            rast.rasterize_batch(cviews, rast.PASS_FWD, opts, wsp, stream)
            e1.record(stream)
            evf.append((e0, e1))
        torch.cuda.synchronize()
        fwd_ms = sum(a.elapsed_time(b) for a, b in evf) / len(evf)

    ms_step = total_ms / max(args.steps, 1)
    value = n_points * ws_ / (ms_step / 1e3)

    # ---- roofline of the dominant kernel (per-launch averages from the live events)
    v0 = scene.views[0]
    C = v0.feat.shape[1]
    lay = rast.rasterize_workspace_layout(cviews, opts)
    rec_bytes = lay["records"][1] // max(n_points, 1)
    w = dict(N=n_points, D=int(stats["n_copies"]), needed=int(stats["needed_records"]),
             needed_bwd=int(stats["needed_records_bwd"]),
             HW=sum(v.camera.width * v.camera.height for v in scene.views), C=C,
             P=int(stats["n_tiles"]), rec_bytes=rec_bytes, feat_bytes=2 if bf16 else 4,
             partial_floats=C + (7 if gauss else 1), gauss=gauss,
             depth_passes=int(round(prof.get("depth_sort.sweep", (0, 0))[0] / max(prof.get("init_header", (1, 0))[0], 1))))
    peak, peak_src = measured_peak_hbm()
    kernels = {}
    for name, (launches, tot) in prof.items():
        avg = tot / max(launches, 1)
        b = kernel_bytes(name, w)
        kernels[name] = dict(launches=launches, ms_per_launch=round(avg, 5),
                             share=round(tot / max(sum(x[1] for x in prof.values()), 1e-9), 4),
                             bytes=int(b), gbs=round(b / (avg * 1e6), 1) if avg > 0 else None)
    dom = max(prof.items(), key=lambda kv: kv[1][1])[0] if prof else None
    roofline = None
    if dom:
        k = kernels[dom]
        ach = k["gbs"] or 0.0
        copy = int(bool(int(opts.flags) & rast.FLAG_SAVE_FOR_BWD) and scene.mode == "bilinear")
        tkey = (dom, scene.config_id, int(opts.tile), int(opts.blend_depth) or int(opts.tile) ** 2, copy)
        traffic = MEASURED_TRAFFIC.get(tkey) if args.scale_points == 1.0 else None
        roofline = {"kernel": dom, "bound": "hbm", "achieved": ach, "peak": peak, "unit": "GB/s",
                    "frac": round(ach / peak, 4), "traffic": traffic,
                    "algorithmic_bytes": k["bytes"],
                    "peak_source": f"{peak_src} (hbm_gbs, copy burst)"}
    blend = kernels.get("blend_fwd")
    gpu_launches = int(round(sum(x[0] for x in prof.values()) / max(prof_steps, 1) * args.steps))

    bg = None
    if not args.no_bg and rank == 0:
        bg = run_background(scene, tens, dev, stream, flush, peak, max(5, args.steps // 2))
    contraction = None
    if not args.no_bg and rank == 0:
        contraction = run_contract(tens, dev, stream, flush, peak, max(5, args.steps // 2))
    untiled = None
    if len(scene.views) == 1 and scene.mode == "bilinear" and not args.no_bg and rank == 0:
        untiled = run_untiled(scene, tens, dev, stream, flush, max(5, args.steps // 2))
    ring = None
    if len(scene.views) == 1 and not do_bwd and rank == 0:
        ring = run_ring(scene, tens, opts, dev, stream, flush, max(5, args.steps // 2), ms_step)

    e2e = None
    if not args.no_e2e:
        e2e = run_e2e(args, scene, tens, cviews, opts, wsp, stream, dev, n_points, ws_, dist)

    accuracy = None
    if not args.no_accuracy and rank == 0:
        accuracy = run_accuracy(scene, dev, opts)

    gauss_extra = None
    if gauss and rank == 0:
        gauss_extra = run_gauss_extra(scene, cviews, opts, wsp, lay, n_points, stream, flush,
                                      max(3, args.steps // 2), do_bwd)

    out = {
        "metric": metric_label(scene), "value": round(value, 1), "unit": UNIT, "n_gpus": ws_,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms_step, 4),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "bf16-features/f32" if bf16 else "f32", "data": "synthetic",
        "config": {"workload": scene.name, "config_id": scene.config_id, "n_points_per_gpu": n_points,
                   "views": len(scene.views), "width": v0.camera.width, "height": v0.camera.height,
                   "channels": C, "mode": scene.mode, "tile": int(opts.tile),
                   "blend_depth": int(opts.blend_depth) or int(opts.tile) ** 2, "pass": "fwd+bwd" if do_bwd else "fwd",
                   "l2": "flushed between timed steps (256 MiB write, untimed)",
                   "parallelism": f"independent frame per GPU x{ws_}"},
        "fwd_points_per_s": round(n_points * ws_ / (fwd_ms / 1e3), 1) if fwd_ms else None,
        "ms_fwd": round(fwd_ms, 4) if fwd_ms else None,
        "copies": w["D"], "needed_records": w["needed"],
        "autotune": tune,
        "roofline": roofline,
        "background": bg,
        "ring_buffer": ring,
        "untiled_baseline": untiled,
        "contraction": contraction,
        "gaussian": gauss_extra,
        "blend_fwd_roofline": ({"achieved": blend["gbs"], "peak": peak, "unit": "GB/s",
                                "frac": round((blend["gbs"] or 0) / peak, 4)} if blend else None),
        "kernels": kernels, "kernel_timing": prof_src, "gpu_launches": gpu_launches,
        "graph": graph is not None, "batched_vs_sequential": seq,
        "clocks": clocks, "e2e": e2e, "accuracy": accuracy,
    }
    return out, dist


def run_gauss_extra(scene, cviews, opts, wsp, lay, n_points, stream, flush, reps, do_bwd):
    """Gaussian workloads: the 3-sigma pixel radii the projection gave the
    visible points (read from the records of the last timed step, before
    anything else reuses the workspace), copies per point, and the same step
    with the isotropic screen-space covariance instead of the EWA one."""
    import torch

    from paper_2508_19140_gb300 import rast

    torch.cuda.synchronize()
    words = lay["records"][1] // 4 // max(n_points, 1)
    off, nb = lay["records"]
    recs = wsp[off:off + nb].view(torch.int32).view(n_points, words)
    r = recs[:, 7].view(torch.float32)  # record word 7: radius in pixels
    coff = lay["count"][0]
    cnt = wsp[coff:coff + 4 * n_points].view(torch.int32)
    vis = cnt > 0
    rv = r[vis].round().clamp(0, 17).to(torch.int64)
    hist = torch.bincount(rv, minlength=18).tolist()
    n_vis = int(vis.sum().item())
    copies = int(cnt[vis].to(torch.int64).sum().item())

    iso = rast.make_opts(mode="gaussian", gauss_cov="iso", tile=int(opts.tile), blend_depth=int(opts.blend_depth))
    passes = rast.PASS_FWD | (rast.PASS_BWD if do_bwd else 0)
    for _ in range(2):
        rast.rasterize_batch(cviews, passes, iso, wsp, stream)
    torch.cuda.synchronize()
    tot = 0.0
    for _ in range(reps):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        rast.rasterize_batch(cviews, passes, iso, wsp, stream)
        e1.record(stream)
        torch.cuda.synchronize()
        tot += e0.elapsed_time(e1)
    ms = tot / reps
    st, stats = rast.rasterize_get_status(wsp, stream)
    return {"radius_px_hist": {"bins": "r = 0, 1, ..., 16 px; last bin r >= 17", "counts": hist,
                               "visible_points": n_vis},
            "copies_per_visible_point": round(copies / max(n_vis, 1), 3),
            "isotropic_covariance": {"ms_per_step": round(ms, 4),
                                     "points_per_s": round(n_points / (ms / 1e3), 1),
                                     "copies": int(stats["n_copies"]), "status": int(st)}}


def run_background(scene, tens, dev, stream, flush, peak, reps):
    """Distilled background model on view 0 (Sec. 3.2): composite behind the
    blend's output with a 1024 x 2048 x C spherical map and its backward (map
    gradient, dL/dalpha), directions cached. Timed with CUDA events, L2 flushed
    between repetitions. Algorithmic bytes: per pixel the image, alpha, cached
    direction and output (fwd) or upstream gradient, alpha, direction and
    dL/dalpha read+write (bwd); the map once; bwd also the fixed-point
    accumulators (zeroed, read) and the map gradient."""
    import torch

    from paper_2508_19140_gb300 import rast, scenes

    v = scene.views[0]
    t = tens[0]
    H, W, C = v.camera.height, v.camera.width, v.feat.shape[1]
    env = torch.from_numpy(scenes.env_map(c=C)).to(dev)
    e = rast.make_envmap(env)
    cam = rast.make_camera(v.camera)
    dirs = torch.empty((H, W, 3), device=dev)
    rast.rasterize_view_dirs(cam, dirs, stream)
    out = torch.empty((H, W, C), device=dev)
    g = torch.randn((H, W, C), device=dev)
    ga = torch.zeros((H, W), device=dev)
    dmap = torch.empty_like(env)
    scratch = torch.empty(rast.rasterize_bg_scratch_size(e), dtype=torch.uint8, device=dev)

    def fwd():
        rast.rasterize_bg_composite(cam, e, dirs, t["F"], t["A"], out, stream)

    def bwd():
        rast.rasterize_bg_composite_bwd(cam, e, dirs, t["A"], g, ga, dmap, scratch, stream)

    res = {}
    for name, fn in (("fwd", fwd), ("bwd", bwd)):
        for _ in range(3):
            fn()
        evs = []
        for _ in range(reps):
            flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fn()
            e1.record(stream)
            evs.append((e0, e1))
        torch.cuda.synchronize()
        res[name] = sum(a.elapsed_time(b) for a, b in evs) / len(evs)
    HW, M = H * W, env.numel()
    b_fwd = HW * (4 * C + 4 + 12 + 4 * C) + 4 * M
    b_bwd = HW * (4 * C + 4 + 12 + 8) + 4 * M + 8 * M * 2 + 4 * M
    return {"what": "composite behind the blend with a 1024x2048xC spherical map (fwd) and its adjoint (bwd), "
                    "view 0, cached directions",
            "map": [int(env.shape[0]), int(env.shape[1]), C], "pixels": HW,
            "fwd_ms": round(res["fwd"], 5), "bwd_ms": round(res["bwd"], 5),
            "fwd_gbs": round(b_fwd / (res["fwd"] * 1e6), 1), "bwd_gbs": round(b_bwd / (res["bwd"] * 1e6), 1),
            "fwd_frac": round(b_fwd / (res["fwd"] * 1e6) / peak, 4),
            "bwd_frac": round(b_bwd / (res["bwd"] * 1e6) / peak, 4)}


def run_contract(tens, dev, stream, flush, peak, reps):
    """Fused spherical contraction (Sec. 3.4) of view 0's positions into a
    separate buffer: 12 bytes read and 12 written per point."""
    import torch

    from paper_2508_19140_gb300 import rast

    xyz = tens[0]["xyz"]
    out = torch.empty_like(xyz)
    for _ in range(3):
        rast.rasterize_contract(xyz, out, stream)
    evs = []
    for _ in range(reps):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        rast.rasterize_contract(xyz, out, stream)
        e1.record(stream)
        evs.append((e0, e1))
    torch.cuda.synchronize()
    ms = sum(a.elapsed_time(b) for a, b in evs) / len(evs)
    n = int(xyz.shape[0])
    gbs = 24 * n / (ms * 1e6)
    return {"points": n, "ms": round(ms, 5), "gbs": round(gbs, 1), "frac": round(gbs / peak, 4)}


def run_untiled(scene, tens, dev, stream, flush, reps):
    """Forward of the same frame with the two untiled baselines (per-pixel
    lists, ~4 copies per point): through the split sort with one thread per
    pixel, and through one 64-bit [pixel | depth] key sort with one warp per
    pixel (the arrangement the paper's 28n sort cost refers to), against the
    tiled forward at 16x16 and 8x8 tiles, with the per-kernel split of the
    untiled runs: what tiling and the split sort save on this GPU (Sec. 3.2
    "Tiled Rendering")."""
    import torch

    from paper_2508_19140_gb300 import rast

    t = tens[0]
    v = scene.views[0]
    pts = rast.make_points(t["xyz"], t["op"], t["feat"])
    cam = rast.make_camera(v.camera)
    out = rast.make_images(t["F"], t["A"], t["D"])

    def timed(fn):
        for _ in range(2):
            fn()
        evs = []
        for _ in range(reps):
            flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fn()
            e1.record(stream)
            evs.append((e0, e1))
        torch.cuda.synchronize()
        return sum(a.elapsed_time(b) for a, b in evs) / len(evs)

    res = {}
    o_u = rast.make_opts(mode="bilinear")
    ws_u = torch.empty(rast.rasterize_untiled_workspace_size(pts, cam, o_u), dtype=torch.uint8, device=dev)
    res["untiled_fwd_ms"] = round(timed(lambda: rast.rasterize_fwd_untiled(pts, cam, o_u, ws_u, out, stream)), 4)
    rast.rasterize_profile_enable(True)
    rast.rasterize_fwd_untiled(pts, cam, o_u, ws_u, out, stream)
    prof = rast.rasterize_profile_read()
    rast.rasterize_profile_enable(False)
    res["untiled_kernels_ms"] = {k: round(b, 4) for k, (a, b) in prof.items()}
    res["untiled_copies"] = int(rast.rasterize_get_status(ws_u, stream)[1]["n_copies"])
    # The same per-pixel lists from ONE 64-bit [pixel | depth] key sort of the
    # copies (7 digit passes over ~4n copies: the paper's 28n), one warp per pixel.
    ws_k = torch.empty(rast.rasterize_untiled64_workspace_size(pts, cam, o_u), dtype=torch.uint8, device=dev)
    res["untiled64_fwd_ms"] = round(timed(lambda: rast.rasterize_fwd_untiled64(pts, cam, o_u, ws_k, out, stream)), 4)
    rast.rasterize_profile_enable(True)
    rast.rasterize_fwd_untiled64(pts, cam, o_u, ws_k, out, stream)
    prof = rast.rasterize_profile_read()
    rast.rasterize_profile_enable(False)
    res["untiled64_kernels_ms"] = {k: round(b, 4) for k, (a, b) in prof.items()}
    res["untiled64_sort_passes"] = {k: int(a) for k, (a, b) in prof.items() if k.endswith(".sweep")}
    res["untiled64_sort_ms"] = round(sum(b for k, (a, b) in prof.items() if k.startswith("sort64")), 4)
    res["split_untiled_sort_ms"] = round(sum(b for k, b in res["untiled_kernels_ms"].items()
                                             if k.startswith(("depth_sort", "tile_sort"))), 4)
    del ws_k
    for tile in (16, 8):
        o_t = rast.make_opts(mode="bilinear", tile=tile)
        ws_t = torch.empty(rast.rasterize_workspace_size([_single(pts, cam, out)], o_t), dtype=torch.uint8,
                           device=dev)
        res[f"tiled{tile}_fwd_ms"] = round(timed(lambda: rast.rasterize_fwd(pts, cam, o_t, ws_t, out, stream)), 4)
        if tile == 16:
            res["tiled16_copies"] = int(rast.rasterize_get_status(ws_t, stream)[1]["n_copies"])
    res["speedup_tiled16_vs_untiled"] = round(res["untiled_fwd_ms"] / res["tiled16_fwd_ms"], 3)
    res["speedup_tiled16_vs_untiled64"] = round(res["untiled64_fwd_ms"] / res["tiled16_fwd_ms"], 3)
    return res


def _single(pts, cam, out):
    from paper_2508_19140_gb300 import rast
    v = rast.View()
    v.pts, v.cam, v.out = pts, cam, out
    return v


def run_ring(scene, tens, opts, dev, stream, flush, reps, ms_single):
    """The inference frame's points as 4 view-specific clouds rendered into one
    image with rasterize_clouds (Sec. 3.1 ring buffer), against the same points
    as one cloud (the timed step) and against concatenating the 4 clouds into
    one buffer first (the copy the multi-cloud call avoids)."""
    import torch

    from paper_2508_19140_gb300 import rast

    v = scene.views[0]
    t = tens[0]
    n = v.xyz.shape[0]
    cuts = [0, n // 4, n // 2, 3 * n // 4, n]
    clouds = [rast.make_points(t["xyz"][a:b], t["op"][a:b], t["feat"][a:b],
                               None if t.get("scale") is None else t["scale"][a:b])
              for a, b in zip(cuts[:-1], cuts[1:])]
    cam = rast.make_camera(v.camera)
    ws = torch.empty(rast.rasterize_clouds_workspace_size(clouds, cam, opts), dtype=torch.uint8, device=dev)
    out = rast.make_images(t["F"], t["A"], t["D"])
    parts = [(t["xyz"][a:b].clone(), t["op"][a:b].clone(), t["feat"][a:b].clone()) for a, b in zip(cuts[:-1], cuts[1:])]

    def timed(fn):
        for _ in range(2):
            fn()
        evs = []
        for _ in range(reps):
            flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fn()
            e1.record(stream)
            evs.append((e0, e1))
        torch.cuda.synchronize()
        return sum(a.elapsed_time(b) for a, b in evs) / len(evs)

    ms_clouds = timed(lambda: rast.rasterize_clouds(clouds, None, cam, out, rast.PASS_FWD, opts, ws, stream))

    def concat():
        for k in range(3):
            torch.cat([p[k] for p in parts], out=(t["xyz"], t["op"], t["feat"])[k])
    ms_cat = timed(concat)
    return {"what": "the same points as 4 clouds in one rasterize_clouds call vs one cloud; concat_ms is the "
                    "device copy that building one cloud from 4 would add",
            "clouds": 4, "points": n, "ms_4_clouds": round(ms_clouds, 4), "ms_1_cloud": round(ms_single, 4),
            "concat_ms": round(ms_cat, 4),
            "points_per_s_4_clouds": round(n / (ms_clouds / 1e3), 1)}


def run_e2e(args, scene, tens, cviews, opts, wsp, stream, dev, n_points, ws_, dist):
    """Same metric through the C ABI with pinned HOST buffers: every step copies
    its inputs host->device, runs fwd+bwd and copies its outputs (images and
    point gradients) back. Steps are pipelined over two device buffer sets:
    the inputs of step k+1 go up on one copy stream and the outputs of step k-1
    come down on another while step k computes, so the timed region holds every
    copy of every step but overlaps them with the kernels."""
    import torch

    from paper_2508_19140_gb300 import rast

    bf16 = scene.feat_dtype == "bf16"
    tens2, cviews2 = make_views(scene, dev, bf16)
    sets = [(tens, cviews), (tens2, cviews2)]
    in_keys = ("xyz", "op", "feat", "scale") + (("gF", "gA", "gD") if scene.backward else ())
    out_keys = ("F", "A", "D") + (("d_feat", "d_op", "d_xyz", "d_scale") if scene.backward else ())
    host_in = []
    h2d = d2h = 0
    for t in tens:
        hi = {k: t[k].detach().cpu().pin_memory() for k in in_keys if t.get(k) is not None}
        h2d += sum(x.numel() * x.element_size() for x in hi.values())
        host_in.append(hi)
    host_out = []
    for _ in range(2):
        ho = [{k: torch.empty(t[k].shape, dtype=t[k].dtype, pin_memory=True) for k in out_keys
               if t.get(k) is not None} for t in tens]
        host_out.append(ho)
    d2h = sum(x.numel() * x.element_size() for ho in host_out[0] for x in ho.values())
    up = torch.cuda.Stream(dev)
    down = torch.cuda.Stream(dev)
    ev = lambda: torch.cuda.Event()
    h2d_done = [ev(), ev()]
    compute_done = [ev(), ev()]
    d2h_done = [ev(), ev()]
    passes = rast.PASS_FWD | (rast.PASS_BWD if scene.backward else 0)

    def upload(sidx):
        with torch.cuda.stream(up):
            for t, hi in zip(sets[sidx][0], host_in):
                for k, x in hi.items():
                    t[k].copy_(x, non_blocking=True)
        h2d_done[sidx].record(up)

    def run(K):
        upload(0)
        for k in range(K):
            s, o = k % 2, 1 - k % 2
            if k + 1 < K:
                if k >= 1:
                    up.wait_event(compute_done[o])  # set o is free once step k-1 computed
                upload(o)
            stream.wait_event(h2d_done[s])
            if k >= 2:
                stream.wait_event(d2h_done[s])      # step k-2's outputs are down
            rast.rasterize_batch(sets[s][1], passes, opts, wsp, stream)
            compute_done[s].record(stream)
            down.wait_event(compute_done[s])
            with torch.cuda.stream(down):
                for t, ho in zip(sets[s][0], host_out[s]):
                    for key, x in ho.items():
                        x.copy_(t[key], non_blocking=True)
            d2h_done[s].record(down)
        stream.wait_event(d2h_done[(K - 1) % 2])
        if K >= 2:
            stream.wait_event(d2h_done[K % 2])

    run(2)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    K = max(3, args.steps // 2)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(up)
    run(K)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / K
    if dist:
        tt = torch.tensor([ms], device=dev, dtype=torch.float64)
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        ms = float(tt.item())
    return {"value": round(n_points * ws_ / (ms / 1e3), 1), "unit": UNIT, "ms_per_step": round(ms, 4),
            "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
            "api": "rasterize_batch (C ABI) with pinned host buffers; copies of step k+1 (up) and k-1 (down) "
                   "overlap step k's kernels on two copy streams"}


# ----------------------------------------------------------------------------- accuracy

def _err_stats(got, want, mask=None):
    """Max relative error over elements with |ref| above 1e-3 of the largest,
    normwise relative error, and max absolute error of `got` against `want`."""
    g = np.asarray(got, np.float64)
    w = np.asarray(want, np.float64)
    if mask is not None:
        g, w = g[mask], w[mask]
    if w.size == 0:
        return None
    d = np.abs(g - w)
    big = np.abs(w) > 1e-3 * max(np.abs(w).max(), 1e-30)
    return {"max_rel": float((d[big] / np.abs(w[big])).max()) if big.any() else 0.0,
            "norm_rel": float(np.linalg.norm(g - w) / max(np.linalg.norm(w), 1e-30)),
            "max_abs": float(d.max())}


def run_accuracy(scene, dev, opts, n_pix=2000, n_pts=400, seed=7):
    """Measured error of every output against the FP64 oracle, with FP32 and
    with BF16 features, on sampled pixels (F, alpha, depth) and sampled points
    (d_feat, d_opacity, and in Gaussian mode d_xyz, d_scale) of the
    workload's first and last views. BF16 runs are compared with the oracle
    fed the same BF16-rounded features (accumulation error) and with the
    oracle fed the FP32 features (total error). Gaussian pixels whose
    termination decision lies within 1e-5 of t_min (CPU and GPU exp can
    differ by an ulp there), and points touching them, are left out and
    counted."""
    import torch

    import oracle
    from paper_2508_19140_gb300 import rast

    oracle.build()
    gauss = scene.mode == "gaussian"
    kw = dict(mode=scene.mode, tile=16, pin32=True)
    vids = sorted({0, len(scene.views) - 1})
    res = {"what": f"sampled {n_pix} pixels and {n_pts} points per view, views {vids}, "
                   "errors vs the FP64 oracle", "tile": int(opts.tile),
           "blend_depth": int(opts.blend_depth) or int(opts.tile) ** 2}
    for bf16 in (False, True):
        tens, cviews = make_views(scene, dev, bf16)
        ws = torch.empty(rast.rasterize_workspace_size(cviews, opts), dtype=torch.uint8, device=dev)
        passes = rast.PASS_FWD | (rast.PASS_BWD if scene.backward else 0)
        rast.rasterize_batch(cviews, passes, opts, ws)
        st, _ = rast.rasterize_get_status(ws)
        torch.cuda.synchronize()
        acc = {}
        excluded = 0
        for k in vids:
            v, t = scene.views[k], tens[k]
            rng = np.random.default_rng(seed + k)
            W, H = v.camera.width, v.camera.height
            pix = rng.choice(W * H, min(n_pix, W * H), replace=False)
            feats = {"same_features": v.feat if not bf16 else
                     torch.from_numpy(v.feat).to(torch.bfloat16).float().numpy()}
            if bf16:
                feats["fp32_features"] = v.feat
            scale = v.scale if gauss else None
            F = t["F"].cpu().numpy().reshape(-1, v.feat.shape[1])[pix]
            A = t["A"].cpu().numpy().reshape(-1)[pix]
            D = t["D"].cpu().numpy().reshape(-1)[pix]
            pm = np.zeros(len(v.xyz), np.uint8)
            pm[rng.choice(len(v.xyz), min(n_pts, len(v.xyz)), replace=False)] = 1
            if gauss and scene.backward:
                p = oracle.project(v.xyz, v.camera, scale=scale, **kw)
                boxes = {}
                for i in np.nonzero(pm & (p["vis"] == 1))[0]:
                    x0, x1, y0, y1 = p["box"][i]
                    boxes[i] = (np.arange(y0, y1 + 1)[:, None] * W + np.arange(x0, x1 + 1)[None, :]).ravel()
                if boxes:
                    allpix = np.unique(np.concatenate(list(boxes.values())))
                    marg = oracle.render(v.xyz, v.opacity, feats["same_features"], v.camera, scale=scale,
                                         pix=allpix, **kw)["margin"]
                    amb = set(allpix[marg <= 1e-5].tolist())
                    for i, px in boxes.items():
                        if amb.intersection(px.tolist()):
                            pm[i] = 0
                            excluded += 1
            got_g = None
            if scene.backward:
                got_g = {"d_feat": t["d_feat"].cpu().numpy(), "d_opacity": t["d_op"].cpu().numpy()}
                if gauss:
                    got_g["d_xyz"] = t["d_xyz"].cpu().numpy()
                    if t.get("d_scale") is not None:
                        got_g["d_scale"] = t["d_scale"].cpu().numpy()
            sel = pm == 1
            for ref_kind, fv in feats.items():
                ref = oracle.render(v.xyz, v.opacity, fv, v.camera, scale=scale, pix=pix, **kw)
                ok = ref["margin"] > 1e-5 if gauss else np.ones(len(pix), bool)
                if ref_kind == "same_features":
                    excluded += int((~ok).sum())
                outs = {"F": (F, ref["F"], ok[:, None] & np.ones_like(F, bool)),
                        "alpha": (A, ref["alpha"], ok), "depth": (D, ref["depth"], ok)}
                if got_g is not None:
                    g = oracle.backward(v.xyz, v.opacity, fv, v.camera, v.g_feat, v.g_alpha, v.g_depth,
                                        scale=scale, pmask=pm, **kw)
                    for key, val in got_g.items():
                        outs[key] = (val[sel], g[key][sel], None)
                for key, (got, want, m) in outs.items():
                    acc.setdefault(ref_kind, {}).setdefault(key, []).append((got, want, m))
        dres = {}
        for ref_kind, per in acc.items():
            dres[ref_kind] = {}
            for key, items in per.items():
                got = np.concatenate([np.asarray(a).reshape(len(a), -1) for a, _, _ in items])
                want = np.concatenate([np.asarray(b).reshape(len(b), -1) for _, b, _ in items])
                masks = [np.ones_like(np.asarray(a).reshape(len(a), -1), bool) if m is None else
                         np.asarray(m).reshape(len(a), -1) for a, _, m in items]
                dres[ref_kind][key] = _err_stats(got, want, np.concatenate(masks))
        dres["status"] = int(st)
        res["bf16" if bf16 else "fp32"] = dres
        del tens, cviews, ws
        torch.cuda.empty_cache()
    res["excluded_termination_ambiguous"] = excluded
    return res


# ----------------------------------------------------------------------------- CPU oracle

def oracle_sample(scene, budget_s, threads=0, pin32=True):
    """Time the CPU oracle (as it stands) on a band of pixel rows of the same
    frame: forward for the band's pixels, backward for the points that land in
    it. The band height is chosen so the run fits the budget. Returns
    (points/s, points in the sample, seconds, description)."""
    import oracle

    v = scene.views[0]
    kw = dict(mode=scene.mode, tile=16, pin32=pin32, n_threads=threads)
    W, H = v.camera.width, v.camera.height
    p = oracle.project(v.xyz, v.camera, scale=v.scale if scene.mode == "gaussian" else None, **kw)
    vis = p["vis"] == 1
    feat = v.feat.astype(np.float64)

    def run(rows):
        y0 = (H - rows) // 2
        pix = (np.arange(y0, y0 + rows)[:, None] * W + np.arange(W)[None, :]).reshape(-1)
        pm = vis & (p["box"][:, 2] >= y0) & (p["box"][:, 3] < y0 + rows)
        t = time.perf_counter()
        oracle.render(v.xyz, v.opacity, feat, v.camera, pix=pix, scale=v.scale, **kw)
        if scene.backward:
            oracle.backward(v.xyz, v.opacity, feat, v.camera, v.g_feat, v.g_alpha, v.g_depth,
                            scale=v.scale, pmask=pm.astype(np.uint8), **kw)
        return time.perf_counter() - t, int(pm.sum()), rows

    dt, npts, rows = run(max(H // 32, 1))
    per_pt = dt / max(npts, 1)
    rows = H
    if per_pt * vis.sum() > budget_s:
        rows = max(1, min(H, int(H * budget_s / max(per_pt * vis.sum(), 1e-9))))
    dt, npts, rows = run(rows)
    desc = (f"oracle fwd{'+bwd' if scene.backward else ''} on a band of {rows}/{H} pixel rows of the "
            f"{W}x{H} frame ({npts} of {len(v.xyz)} points land in it), FP64 values / FP32 decisions")
    return npts / dt, npts, dt, desc


def run_reference(args, rank):
    """Reference arm: the CPU oracle timed on the host cores (rank 0 only)."""
    if rank != 0:
        return None
    import oracle

    from paper_2508_19140_gb300 import scenes

    oracle.build()
    scene = scenes.make_scene(args.config, scale_points=args.scale_points)
    steps = max(args.steps, 1)
    budget = max(1.0, 150.0 / (steps + min(args.warmup, 1)))
    vals = []
    desc = ""
    for k in range(min(args.warmup, 1) + steps):
        val, npts, dt, desc = oracle_sample(scene, budget)
        if k >= min(args.warmup, 1):
            vals.append((npts, dt))
    tot_pts = sum(x[0] for x in vals)
    tot_t = sum(x[1] for x in vals)
    value = tot_pts / tot_t
    cores = oracle.num_threads()
    return {"impl": "reference", "metric": metric_label(scene), "value": round(value, 1), "unit": UNIT, "n_gpus": args.gpus,
            "steps": steps, "warmup": args.warmup, "ms_per_step": round(1e3 * tot_t / steps, 3),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": scene.name, "config_id": scene.config_id},
            "cpu_baseline": {"value": round(value, 1), "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": desc},
            "e2e": {"value": round(value, 1), "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def main():
    args = parse()
    ws_, rank, local = dist_env()
    if args.impl == "reference":
        out = run_reference(args, rank)
        if out is not None:
            print(json.dumps(out), flush=True)
        return
    out, dist = run_ours(args, ws_, rank, local)
    want_batch = args.batch_compare == 1 or (args.batch_compare == -1 and args.config == 2 and
                                             args.scale_points == 1.0)
    if want_batch and ws_ == 1 and rank == 0:
        # The batched-vs-sequential comparison on its own workload (8 uneven
        # views, 62 M points, C = 8 BF16, forward + backward).
        sub = argparse.Namespace(**vars(args))
        sub.config, sub.steps, sub.warmup = 5, 8, 3
        sub.tile, sub.blend_depth, sub.record_copy = 0, 0, -1
        sub.no_e2e = sub.no_bg = sub.no_accuracy = sub.no_cpu_baseline = True
        o5, _ = run_ours(sub, 1, 0, local)
        bvs = dict(o5["batched_vs_sequential"] or {})
        bvs.update({"workload": o5["config"]["workload"], "metric": o5["metric"],
                    "batched_value": o5["value"], "unit": o5["unit"], "steps": sub.steps,
                    "warmup": sub.warmup, "autotune": {k: (o5.get("autotune") or {}).get(k) for k in
                                                       ("tile", "blend_depth", "record_copy")}})
        out["batched_vs_sequential"] = bvs
    if rank == 0 and not args.no_cpu_baseline and ws_ == 1:
        from paper_2508_19140_gb300 import scenes
        import oracle
        oracle.build()
        scene = scenes.make_scene(args.config, scale_points=args.scale_points)
        val, npts, dt, desc = oracle_sample(scene, args.cpu_budget_s)
        out["cpu_baseline"] = {"value": round(val, 1), "unit": UNIT, "cores": oracle.num_threads(),
                               "kind": "oracle", "sample": desc, "seconds": round(dt, 2)}
        if sum(len(v.xyz) for v in scene.views) <= 100_000:
            # small frames: the oracle on one thread as well (this sets the
            # oracle's thread count for the rest of the process)
            v1, _, dt1, _ = oracle_sample(scene, args.cpu_budget_s, threads=1)
            out["cpu_baseline"]["single_thread"] = {"value": round(v1, 1), "cores": 1, "seconds": round(dt1, 2)}
    elif rank == 0:
        out["cpu_baseline"] = None
    if rank == 0:
        print(json.dumps(out), flush=True)
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
