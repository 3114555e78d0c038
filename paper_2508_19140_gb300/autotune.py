"""Autotuner for the rasterizer's work split: tile edge, blend depth and,
for training steps, whether the forward keeps a tile-ordered copy of the
records for the backward.

The paper renders with 16x16 tiles (Sec. 3.2, "Tiled Rendering"); the tile
edge and the number of records staged per blend batch change only how the
work is split over CTAs and barriers, never the images (the per-pixel
compositing order is the (depth, point index) order whatever the tiling, and
the kernels keep the same FP32 operations). Which split is fastest depends on
the workload: smaller tiles shorten the longest tile list (the blend's
critical path in dense regions) but create more point-tile copies to sort and
reduce. So the choice is measured, not guessed:

  * the candidates are the compiled (tile, depth) pairs the library reports
    (``rasterize_tune_candidates``), default first; when the caller runs a
    bilinear backward on the workspace and allows the record copy
    (RAST_FLAG_SAVE_FOR_BWD in its opts), each pair is also tried with the
    copy, after every pair without it (the copy costs the forward one
    sequential write per record and saves the backward its random gathers:
    it pays off once the records no longer fit in L2);
  * each is timed on the caller's own views for the caller's passes (whole
    step: projection, both sorts, blend, and the backward when asked), with
    CUDA events on the caller's stream after warm-up, L2 flushed between
    repetitions, median of the repetitions;
  * the winner is cached in a JSON file keyed by (GPU name, splat mode,
    channels, feature dtype, pass, number of views, pixel-count bucket,
    point-count bucket), so a later process with a similar workload skips
    the timing. Buckets are powers of two of the totals.

Timing runs the real kernels and overwrites the views' output (and gradient)
buffers; it allocates one workspace per candidate for the duration of the
call. The cache file is ``$INPC_RAST_TUNE_CACHE`` or
``~/.cache/inpc_rast/autotune.json``; writes go through a temporary file and
a rename, so concurrent processes never read a torn file.
"""
from __future__ import annotations

import ctypes as ct
import json
import math
import os
import tempfile
import time
from dataclasses import dataclass, field

from . import rast

L2_FLUSH_BYTES = 256 << 20  # larger than the 129 MB L2 of the target GPU


def cache_path() -> str:
    p = os.environ.get("INPC_RAST_TUNE_CACHE")
    if p:
        return p
    return os.path.join(os.path.expanduser("~"), ".cache", "inpc_rast", "autotune.json")


def _bucket(x: int) -> int:
    return int(round(math.log2(x))) if x > 0 else 0


def _view_totals(cviews):
    px = sum(int(v.cam.width) * int(v.cam.height) for v in cviews)
    pts = sum(int(v.pts.n) for v in cviews)
    return px, pts


def tune_key(device_name: str, opts, cviews, passes: int) -> str:
    """Cache key of a workload (the split only depends on these)."""
    px, pts = _view_totals(cviews)
    v0 = cviews[0].pts
    mode = {rast.BILINEAR: "bilinear", rast.GAUSSIAN: "gaussian"}.get(int(opts.mode), str(opts.mode))
    dt = "bf16" if int(v0.feat_dtype) == rast.BF16 else "f32"
    return (f"{device_name}|{mode}|C{int(v0.channels)}|{dt}|pass{int(passes)}|views{len(cviews)}"
            f"|px2^{_bucket(px)}|pts2^{_bucket(pts)}")


def select(timings: dict, margin: float = 0.01) -> tuple:
    """Fastest candidate, where a later candidate must beat the best
    earlier one by more than `margin` (relative): near-ties, which run-to-run
    noise would otherwise decide, go to the earlier candidate (the default
    first), so the choice is stable."""
    best, best_ms = None, math.inf
    for cand, ms in timings.items():
        if ms is not None and ms < best_ms * (1.0 - margin):
            best, best_ms = cand, ms
    return best


@dataclass
class TuneResult:
    tile: int
    blend_depth: int
    timings_ms: dict = field(default_factory=dict)
    key: str = ""
    from_cache: bool = False
    save_copy: bool = False  # RAST_FLAG_SAVE_FOR_BWD in the chosen opts


def _label(cand) -> str:
    t, d, save = cand
    return f"{t}x{d}" + ("+copy" if save else "")


def candidates_for(opts, passes: int, pairs) -> list:
    """(tile, depth, save_copy) triples to time: every pair as the caller's
    flag has it, and, when the copy can matter (bilinear, a backward, the
    caller allows it), every pair again with the copy."""
    allow = bool(int(opts.flags) & rast.FLAG_SAVE_FOR_BWD)
    bilinear = int(opts.mode) == rast.BILINEAR
    if allow and (passes & rast.PASS_BWD) and bilinear:
        return [(t, d, False) for t, d in pairs] + [(t, d, True) for t, d in pairs]
    return [(t, d, allow and bilinear) for t, d in pairs]  # Gaussian mode keeps no record copy


def load_cache(path: str | None = None) -> dict:
    path = path or cache_path()
    try:
        with open(path) as f:
            d = json.load(f)
        return d if isinstance(d, dict) else {}
    except (OSError, ValueError):
        return {}


def store_cache(key: str, res: TuneResult, path: str | None = None):
    path = path or cache_path()
    os.makedirs(os.path.dirname(path) or ".", exist_ok=True)
    d = load_cache(path)
    d[key] = {"tile": res.tile, "blend_depth": res.blend_depth, "save_copy": bool(res.save_copy),
              "timings_ms": {_label(c): ms for c, ms in res.timings_ms.items()},
              "time": time.strftime("%Y-%m-%dT%H:%M:%S")}
    fd, tmp = tempfile.mkstemp(prefix=".autotune.", dir=os.path.dirname(path) or ".")
    with os.fdopen(fd, "w") as f:
        json.dump(d, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def with_split(opts, tile: int, depth: int, save_copy: bool | None = None):
    """A copy of `opts` with this split (and the record-copy flag set or
    cleared, unless save_copy is None)."""
    o = rast.Opts()
    ct.memmove(ct.byref(o), ct.byref(opts), ct.sizeof(rast.Opts))
    o.tile, o.blend_depth = int(tile), int(depth)
    if save_copy is not None:
        o.flags = (int(o.flags) | rast.FLAG_SAVE_FOR_BWD) if save_copy else (int(o.flags) & ~rast.FLAG_SAVE_FOR_BWD)
    return o


def cuda_timer(cviews, passes: int, stream=None, reps: int = 5, warmup: int = 2):
    """Returns timer(opts) -> median ms of one rasterize_batch call."""
    import torch

    dev = torch.cuda.current_device()
    s = stream if stream is not None else torch.cuda.current_stream(dev)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)

    def timer(opts):
        nbytes = rast.rasterize_workspace_size(cviews, opts)
        ws = torch.empty(nbytes, dtype=torch.uint8, device=dev)
        for _ in range(warmup):
            rast.rasterize_batch(cviews, passes, opts, ws, s)
        st, _ = rast.rasterize_get_status(ws, s)
        if st != rast.RAST_OK:
            return None  # capacity or other failure: not a candidate
        out = []
        for _ in range(reps):
            flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(s)
            rast.rasterize_batch(cviews, passes, opts, ws, s)
            e1.record(s)
            e1.synchronize()
            out.append(e0.elapsed_time(e1))
        del ws
        out.sort()
        return out[len(out) // 2]

    return timer


def autotune(cviews, opts, passes: int = rast.PASS_FWD | rast.PASS_BWD, stream=None, *,
             device_name: str | None = None, timer=None, use_cache: bool = True,
             cache_file: str | None = None, candidates=None) -> TuneResult:
    """Pick (tile, blend_depth, record copy) for these views; returns the
    result and leaves ``opts`` untouched (apply it with ``with_split``)."""
    if device_name is None:
        import torch
        device_name = torch.cuda.get_device_name()
    allow = bool(int(opts.flags) & rast.FLAG_SAVE_FOR_BWD)
    key = tune_key(device_name, opts, cviews, passes)
    if use_cache:
        hit = load_cache(cache_file).get(key)
        if hit and "tile" in hit and "blend_depth" in hit:
            return TuneResult(int(hit["tile"]), int(hit["blend_depth"]), {}, key, True,
                              bool(hit.get("save_copy", False)) and allow)
    if candidates is None:
        candidates = rast.rasterize_tune_candidates(int(opts.mode))
    cands = candidates_for(opts, passes, [c[:2] for c in candidates])
    if timer is None:
        timer = cuda_timer(cviews, passes, stream)
    timings = {}
    for c in cands:
        timings[c] = timer(with_split(opts, c[0], c[1], c[2]))
    best = select(timings)
    if best is None:
        raise RuntimeError(f"autotune: no candidate ran ({timings})")
    res = TuneResult(best[0], best[1], timings, key, False, bool(best[2]))
    if use_cache:
        store_cache(key, res, cache_file)
    return res
