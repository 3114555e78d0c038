"""Thin Python binding of the C ABI in ``include/inpc_rast.h``.

Argument marshalling only: every step of the rasterizer runs in the CUDA
library ``_build/libinpcrast.so``. PyTorch provides device memory and the
stream. There is no CPU fallback: if the library is missing the import of a
compute function raises.

Low level (same names as the C ABI): ``rasterize_fwd``, ``rasterize_bwd``,
``rasterize_batch``, ``rasterize_workspace_size``, ``rasterize_get_status``,
``rasterize_workspace_layout``, ``rasterize_profile_enable``,
``rasterize_profile_read``. High level: ``rasterize`` / ``RasterizePoints``
(autograd, one view) and ``rasterize_views`` (autograd, several views in one
batched call).
"""
from __future__ import annotations

import ctypes as ct
import os
import threading

import numpy as np
import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libinpcrast.so")
_lib = None
_lock = threading.Lock()

RAST_OK, RAST_ERR_ARG, RAST_ERR_CAPACITY, RAST_ERR_CUDA, RAST_ERR_TIMEOUT, RAST_ERR_NOT_SUPPORTED = range(6)
BILINEAR, GAUSSIAN = 0, 1
GAUSS_EWA, GAUSS_ISO = 0, 1
F32, BF16 = 0, 1
PASS_FWD, PASS_BWD = 1, 2
FLAG_TEST_SORT_STALL = 1  # RAST_FLAG_TEST_SORT_STALL: failure-path tests only
FLAG_SAVE_FOR_BWD = 2     # RAST_FLAG_SAVE_FOR_BWD: the forward keeps a tile-ordered record copy for the backward
FLAG_TEST_BLEND_STALL = 4  # RAST_FLAG_TEST_BLEND_STALL: failure-path tests only


class RastError(RuntimeError):
    def __init__(self, status, what=""):
        self.status = int(status)
        super().__init__(f"{what}: {status_string(status)} ({status})")


class Camera(ct.Structure):
    _fields_ = [("fx", ct.c_float), ("fy", ct.c_float), ("cx", ct.c_float), ("cy", ct.c_float),
                ("R", ct.c_float * 9), ("t", ct.c_float * 3), ("near_z", ct.c_float),
                ("far_z", ct.c_float), ("width", ct.c_int32), ("height", ct.c_int32)]


class Points(ct.Structure):
    _fields_ = [("n", ct.c_int64), ("xyz", ct.c_void_p), ("opacity", ct.c_void_p),
                ("feat", ct.c_void_p), ("feat_dtype", ct.c_int32), ("channels", ct.c_int32),
                ("scale", ct.c_void_p)]


class Opts(ct.Structure):
    _fields_ = [("mode", ct.c_int32), ("gauss_cov", ct.c_int32), ("tile", ct.c_int32),
                ("blend_depth", ct.c_int32), ("t_min", ct.c_float), ("alpha_max", ct.c_float),
                ("dilation", ct.c_float), ("max_copies", ct.c_int32), ("flags", ct.c_int32)]


class Images(ct.Structure):
    _fields_ = [("feat", ct.c_void_p), ("alpha", ct.c_void_p), ("depth", ct.c_void_p)]


class Grads(ct.Structure):
    _fields_ = [("g_feat", ct.c_void_p), ("g_alpha", ct.c_void_p), ("g_depth", ct.c_void_p),
                ("d_feat", ct.c_void_p), ("d_opacity", ct.c_void_p), ("d_xyz", ct.c_void_p),
                ("d_scale", ct.c_void_p)]


class View(ct.Structure):
    _fields_ = [("pts", Points), ("cam", Camera), ("out", Images), ("grad", Grads)]


class Stats(ct.Structure):
    _fields_ = [("status", ct.c_int32), ("n_views", ct.c_int32), ("n_points", ct.c_int64),
                ("n_copies", ct.c_int64), ("copy_capacity", ct.c_int64),
                ("needed_records", ct.c_int64), ("n_tiles", ct.c_int64), ("n_pixels", ct.c_int64),
                ("needed_records_bwd", ct.c_int64)]


class ProfileEntry(ct.Structure):
    _fields_ = [("name", ct.c_char * 32), ("launches", ct.c_int32), ("total_ms", ct.c_double)]


class EnvMap(ct.Structure):
    _fields_ = [("map", ct.c_void_p), ("height", ct.c_int32), ("width", ct.c_int32),
                ("channels", ct.c_int32)]


class WsEntry(ct.Structure):
    _fields_ = [("name", ct.c_char * 24), ("offset", ct.c_int64), ("bytes", ct.c_int64)]


# Every function the header declares, with its ctypes signature.
SIGNATURES = {
    "rast_default_opts": (None, [ct.POINTER(Opts)]),
    "rasterize_workspace_size": (ct.c_size_t, [ct.POINTER(View), ct.c_int32, ct.POINTER(Opts)]),
    "rasterize_fwd": (ct.c_int, [ct.POINTER(Points), ct.POINTER(Camera), ct.POINTER(Opts),
                                 ct.c_void_p, ct.c_size_t, ct.POINTER(Images), ct.c_void_p]),
    "rasterize_fwd_noalloc": (ct.c_int, [ct.POINTER(Points), ct.POINTER(Camera), ct.POINTER(Opts),
                                         ct.POINTER(Images), ct.c_void_p]),
    "rasterize_bwd": (ct.c_int, [ct.POINTER(Points), ct.POINTER(Camera), ct.POINTER(Opts),
                                 ct.c_void_p, ct.c_size_t, ct.POINTER(Grads), ct.c_void_p]),
    "rasterize_batch": (ct.c_int, [ct.POINTER(View), ct.c_int32, ct.c_int32, ct.POINTER(Opts),
                                   ct.c_void_p, ct.c_size_t, ct.c_void_p]),
    "rasterize_get_status": (ct.c_int, [ct.c_void_p, ct.c_size_t, ct.c_void_p, ct.POINTER(Stats)]),
    "rasterize_noalloc_get_status": (ct.c_int, [ct.c_void_p, ct.POINTER(Stats)]),
    "rasterize_status_string": (ct.c_char_p, [ct.c_int]),
    "rasterize_workspace_layout": (ct.c_int32, [ct.POINTER(View), ct.c_int32, ct.POINTER(Opts),
                                                ct.POINTER(WsEntry), ct.c_int32]),
    "rasterize_profile_enable": (None, [ct.c_int32]),
    "rasterize_profile_read": (ct.c_int32, [ct.POINTER(ProfileEntry), ct.c_int32]),
    "rasterize_untiled_workspace_size": (ct.c_size_t, [ct.POINTER(Points), ct.POINTER(Camera), ct.POINTER(Opts)]),
    "rasterize_fwd_untiled": (ct.c_int, [ct.POINTER(Points), ct.POINTER(Camera), ct.POINTER(Opts), ct.c_void_p,
                                         ct.c_size_t, ct.POINTER(Images), ct.c_void_p]),
    "rasterize_untiled64_workspace_size": (ct.c_size_t, [ct.POINTER(Points), ct.POINTER(Camera), ct.POINTER(Opts)]),
    "rasterize_untiled64_workspace_layout": (ct.c_int32, [ct.POINTER(Points), ct.POINTER(Camera), ct.POINTER(Opts),
                                                          ct.POINTER(WsEntry), ct.c_int32]),
    "rasterize_fwd_untiled64": (ct.c_int, [ct.POINTER(Points), ct.POINTER(Camera), ct.POINTER(Opts), ct.c_void_p,
                                           ct.c_size_t, ct.POINTER(Images), ct.c_void_p]),
    "rasterize_clouds_workspace_size": (ct.c_size_t, [ct.POINTER(Points), ct.c_int32, ct.POINTER(Camera),
                                                      ct.POINTER(Opts)]),
    "rasterize_clouds": (ct.c_int, [ct.POINTER(Points), ct.POINTER(Grads), ct.c_int32, ct.POINTER(Camera),
                                    ct.POINTER(Images), ct.c_int32, ct.POINTER(Opts), ct.c_void_p, ct.c_size_t,
                                    ct.c_void_p]),
    "rasterize_contract": (ct.c_int, [ct.c_void_p, ct.c_void_p, ct.c_int64, ct.c_void_p]),
    "rasterize_view_dirs": (ct.c_int, [ct.POINTER(Camera), ct.c_void_p, ct.c_void_p]),
    "rasterize_bg_composite": (ct.c_int, [ct.POINTER(Camera), ct.POINTER(EnvMap), ct.c_void_p, ct.c_void_p,
                                          ct.c_void_p, ct.c_void_p, ct.c_void_p]),
    "rasterize_bg_scratch_size": (ct.c_size_t, [ct.POINTER(EnvMap)]),
    "rasterize_bg_composite_bwd": (ct.c_int, [ct.POINTER(Camera), ct.POINTER(EnvMap), ct.c_void_p, ct.c_void_p,
                                              ct.c_void_p, ct.c_void_p, ct.c_void_p, ct.c_void_p, ct.c_size_t,
                                              ct.c_void_p]),
    "rasterize_tune_candidates": (ct.c_int32, [ct.c_int32, ct.POINTER(ct.c_int32), ct.POINTER(ct.c_int32),
                                               ct.c_int32]),
    "rasterize_version": (ct.c_char_p, []),
}


def library_path() -> str:
    return LIB_PATH


def load_library(path: str | None = None):
    """Load the CUDA library. Raises if it has not been built."""
    global _lib
    with _lock:
        if _lib is None:
            p = path or LIB_PATH
            if not os.path.exists(p):
                raise RuntimeError(
                    f"CUDA rasterizer library not found at {p}; build it with "
                    "paper_2508_19140_gb300.build.build() (there is no CPU fallback)")
            L = ct.CDLL(p)
            for name, (res, args) in SIGNATURES.items():
                fn = getattr(L, name)
                fn.restype = res
                fn.argtypes = args
            _lib = L
    return _lib


def status_string(s) -> str:
    try:
        return load_library().rasterize_status_string(int(s)).decode()
    except RuntimeError:
        return f"status {int(s)}"


def _check(status, what):
    if status != RAST_OK:
        raise RastError(status, what)


# ---------------------------------------------------------------- marshalling

def make_opts(mode="bilinear", gauss_cov="ewa", tile=16, blend_depth=0, t_min=1e-4,
              alpha_max=0.99, dilation=0.16, max_copies=0, flags=0) -> Opts:
    o = Opts()
    load_library().rast_default_opts(ct.byref(o))
    o.mode = {"bilinear": BILINEAR, "gaussian": GAUSSIAN}.get(mode, mode)
    o.gauss_cov = {"ewa": GAUSS_EWA, "iso": GAUSS_ISO}.get(gauss_cov, gauss_cov)
    o.tile, o.blend_depth = int(tile), int(blend_depth)
    o.t_min, o.alpha_max, o.dilation = float(t_min), float(alpha_max), float(dilation)
    o.max_copies = int(max_copies)
    o.flags = int(flags)
    return o


def make_camera(cam) -> Camera:
    """From any object with fx, fy, cx, cy, R (3x3), t (3), width, height, near, far."""
    c = Camera()
    c.fx, c.fy, c.cx, c.cy = float(cam.fx), float(cam.fy), float(cam.cx), float(cam.cy)
    R = np.asarray(cam.R, np.float32).reshape(9)
    t = np.asarray(cam.t, np.float32).reshape(3)
    for k in range(9):
        c.R[k] = float(R[k])
    for k in range(3):
        c.t[k] = float(t[k])
    c.near_z = float(getattr(cam, "near", 0.2))
    c.far_z = float(getattr(cam, "far", 1e4))
    c.width, c.height = int(cam.width), int(cam.height)
    return c


def _nbytes(t) -> int:
    """Size in bytes of a workspace or scratch tensor (any dtype)."""
    return int(t.numel() * t.element_size())


def _ptr(t):
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError("device tensors are required (the rasterizer runs on the GPU only)")
    if not t.is_contiguous():
        raise ValueError("tensors must be contiguous")
    return ct.c_void_p(t.data_ptr())


def make_points(xyz, opacity, feat, scale=None) -> Points:
    p = Points()
    p.n = int(xyz.shape[0])
    p.xyz, p.opacity, p.feat = _ptr(xyz), _ptr(opacity), _ptr(feat)
    if feat.dtype == torch.float32:
        p.feat_dtype = F32
    elif feat.dtype == torch.bfloat16:
        p.feat_dtype = BF16
    else:
        raise ValueError("features must be float32 or bfloat16")
    p.channels = int(feat.shape[1])
    p.scale = _ptr(scale)
    return p


def make_images(feat, alpha=None, depth=None) -> Images:
    im = Images()
    im.feat, im.alpha, im.depth = _ptr(feat), _ptr(alpha), _ptr(depth)
    return im


def make_grads(g_feat, g_alpha=None, g_depth=None, d_feat=None, d_opacity=None, d_xyz=None,
               d_scale=None) -> Grads:
    g = Grads()
    g.g_feat, g.g_alpha, g.g_depth = _ptr(g_feat), _ptr(g_alpha), _ptr(g_depth)
    g.d_feat, g.d_opacity, g.d_xyz, g.d_scale = _ptr(d_feat), _ptr(d_opacity), _ptr(d_xyz), _ptr(d_scale)
    return g


def _stream(stream):
    if stream is None:
        stream = torch.cuda.current_stream()
    return ct.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))


def _view_array(views):
    arr = (View * len(views))()
    for k, v in enumerate(views):
        arr[k] = v
    return arr


# ---------------------------------------------------------------- C ABI, same names

def rasterize_workspace_size(views, opts: Opts) -> int:
    arr = _view_array(views)
    n = load_library().rasterize_workspace_size(arr, len(views), ct.byref(opts))
    if n == 0:
        raise RastError(RAST_ERR_ARG, "rasterize_workspace_size")
    return int(n)


def rasterize_fwd(points: Points, camera: Camera, opts: Opts, workspace, out: Images, stream=None):
    s = load_library().rasterize_fwd(ct.byref(points), ct.byref(camera), ct.byref(opts),
                                     _ptr(workspace), _nbytes(workspace), ct.byref(out), _stream(stream))
    _check(s, "rasterize_fwd")


def rasterize_fwd_noalloc(points: Points, camera: Camera, opts: Opts, out: Images, stream=None):
    """Forward of one view without a workspace or any device allocation (the
    library's static 16 MiB scratch holds the intermediates); raises RastError
    with RAST_ERR_CAPACITY when the problem does not fit. Errors the GPU
    raises during the pass are read with rasterize_noalloc_get_status."""
    s = load_library().rasterize_fwd_noalloc(ct.byref(points), ct.byref(camera), ct.byref(opts),
                                             ct.byref(out), _stream(stream))
    _check(s, "rasterize_fwd_noalloc")


def rasterize_noalloc_get_status(stream=None):
    """(status, counters) of the last rasterize_fwd_noalloc on this device."""
    st = Stats()
    s = load_library().rasterize_noalloc_get_status(_stream(stream), ct.byref(st))
    stats = {f: getattr(st, f) for f, _ in Stats._fields_}
    return int(s), stats


def rasterize_bwd(points: Points, camera: Camera, opts: Opts, workspace, grads: Grads, stream=None):
    s = load_library().rasterize_bwd(ct.byref(points), ct.byref(camera), ct.byref(opts),
                                     _ptr(workspace), _nbytes(workspace), ct.byref(grads), _stream(stream))
    _check(s, "rasterize_bwd")


def rasterize_batch(views, pass_: int, opts: Opts, workspace, stream=None):
    arr = _view_array(views)
    s = load_library().rasterize_batch(arr, len(views), int(pass_), ct.byref(opts), _ptr(workspace),
                                       _nbytes(workspace), _stream(stream))
    _check(s, "rasterize_batch")


def rasterize_get_status(workspace, stream=None):
    st = Stats()
    s = load_library().rasterize_get_status(_ptr(workspace), _nbytes(workspace), _stream(stream),
                                            ct.byref(st))
    stats = {f: getattr(st, f) for f, _ in Stats._fields_}
    return int(s), stats


def rasterize_workspace_layout(views, opts: Opts) -> dict:
    arr = _view_array(views)
    L = load_library()
    n = L.rasterize_workspace_layout(arr, len(views), ct.byref(opts), None, 0)
    if n < 0:
        raise RastError(RAST_ERR_ARG, "rasterize_workspace_layout")
    ents = (WsEntry * n)()
    L.rasterize_workspace_layout(arr, len(views), ct.byref(opts), ents, n)
    return {e.name.decode(): (int(e.offset), int(e.bytes)) for e in ents}


def rasterize_profile_enable(on: bool):
    load_library().rasterize_profile_enable(1 if on else 0)


def rasterize_profile_read() -> dict:
    L = load_library()
    ents = (ProfileEntry * 64)()
    n = L.rasterize_profile_read(ents, 64)
    return {ents[k].name.decode(): (int(ents[k].launches), float(ents[k].total_ms))
            for k in range(min(n, 64))}


def rasterize_untiled_workspace_size(points: Points, camera: Camera, opts: Opts) -> int:
    n = load_library().rasterize_untiled_workspace_size(ct.byref(points), ct.byref(camera), ct.byref(opts))
    if n == 0:
        raise RastError(RAST_ERR_ARG, "rasterize_untiled_workspace_size")
    return int(n)


def rasterize_fwd_untiled(points: Points, camera: Camera, opts: Opts, workspace, out: Images, stream=None):
    _check(load_library().rasterize_fwd_untiled(ct.byref(points), ct.byref(camera), ct.byref(opts),
                                                _ptr(workspace), _nbytes(workspace),
                                                ct.byref(out), _stream(stream)),
           "rasterize_fwd_untiled")


def rasterize_untiled64_workspace_size(points: Points, camera: Camera, opts: Opts) -> int:
    n = load_library().rasterize_untiled64_workspace_size(ct.byref(points), ct.byref(camera), ct.byref(opts))
    if n == 0:
        raise RastError(RAST_ERR_ARG, "rasterize_untiled64_workspace_size")
    return int(n)


def rasterize_untiled64_workspace_layout(points: Points, camera: Camera, opts: Opts) -> dict:
    L = load_library()
    n = L.rasterize_untiled64_workspace_layout(ct.byref(points), ct.byref(camera), ct.byref(opts), None, 0)
    if n < 0:
        raise RastError(RAST_ERR_ARG, "rasterize_untiled64_workspace_layout")
    ents = (WsEntry * n)()
    L.rasterize_untiled64_workspace_layout(ct.byref(points), ct.byref(camera), ct.byref(opts), ents, n)
    return {e.name.decode(): (int(e.offset), int(e.bytes)) for e in ents}


def rasterize_fwd_untiled64(points: Points, camera: Camera, opts: Opts, workspace, out: Images, stream=None):
    s = load_library().rasterize_fwd_untiled64(ct.byref(points), ct.byref(camera), ct.byref(opts),
                                               _ptr(workspace), _nbytes(workspace), ct.byref(out), _stream(stream))
    _check(s, "rasterize_fwd_untiled64")


def rasterize_clouds_workspace_size(clouds, camera: Camera, opts: Opts) -> int:
    arr = (Points * len(clouds))(*clouds)
    n = load_library().rasterize_clouds_workspace_size(arr, len(clouds), ct.byref(camera), ct.byref(opts))
    if n == 0:
        raise RastError(RAST_ERR_ARG, "rasterize_clouds_workspace_size")
    return int(n)


def rasterize_clouds(clouds, grads, camera: Camera, out: Images, pass_: int, opts: Opts, workspace,
                     stream=None):
    """clouds: list of Points; grads: list of Grads (one per cloud) or None."""
    arr = (Points * len(clouds))(*clouds)
    garr = None if grads is None else (Grads * len(grads))(*grads)
    _check(load_library().rasterize_clouds(arr, garr, len(clouds), ct.byref(camera), ct.byref(out), int(pass_),
                                           ct.byref(opts), _ptr(workspace),
                                           _nbytes(workspace), _stream(stream)),
           "rasterize_clouds")


def rasterize_contract(xyz, out, stream=None):
    """Spherical contraction of [n, 3] positions (out may be xyz)."""
    _check(load_library().rasterize_contract(_ptr(xyz), _ptr(out), int(xyz.shape[0]), _stream(stream)),
           "rasterize_contract")


def make_envmap(env) -> EnvMap:
    """env: device FP32 tensor [H_b, W_b, C] (contiguous)."""
    e = EnvMap()
    e.map = _ptr(env)
    e.height, e.width, e.channels = int(env.shape[0]), int(env.shape[1]), int(env.shape[2])
    return e


def rasterize_view_dirs(camera: Camera, dirs, stream=None):
    _check(load_library().rasterize_view_dirs(ct.byref(camera), _ptr(dirs), _stream(stream)),
           "rasterize_view_dirs")


def rasterize_bg_composite(camera: Camera, env: EnvMap, dirs, feat, alpha, out, stream=None):
    _check(load_library().rasterize_bg_composite(ct.byref(camera), ct.byref(env), _ptr(dirs), _ptr(feat),
                                                 _ptr(alpha), _ptr(out), _stream(stream)),
           "rasterize_bg_composite")


def rasterize_bg_scratch_size(env: EnvMap) -> int:
    return int(load_library().rasterize_bg_scratch_size(ct.byref(env)))


def rasterize_bg_composite_bwd(camera: Camera, env: EnvMap, dirs, alpha, g, g_alpha, d_map, scratch,
                               stream=None):
    _check(load_library().rasterize_bg_composite_bwd(ct.byref(camera), ct.byref(env), _ptr(dirs), _ptr(alpha),
                                                     _ptr(g), _ptr(g_alpha), _ptr(d_map), _ptr(scratch),
                                                     _nbytes(scratch),
                                                     _stream(stream)),
           "rasterize_bg_composite_bwd")


def rasterize_tune_candidates(mode="bilinear"):
    """Compiled (tile, blend_depth) pairs for a splat mode, default first."""
    m = {"bilinear": BILINEAR, "gaussian": GAUSSIAN}.get(mode, mode)
    L = load_library()
    n = L.rasterize_tune_candidates(int(m), None, None, 0)
    if n < 0:
        raise RastError(RAST_ERR_ARG, "rasterize_tune_candidates")
    tiles, depths = (ct.c_int32 * max(n, 1))(), (ct.c_int32 * max(n, 1))()
    L.rasterize_tune_candidates(int(m), tiles, depths, n)
    return [(int(tiles[k]), int(depths[k])) for k in range(n)]


def rasterize_version() -> str:
    return load_library().rasterize_version().decode()


# ---------------------------------------------------------------- autograd

def _alloc_ws(views, opts, device):
    n = rasterize_workspace_size(views, opts)
    return torch.empty(n, dtype=torch.uint8, device=device)


class _Batch(torch.autograd.Function):
    """Differentiable batched rasterization. Inputs are flattened per view as
    (xyz, opacity, feat, scale) tuples; outputs are (F, alpha, depth) per view."""

    @staticmethod
    def forward(ctx, cams, opts_kw, check, n_views, *flat):
        if any(ctx.needs_input_grad[4:]):
            # a backward will follow: keep the tile-ordered record copy for it
            opts_kw = dict(opts_kw, flags=int(opts_kw.get("flags", 0)) | FLAG_SAVE_FOR_BWD)
        opts = make_opts(**opts_kw)
        dev = flat[0].device
        pts, views, outs = [], [], []
        for k in range(n_views):
            xyz, op, feat, scale = flat[4 * k: 4 * k + 4]
            cam = cams[k]
            H, W, C = cam.height, cam.width, feat.shape[1]
            F = torch.empty((H, W, C), dtype=torch.float32, device=dev)
            A = torch.empty((H, W), dtype=torch.float32, device=dev)
            Dp = torch.empty((H, W), dtype=torch.float32, device=dev)
            v = View()
            v.pts = make_points(xyz, op, feat, scale)
            v.cam = make_camera(cam)
            v.out = make_images(F, A, Dp)
            views.append(v)
            outs += [F, A, Dp]
            pts.append((xyz, op, feat, scale))
        ws = _alloc_ws(views, opts, dev)
        rasterize_batch(views, PASS_FWD, opts, ws)
        if check:
            st, stats = rasterize_get_status(ws)
            if st != RAST_OK:
                raise RastError(st, f"rasterize forward ({stats})")
        ctx.cams, ctx.opts_kw, ctx.n_views = cams, opts_kw, n_views
        ctx.save_for_backward(ws, *[t for p in pts for t in p if t is not None])
        ctx.has_scale = [p[3] is not None for p in pts]
        ctx.feat_dtypes = [p[2].dtype for p in pts]
        return tuple(outs)

    @staticmethod
    def backward(ctx, *gouts):
        saved = ctx.saved_tensors
        ws = saved[0]
        it = iter(saved[1:])
        opts = make_opts(**ctx.opts_kw)
        gauss = opts.mode == GAUSSIAN
        dev = ws.device
        views, grads_out = [], []
        for k in range(ctx.n_views):
            xyz, op, feat = next(it), next(it), next(it)
            scale = next(it) if ctx.has_scale[k] else None
            gF, gA, gD = gouts[3 * k: 3 * k + 3]
            if gF is None:
                gF = torch.zeros((ctx.cams[k].height, ctx.cams[k].width, feat.shape[1]),
                                 dtype=torch.float32, device=dev)
            else:
                gF = gF.contiguous().float()
            gA = None if gA is None else gA.contiguous().float()
            gD = None if gD is None else gD.contiguous().float()
            n = xyz.shape[0]
            d_feat = torch.empty((n, feat.shape[1]), dtype=torch.float32, device=dev)
            d_op = torch.empty((n,), dtype=torch.float32, device=dev)
            d_xyz = torch.empty((n, 3), dtype=torch.float32, device=dev) if gauss else None
            d_scale = torch.empty((n,), dtype=torch.float32, device=dev) if (gauss and scale is not None) else None
            v = View()
            v.pts = make_points(xyz, op, feat, scale)
            v.cam = make_camera(ctx.cams[k])
            v.grad = make_grads(gF, gA, gD, d_feat, d_op, d_xyz, d_scale)
            views.append(v)
            grads_out.append([d_xyz, d_op, d_feat, d_scale])
            # keep upstream gradient tensors alive until the launch is enqueued
            v._keep = (gF, gA, gD)
        rasterize_batch(views, PASS_BWD, opts, ws)
        flat = []
        for k, (d_xyz, d_op, d_feat, d_scale) in enumerate(grads_out):
            # dL/df is FP32; cast to the features' dtype only after the kernels
            # that write it are enqueued
            flat += [d_xyz, d_op, d_feat.to(ctx.feat_dtypes[k]), d_scale]
        return (None, None, None, None) + tuple(flat)


def rasterize_views(items, mode="bilinear", gauss_cov="ewa", check=True, **opt_kw):
    """items: list of (xyz [N,3] f32, opacity [N] f32, feat [N,C] f32|bf16,
    camera, scale [N] f32 or None). Returns a list of (F, alpha, depth)."""
    cams = [it[3] for it in items]
    flat = []
    for it in items:
        xyz, op, feat, cam = it[:4]
        scale = it[4] if len(it) > 4 else None
        flat += [xyz.contiguous(), op.contiguous(), feat.contiguous(),
                 None if scale is None else scale.contiguous()]
    kw = dict(mode=mode, gauss_cov=gauss_cov, **opt_kw)
    outs = _Batch.apply(cams, kw, check, len(items), *flat)
    return [tuple(outs[3 * k: 3 * k + 3]) for k in range(len(items))]


def rasterize(xyz, opacity, feat, camera, scale=None, mode="bilinear", gauss_cov="ewa",
              check=True, **opt_kw):
    """Differentiable rasterization of one view: returns (F [H,W,C], alpha [H,W], depth [H,W])."""
    return rasterize_views([(xyz, opacity, feat, camera, scale)], mode=mode, gauss_cov=gauss_cov,
                           check=check, **opt_kw)[0]


RasterizePoints = _Batch
