"""CPU oracle for the tiled point rasterizer -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package. It is a plain, slow, FP64 restatement
of what the rasterizer computes (see ``oracle.cpp`` for the definition and the
passages it follows) and shares no code with the CUDA path.
"""
from __future__ import annotations

import ctypes as ct
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.cpp")
_SRCS = [_SRC, os.path.join(_HERE, "envmap.cpp")]
_OUT_DIR = os.path.join(_HERE, "_build")
# A prebuilt oracle library to load instead of building this one: the
# planted-mistake test points it at deliberately broken variants.
_OVERRIDE = os.environ.get("INPC_ORACLE_LIB")
_LIB_PATH = _OVERRIDE or os.path.join(_OUT_DIR, "liboracle.so")
_lock = threading.Lock()
_lib = None

MODE = {"bilinear": 0, "gaussian": 1}
GAUSS_COV = {"ewa": 0, "iso": 1}


class OrcCamera(ct.Structure):
    _fields_ = [("fx", ct.c_float), ("fy", ct.c_float), ("cx", ct.c_float), ("cy", ct.c_float),
                ("R", ct.c_float * 9), ("t", ct.c_float * 3), ("near_z", ct.c_float),
                ("far_z", ct.c_float), ("width", ct.c_int32), ("height", ct.c_int32)]


class OrcOpts(ct.Structure):
    _fields_ = [("mode", ct.c_int32), ("gauss_cov", ct.c_int32), ("tile", ct.c_int32),
                ("pin32", ct.c_int32), ("t_min", ct.c_float), ("alpha_max", ct.c_float),
                ("dilation", ct.c_float), ("n_threads", ct.c_int32)]


def compile_command(sources, out):
    """g++ command line that builds the oracle library from `sources`."""
    return ["g++", "-O2", "-std=c++17", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
            "-fno-fast-math", *sources, "-o", out]


def build(force: bool = False) -> str:
    """Compile the oracle (g++, -ffp-contract=off so FP32 decisions round op by op)."""
    if _OVERRIDE:
        return _OVERRIDE
    os.makedirs(_OUT_DIR, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and all(os.path.getmtime(_LIB_PATH) >= os.path.getmtime(s) for s in _SRCS)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    subprocess.run(compile_command(_SRCS, tmp), check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = ct.CDLL(_LIB_PATH)
            P = ct.c_void_p
            L.orc_num_threads.restype = ct.c_int
            L.orc_project.argtypes = [ct.c_int64, P, P, P, P, P, P, P, P, P, P, P, P]
            L.orc_project.restype = None
            L.orc_tile_lists.argtypes = [ct.c_int64, P, P, P, P, P, P, P]
            L.orc_tile_lists.restype = ct.c_int64
            L.orc_render.argtypes = [ct.c_int64, P, P, P, P, ct.c_int32, P, P, ct.c_int64, P,
                                     P, P, P, P, P, P, P, P, P, P]
            L.orc_render.restype = None
            L.orc_backward.argtypes = [ct.c_int64, P, P, P, P, ct.c_int32, P, P, P, P, P, P,
                                       P, P, P, P]
            L.orc_backward.restype = None
            L.orc_env_dirs.argtypes = [P, P]
            L.orc_env_dirs.restype = None
            L.orc_env_composite.argtypes = [P, P, ct.c_int32, ct.c_int32, ct.c_int32, P, P, P, P, P]
            L.orc_env_composite.restype = None
            L.orc_env_backward.argtypes = [P, P, ct.c_int32, ct.c_int32, ct.c_int32, P, P, P, P, P]
            L.orc_env_backward.restype = None
            L.orc_contract.argtypes = [ct.c_int64, P, P]
            L.orc_contract.restype = None
            _lib = L
    return _lib


def num_threads() -> int:
    return int(lib().orc_num_threads())


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ct.c_void_p)


def make_camera(cam) -> OrcCamera:
    c = OrcCamera()
    c.fx, c.fy, c.cx, c.cy = float(cam.fx), float(cam.fy), float(cam.cx), float(cam.cy)
    R = np.asarray(cam.R, np.float32).reshape(9)
    t = np.asarray(cam.t, np.float32).reshape(3)
    for k in range(9):
        c.R[k] = float(R[k])
    for k in range(3):
        c.t[k] = float(t[k])
    c.near_z, c.far_z = float(cam.near), float(cam.far)
    c.width, c.height = int(cam.width), int(cam.height)
    return c


def make_opts(mode="bilinear", gauss_cov="ewa", tile=16, pin32=True, t_min=1e-4,
              alpha_max=0.99, dilation=0.16, n_threads=0) -> OrcOpts:
    o = OrcOpts()
    o.mode = MODE[mode] if isinstance(mode, str) else int(mode)
    o.gauss_cov = GAUSS_COV[gauss_cov] if isinstance(gauss_cov, str) else int(gauss_cov)
    o.tile, o.pin32 = int(tile), int(bool(pin32))
    o.t_min, o.alpha_max, o.dilation = float(t_min), float(alpha_max), float(dilation)
    o.n_threads = int(n_threads)
    return o


def _in(a):
    # point inputs are FP64 (FP32 data promotes exactly)
    return None if a is None else np.ascontiguousarray(a, dtype=np.float64)


def _f64(a):
    return None if a is None else np.ascontiguousarray(a, dtype=np.float64)


def project(xyz, camera, scale=None, **kw):
    xyz = _in(xyz)
    n = xyz.shape[0]
    scale = _in(scale)
    out = dict(vis=np.zeros(n, np.int32), zbits=np.zeros(n, np.uint32),
               uvz=np.zeros((n, 3)), conic=np.zeros((n, 3)), box=np.zeros((n, 4), np.int32),
               anchor=np.zeros((n, 2), np.int32), frac=np.zeros((n, 2)), cov=np.zeros((n, 3)))
    cam, opt = make_camera(camera), make_opts(**kw)
    lib().orc_project(n, _ptr(xyz), _ptr(scale), ct.byref(cam), ct.byref(opt),
                      _ptr(out["vis"]), _ptr(out["zbits"]), _ptr(out["uvz"]), _ptr(out["conic"]),
                      _ptr(out["box"]), _ptr(out["anchor"]), _ptr(out["frac"]), _ptr(out["cov"]))
    return out


def tile_lists(xyz, camera, scale=None, want=None, **kw):
    """(tile id, point index) of every copy, ordered by (tile, depth bits, index)."""
    xyz, scale = _in(xyz), _in(scale)
    n = xyz.shape[0]
    cam, opt = make_camera(camera), make_opts(**kw)
    w = None if want is None else np.ascontiguousarray(want, dtype=np.uint8)
    D = lib().orc_tile_lists(n, _ptr(xyz), _ptr(scale), ct.byref(cam), ct.byref(opt), _ptr(w),
                             None, None)
    tiles = np.zeros(max(D, 1), np.int32)
    idx = np.zeros(max(D, 1), np.int32)
    lib().orc_tile_lists(n, _ptr(xyz), _ptr(scale), ct.byref(cam), ct.byref(opt), _ptr(w),
                         _ptr(tiles), _ptr(idx))
    return tiles[:D], idx[:D]


def render(xyz, opacity, feat, camera, scale=None, pix=None, **kw):
    """Forward render (all pixels, or the flat pixel indices ``pix``)."""
    xyz, opacity, scale = _in(xyz), _in(opacity), _in(scale)
    feat = _f64(feat)
    n, C = feat.shape
    W, H = int(camera.width), int(camera.height)
    pixa = None if pix is None else np.ascontiguousarray(pix, dtype=np.int64)
    k = W * H if pixa is None else len(pixa)
    out = dict(F=np.zeros((k, C)), alpha=np.zeros(k), depth=np.zeros(k), t_final=np.zeros(k),
               n_blend=np.zeros(k, np.int32), n_cover=np.zeros(k, np.int32),
               last_pos=np.zeros(k, np.int32), stop_pos=np.zeros(k, np.int32),
               margin=np.zeros(k))
    needed = np.zeros(1, np.int64)
    cam, opt = make_camera(camera), make_opts(**kw)
    lib().orc_render(n, _ptr(xyz), _ptr(opacity), _ptr(scale), _ptr(feat), C, ct.byref(cam),
                     ct.byref(opt), k, _ptr(pixa), _ptr(out["F"]), _ptr(out["alpha"]),
                     _ptr(out["depth"]), _ptr(out["t_final"]), _ptr(out["n_blend"]),
                     _ptr(out["n_cover"]), _ptr(out["last_pos"]), _ptr(out["stop_pos"]),
                     _ptr(out["margin"]), _ptr(needed))
    out["needed"] = int(needed[0])
    if pixa is None:
        out = {key: (v.reshape((H, W) + v.shape[1:]) if isinstance(v, np.ndarray) else v)
               for key, v in out.items()}
    return out


def backward(xyz, opacity, feat, camera, g_feat, g_alpha=None, g_depth=None, scale=None,
             pmask=None, **kw):
    """Adjoint: returns d_feat, d_opacity, d_xyz, d_scale (FP64)."""
    xyz, opacity, scale = _in(xyz), _in(opacity), _in(scale)
    feat = _f64(feat)
    n, C = feat.shape
    gF = _f64(g_feat).reshape(-1)
    gA = None if g_alpha is None else _f64(g_alpha).reshape(-1)
    gD = None if g_depth is None else _f64(g_depth).reshape(-1)
    pm = None if pmask is None else np.ascontiguousarray(pmask, dtype=np.uint8)
    out = dict(d_feat=np.zeros((n, C)), d_opacity=np.zeros(n), d_xyz=np.zeros((n, 3)),
               d_scale=np.zeros(n))
    cam, opt = make_camera(camera), make_opts(**kw)
    lib().orc_backward(n, _ptr(xyz), _ptr(opacity), _ptr(scale), _ptr(feat), C, ct.byref(cam),
                       ct.byref(opt), _ptr(pm), _ptr(gF), _ptr(gA), _ptr(gD),
                       _ptr(out["d_feat"]), _ptr(out["d_opacity"]), _ptr(out["d_xyz"]),
                       _ptr(out["d_scale"]))
    return out


# ----------------------------------------------------------------------------- background model

def env_dirs(camera):
    """Camera-space unit viewing direction of every pixel (H x W x 3), FP64."""
    cam = make_camera(camera)
    out = np.zeros((camera.height, camera.width, 3))
    lib().orc_env_dirs(ct.byref(cam), _ptr(out))
    return out


def env_composite(env, camera, F, alpha, dirs=None):
    """Sec. 3.2 "Faster Background Model Evaluation": out = F + (1 - alpha) f_bg,
    f_bg the bilinear lookup of the spherical map `env` (H_b x W_b x C) along each
    pixel's viewing direction. Returns (out, f_bg)."""
    env = _f64(env)
    Hb, Wb, C = env.shape
    cam = make_camera(camera)
    F, alpha, dirs = _f64(F), _f64(alpha), _f64(dirs)
    out = np.zeros(F.shape)
    bg = np.zeros(F.shape)
    lib().orc_env_composite(ct.byref(cam), _ptr(env), Hb, Wb, C, _ptr(dirs), _ptr(F), _ptr(alpha),
                            _ptr(out), _ptr(bg))
    return out, bg


def env_backward(env, camera, alpha, g, dirs=None):
    """Adjoint of env_composite for upstream gradient g (H x W x C): returns
    (dL/dalpha [H x W], dL/dmap [H_b x W_b x C]); dL/dF is g itself."""
    env = _f64(env)
    Hb, Wb, C = env.shape
    cam = make_camera(camera)
    alpha, g, dirs = _f64(alpha), _f64(g), _f64(dirs)
    d_alpha = np.zeros(alpha.shape)
    d_map = np.zeros(env.shape)
    lib().orc_env_backward(ct.byref(cam), _ptr(env), Hb, Wb, C, _ptr(dirs), _ptr(alpha), _ptr(g),
                           _ptr(d_alpha), _ptr(d_map))
    return d_alpha, d_map


def contract(xyz):
    """Spherical contraction x -> x (|x| <= 1) or (2 - 1/|x|) x/|x|, FP64."""
    x = _f64(xyz).reshape(-1, 3)
    out = np.zeros_like(x)
    lib().orc_contract(x.shape[0], _ptr(x), _ptr(out))
    return out
