"""CPU-only checks of the C ABI library: it builds, loads, exports every
function include/inpc_rast.h declares, and its host-side logic (defaults,
workspace sizing and layout, argument validation) behaves as documented.
No call here launches GPU work."""
import ctypes as ct
import os
import re

import numpy as np
import pytest

from paper_2508_19140_gb300 import build as build_mod
from paper_2508_19140_gb300 import rast

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "inpc_rast.h")


@pytest.fixture(scope="module")
def lib():
    build_mod.build()
    return rast.load_library()


def declared_functions():
    txt = open(HEADER).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    names = re.findall(r"\b([A-Za-z_]\w*)\s*\([^;{]*\)\s*;", txt)
    return sorted({n for n in names if n.startswith(("rast", "rasterize"))})


def test_header_declares_the_boundary():
    fns = declared_functions()
    for need in ("rasterize_fwd", "rasterize_bwd", "rasterize_batch", "rasterize_workspace_size",
                 "rasterize_get_status", "rasterize_status_string"):
        assert need in fns


def test_every_declared_symbol_is_exported(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name
        assert name in rast.SIGNATURES, f"binding lacks {name}"


def test_struct_sizes_match_header_layout(lib):
    # packed C layouts of the public structs (no padding surprises between ABI and binding)
    assert ct.sizeof(rast.Camera) == 4 * 18 + 8
    assert ct.sizeof(rast.Opts) == 9 * 4
    assert ct.sizeof(rast.Points) == 8 + 8 * 3 + 4 + 4 + 8
    assert ct.sizeof(rast.View) == (ct.sizeof(rast.Points) + ct.sizeof(rast.Camera) +
                                    ct.sizeof(rast.Images) + ct.sizeof(rast.Grads))


def test_default_opts(lib):
    o = rast.Opts()
    lib.rast_default_opts(ct.byref(o))
    assert (o.mode, o.gauss_cov, o.tile, o.blend_depth) == (0, 0, 16, 0)
    assert np.float32(o.t_min) == np.float32(1e-4)
    assert np.float32(o.alpha_max) == np.float32(0.99)
    assert np.float32(o.dilation) == np.float32(0.16)


def _fake_view(n=1000, W=100, H=60, C=4, dtype=0):
    v = rast.View()
    v.pts.n = n
    v.pts.xyz = v.pts.opacity = v.pts.feat = 4096  # never dereferenced on the host
    v.pts.feat_dtype = dtype
    v.pts.channels = C
    cam = v.cam
    cam.fx = cam.fy = 80.0
    cam.cx, cam.cy = W / 2, H / 2
    cam.R[0] = cam.R[4] = cam.R[8] = 1.0
    cam.near_z, cam.far_z = 0.2, 1e4
    cam.width, cam.height = W, H
    v.out.feat = 8192
    v.grad.g_feat = 8192
    return v


def _opts(lib, **kw):
    o = rast.Opts()
    lib.rast_default_opts(ct.byref(o))
    for k, val in kw.items():
        setattr(o, k, val)
    return o


def test_workspace_size_and_layout(lib):
    v = _fake_view()
    arr = (rast.View * 1)(v)
    o = _opts(lib)
    size = lib.rasterize_workspace_size(arr, 1, ct.byref(o))
    assert size > 0 and size % 256 == 0
    n = lib.rasterize_workspace_layout(arr, 1, ct.byref(o), None, 0)
    ents = (rast.WsEntry * n)()
    lib.rasterize_workspace_layout(arr, 1, ct.byref(o), ents, n)
    lay = {e.name.decode(): (e.offset, e.bytes) for e in ents}
    for key in ("records", "sorted_keys", "sorted_vals", "ranges", "t_final", "last", "partial"):
        off, nb = lay[key]
        assert off % 256 == 0 and off + nb <= size
    assert lay["records"][1] == 1000 * 8 * 4  # bilinear, 4 f32 features: 32-byte records
    assert lay["ranges"][1] == 7 * 4 * 8      # ceil(100/16) x ceil(60/16) tiles
    assert lay["t_final"][1] == 100 * 60 * 4
    # gaussian: 64-byte records (power-of-two stride), 16 copies per point by default
    og = _opts(lib, mode=1)
    n = lib.rasterize_workspace_layout(arr, 1, ct.byref(og), ents, len(ents))
    lay = {e.name.decode(): (e.offset, e.bytes) for e in ents}
    assert lay["records"][1] == 1000 * 16 * 4
    assert lay["sorted_keys"][1] == 16 * 1000 * 4
    # 8x8 tiles: ceil(100/8) x ceil(60/8) tile ranges
    o8 = _opts(lib, tile=8)
    n = lib.rasterize_workspace_layout(arr, 1, ct.byref(o8), ents, len(ents))
    lay = {e.name.decode(): (e.offset, e.bytes) for e in ents}
    assert lay["ranges"][1] == 13 * 8 * 8


def test_argument_validation_is_synchronous(lib):
    v = _fake_view()
    arr = (rast.View * 1)(v)
    o = _opts(lib)
    ws, big = ct.c_void_p(1 << 20), 1 << 40
    B = lib.rasterize_batch
    assert B(arr, 0, 1, ct.byref(o), ws, big, None) == rast.RAST_ERR_ARG
    assert B(arr, 17, 1, ct.byref(o), ws, big, None) == rast.RAST_ERR_ARG
    assert B(arr, 1, 0, ct.byref(o), ws, big, None) == rast.RAST_ERR_ARG
    assert B(arr, 1, 1, ct.byref(_opts(lib, tile=32)), ws, big, None) == rast.RAST_ERR_NOT_SUPPORTED
    for t, d, m in ((8, 512, 0), (16, 1024, 0), (16, 300, 0), (16, 512, 1), (8, 128, 1)):
        assert B(arr, 1, 1, ct.byref(_opts(lib, tile=t, blend_depth=d, mode=m)), ws, big, None) == \
            rast.RAST_ERR_NOT_SUPPORTED, (t, d, m)
    assert B(arr, 1, 1, ct.byref(_opts(lib, mode=7)), ws, big, None) == rast.RAST_ERR_ARG
    assert B(arr, 1, 1, ct.byref(_opts(lib, alpha_max=1.0)), ws, big, None) == rast.RAST_ERR_ARG
    assert B(arr, 1, 1, ct.byref(_opts(lib, flags=8)), ws, big, None) == rast.RAST_ERR_ARG  # unknown flag
    assert B(arr, 1, 1, ct.byref(o), None, big, None) == rast.RAST_ERR_ARG
    assert B(arr, 1, 1, ct.byref(o), ct.c_void_p((1 << 20) + 4), big, None) == rast.RAST_ERR_ARG
    assert B(arr, 1, 1, ct.byref(o), ws, 1024, None) == rast.RAST_ERR_CAPACITY
    bad = _fake_view(C=5)
    assert B((rast.View * 1)(bad), 1, 1, ct.byref(o), ws, big, None) == rast.RAST_ERR_NOT_SUPPORTED
    bad = _fake_view()
    bad.cam.near_z = 0.0
    assert B((rast.View * 1)(bad), 1, 1, ct.byref(o), ws, big, None) == rast.RAST_ERR_ARG
    bad = _fake_view()
    bad.out.feat = None
    assert B((rast.View * 1)(bad), 1, 1, ct.byref(o), ws, big, None) == rast.RAST_ERR_ARG
    bad = _fake_view()
    bad.grad.g_feat = None
    assert B((rast.View * 1)(bad), 1, 2, ct.byref(o), ws, big, None) == rast.RAST_ERR_ARG
    mixed = (rast.View * 2)(_fake_view(C=4), _fake_view(C=8))
    assert B(mixed, 2, 1, ct.byref(o), ws, big, None) == rast.RAST_ERR_ARG
    assert lib.rasterize_fwd(None, None, ct.byref(o), ws, big, None, None) == rast.RAST_ERR_ARG
    assert lib.rasterize_get_status(None, 0, None, None) == rast.RAST_ERR_ARG


def test_status_strings(lib):
    for s in range(6):
        assert lib.rasterize_status_string(s)
    assert b"sm_103a" in lib.rasterize_version()


def test_product_path_fails_loudly_without_library(tmp_path):
    import importlib
    mod = importlib.reload(rast)
    mod._lib = None
    with pytest.raises(RuntimeError, match="no CPU fallback"):
        mod.load_library(str(tmp_path / "missing.so"))
    mod._lib = None
