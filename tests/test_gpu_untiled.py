"""The untiled baseline (per-pixel lists, the arrangement Sec. 3.2 "Tiled
Rendering" replaces): its per-pixel fragment lists must equal the oracle's
lists at a tile edge of one pixel, bit for bit, and its images must be
bit-identical to the tiled forward (same per-pixel order, same FP32 ops)."""
import numpy as np
import pytest
import torch

import oracle
from paper_2508_19140_gb300 import rast, scenes

from gpu_util import Run
from test_gpu_parity import BILIN, case_view

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


@pytest.fixture(scope="module", autouse=True)
def _need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2508_19140_gb300 import build
    build.build()
    oracle.build()


def _untiled(v, bf16=False):
    xyz = torch.from_numpy(v.xyz).to(DEV)
    op = torch.from_numpy(v.opacity).to(DEV)
    feat = torch.from_numpy(v.feat).to(DEV, torch.bfloat16 if bf16 else torch.float32)
    H, W, C = v.camera.height, v.camera.width, v.feat.shape[1]
    F = torch.full((H, W, C), float("nan"), device=DEV)
    A = torch.full((H, W), float("nan"), device=DEV)
    D = torch.full((H, W), float("nan"), device=DEV)
    pts = rast.make_points(xyz, op, feat)
    cam = rast.make_camera(v.camera)
    opts = rast.make_opts()
    ws = torch.zeros(rast.rasterize_untiled_workspace_size(pts, cam, opts), dtype=torch.uint8, device=DEV)
    rast.rasterize_fwd_untiled(pts, cam, opts, ws, rast.make_images(F, A, D))
    torch.cuda.synchronize()
    st, stats = rast.rasterize_get_status(ws)
    assert st == 0, stats
    return F.cpu().numpy(), A.cpu().numpy(), D.cpu().numpy(), ws, stats


def _same(a, b):
    return np.array_equal(np.asarray(a, np.float32).view(np.uint32), np.asarray(b, np.float32).view(np.uint32))


@pytest.mark.parametrize("name", BILIN)
def test_untiled_equals_tiled_and_oracle_lists(name):
    v = case_view(name)
    F, A, D, ws, stats = _untiled(v)
    ref = Run([v])
    Ft, At, Dt = ref.image()
    assert _same(F, Ft) and _same(A, At) and _same(D, Dt)
    tiles, idx = oracle.tile_lists(v.xyz, v.camera, mode="bilinear", tile=1, pin32=True)
    assert int(stats["n_copies"]) == len(tiles)
    want = oracle.render(v.xyz, v.opacity, v.feat, v.camera, mode="bilinear", tile=1, pin32=True)
    assert int(stats["needed_records"]) == want["needed"]


def test_untiled_full_frame_bf16():
    v = scenes.make_scene(2).views[0]
    F, A, D, ws, stats = _untiled(v, bf16=True)
    ref = Run([v], bf16=True)
    Ft, At, Dt = ref.image()
    assert _same(F, Ft) and _same(A, At) and _same(D, Dt)
    assert 3.5 * len(v.xyz) < int(stats["n_copies"]) <= 4 * len(v.xyz)


def test_untiled_rejects_gaussian():
    v = case_view("gauss")
    xyz = torch.from_numpy(v.xyz).to(DEV)
    op = torch.from_numpy(v.opacity).to(DEV)
    feat = torch.from_numpy(v.feat).to(DEV)
    pts = rast.make_points(xyz, op, feat, torch.from_numpy(v.scale).to(DEV))
    cam = rast.make_camera(v.camera)
    L = rast.load_library()
    o = rast.make_opts(mode="gaussian")
    assert L.rasterize_untiled_workspace_size(rast.ct.byref(pts), rast.ct.byref(cam), rast.ct.byref(o)) == 0
