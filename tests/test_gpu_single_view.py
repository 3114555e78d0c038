"""The per-view entry points rasterize_fwd / rasterize_bwd of the C ABI: the
same images and gradients as rasterize_batch over that one view (bit for bit:
same kernels, same order) and as the oracle (Eq. 1; appendix, corrected
Eq. 2); and the per-stage timing counters (rasterize_profile_*)."""
import numpy as np
import pytest
import torch

import oracle
from paper_2508_19140_gb300 import rast, scenes

from gpu_util import Run, bf16_round

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


@pytest.fixture(scope="module", autouse=True)
def _need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2508_19140_gb300 import build
    build.build()
    oracle.build()


def _t(a, dtype=torch.float32):
    return None if a is None else torch.from_numpy(np.ascontiguousarray(a)).to(DEV, dtype)


def _single(v, mode="bilinear", bf16=False, **okw):
    """rasterize_fwd then rasterize_bwd on one workspace."""
    gauss = mode == "gaussian"
    xyz, op = _t(v.xyz), _t(v.opacity)
    feat = _t(v.feat, torch.bfloat16 if bf16 else torch.float32)
    scale = _t(v.scale) if gauss else None
    H, W, C = v.camera.height, v.camera.width, v.feat.shape[1]
    n = len(v.xyz)
    F = torch.full((H, W, C), float("nan"), device=DEV)
    A = torch.full((H, W), float("nan"), device=DEV)
    D = torch.full((H, W), float("nan"), device=DEV)
    pts = rast.make_points(xyz, op, feat, scale)
    cam = rast.make_camera(v.camera)
    opts = rast.make_opts(mode=mode, **okw)
    view = rast.View()
    view.pts, view.cam = pts, cam
    ws = torch.zeros(rast.rasterize_workspace_size([view], opts), dtype=torch.uint8, device=DEV)
    rast.rasterize_fwd(pts, cam, opts, ws, rast.make_images(F, A, D))
    gF, gA, gD = _t(v.g_feat), _t(v.g_alpha), _t(v.g_depth)
    d = dict(d_feat=torch.full((n, C), float("nan"), device=DEV),
             d_opacity=torch.full((n,), float("nan"), device=DEV),
             d_xyz=torch.full((n, 3), float("nan"), device=DEV) if gauss else None,
             d_scale=torch.full((n,), float("nan"), device=DEV) if gauss else None)
    rast.rasterize_bwd(pts, cam, opts, ws, rast.make_grads(gF, gA, gD, d["d_feat"], d["d_opacity"],
                                                           d["d_xyz"], d["d_scale"]))
    torch.cuda.synchronize()
    st, stats = rast.rasterize_get_status(ws)
    assert st == 0, stats
    img = (F.cpu().numpy(), A.cpu().numpy(), D.cpu().numpy())
    return img, {k: None if x is None else x.cpu().numpy() for k, x in d.items()}


def _bits(a):
    return np.asarray(a, np.float32).view(np.uint32)


CASES = [("bilinear", False, 16, 0, 4), ("bilinear", True, 16, 0, 8), ("bilinear", True, 8, 64, 8),
         ("bilinear", False, 8, 256, 3), ("gaussian", False, 16, 0, 4), ("gaussian", True, 8, 0, 2)]


@pytest.mark.parametrize("mode,bf16,tile,depth,c", CASES)
def test_single_view_calls_equal_batch_and_oracle(mode, bf16, tile, depth, c):
    g = mode == "gaussian"
    v = scenes.random_small_view(51 + c, 5000, 97, 66, c=c, gaussian=g, f=80.0 if g else None)
    img, d = _single(v, mode, bf16, tile=tile, blend_depth=depth)
    r = Run([v], mode=mode, bf16=bf16, backward=True, tile=tile, blend_depth=depth)
    for a, b in zip(img, r.image()):
        assert np.array_equal(_bits(a), _bits(b))
    rg = r.grads()
    for key in ("d_feat", "d_opacity") + (("d_xyz", "d_scale") if g else ()):
        assert np.array_equal(_bits(d[key]), _bits(rg[key])), key
    fv = bf16_round(v.feat) if bf16 else v.feat
    kw = dict(mode=mode, tile=16, pin32=True)
    ref = oracle.render(v.xyz, v.opacity, fv, v.camera, scale=v.scale if g else None, **kw)
    if not g:  # Gaussian images and gradients are covered pixel by pixel in the parity tests
        np.testing.assert_allclose(img[0], ref["F"], rtol=1e-5, atol=1e-7)
        np.testing.assert_allclose(img[1], ref["alpha"], rtol=1e-5, atol=1e-7)
        gr = oracle.backward(v.xyz, v.opacity, fv, v.camera, v.g_feat, v.g_alpha, v.g_depth, **kw)
        for key in ("d_feat", "d_opacity"):
            f = gr[key]
            assert np.linalg.norm(d[key] - f) <= 1e-5 * np.linalg.norm(f), key


def test_profile_counters():
    v = scenes.random_small_view(60, 8000, 120, 90, c=4)
    rast.rasterize_profile_enable(True)
    try:
        Run([v], backward=True)
        torch.cuda.synchronize()
        prof = rast.rasterize_profile_read()
    finally:
        rast.rasterize_profile_enable(False)
    for name in ("project", "depth_sort.sweep", "dup.write", "tile_sort.sweep", "ranges",
                 "blend_fwd", "blend_bwd", "reduce_grads"):
        launches, ms = prof[name]
        assert launches >= 1 and ms > 0.0, (name, prof[name])
    # disabled (which also clears): nothing more is recorded
    Run([v], backward=True)
    torch.cuda.synchronize()
    assert rast.rasterize_profile_read() == {}
