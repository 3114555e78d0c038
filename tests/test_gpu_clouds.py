"""Several point clouds into one image (the ring buffer of view-specific
clouds, Sec. 3.1): the result must equal one cloud holding the clouds
concatenated in order, bit for bit (images, transmittance, last positions,
sorted lists, gradients), and match the oracle on that concatenation."""
import numpy as np
import pytest
import torch

import oracle
from paper_2508_19140_gb300 import rast, scenes

from gpu_util import Run

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
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV, dtype)


def _clouds(sizes, W=120, H=90, c=4, gaussian=False, seed=70):
    views = [scenes.random_small_view(seed + k, n, W, H, c=c, gaussian=gaussian, f=90.0 if gaussian else None)
             for k, n in enumerate(sizes)]
    cam = views[0].camera
    g = views[0]
    return views, cam, g


def _concat(views, g):
    v = scenes.View(camera=views[0].camera,
                    xyz=np.concatenate([x.xyz for x in views]), opacity=np.concatenate([x.opacity for x in views]),
                    feat=np.concatenate([x.feat for x in views]),
                    scale=None if views[0].scale is None else np.concatenate([x.scale for x in views]),
                    g_feat=g.g_feat, g_alpha=g.g_alpha, g_depth=g.g_depth)
    return v


def _run_clouds(views, cam, g, mode, bf16, backward, tile=16, depth=0):
    opts = rast.make_opts(mode=mode, tile=tile, blend_depth=depth)
    H, W, C = cam.height, cam.width, views[0].feat.shape[1]
    keep = []
    pts, grads = [], []
    for v in views:
        xyz, op = _t(v.xyz), _t(v.opacity)
        feat = _t(v.feat, torch.bfloat16 if bf16 else torch.float32)
        sc = _t(v.scale) if mode == "gaussian" else None
        n = len(v.xyz)
        d = dict(d_feat=torch.full((n, C), float("nan"), device=DEV), d_op=torch.full((n,), float("nan"), device=DEV),
                 d_xyz=torch.full((n, 3), float("nan"), device=DEV) if mode == "gaussian" else None,
                 d_scale=torch.full((n,), float("nan"), device=DEV) if mode == "gaussian" else None)
        keep += [xyz, op, feat, sc, d]
        pts.append(rast.make_points(xyz, op, feat, sc))
        grads.append(d)
    F = torch.full((H, W, C), float("nan"), device=DEV)
    A = torch.full((H, W), float("nan"), device=DEV)
    D = torch.full((H, W), float("nan"), device=DEV)
    gF, gA, gD = _t(g.g_feat), _t(g.g_alpha), _t(g.g_depth)
    cgrads = [rast.make_grads(gF, gA, gD, d["d_feat"], d["d_op"], d["d_xyz"], d["d_scale"]) for d in grads]
    c = rast.make_camera(cam)
    ws = torch.zeros(rast.rasterize_clouds_workspace_size(pts, c, opts), dtype=torch.uint8, device=DEV)
    out = rast.make_images(F, A, D)
    rast.rasterize_clouds(pts, None, c, out, rast.PASS_FWD, opts, ws)
    if backward:
        rast.rasterize_clouds(pts, cgrads, c, out, rast.PASS_BWD, opts, ws)
    torch.cuda.synchronize()
    res = dict(F=F.cpu().numpy(), A=A.cpu().numpy(), D=D.cpu().numpy())
    for key in ("d_feat", "d_op", "d_xyz", "d_scale"):
        if grads[0][key] is not None:
            res[key] = np.concatenate([d[key].cpu().numpy() for d in grads])
    return res


def _same(a, b):
    return np.array_equal(np.asarray(a, np.float32).view(np.uint32), np.asarray(b, np.float32).view(np.uint32))


@pytest.mark.parametrize("mode,bf16,tile,depth", [("bilinear", False, 16, 0), ("bilinear", True, 8, 128),
                                                  ("gaussian", False, 16, 0), ("gaussian", True, 8, 0)])
def test_clouds_equal_concatenation(mode, bf16, tile, depth):
    g_ = mode == "gaussian"
    views, cam, g = _clouds([3000, 0, 5000, 1200], gaussian=g_, c=8 if bf16 else 4)
    got = _run_clouds(views, cam, g, mode, bf16, True, tile, depth)
    cat = _concat(views, g)
    ref = Run([cat], mode=mode, bf16=bf16, backward=True, tile=tile, blend_depth=depth)
    F, A, D = ref.image()
    assert _same(got["F"], F) and _same(got["A"], A) and _same(got["D"], D)
    rg = ref.grads()
    assert _same(got["d_feat"], rg["d_feat"]) and _same(got["d_op"], rg["d_opacity"])
    if g_:
        assert _same(got["d_xyz"], rg["d_xyz"]) and _same(got["d_scale"], rg["d_scale"])


def test_clouds_match_oracle():
    views, cam, g = _clouds([4000, 2500, 6000, 3500])
    got = _run_clouds(views, cam, g, "bilinear", False, True)
    cat = _concat(views, g)
    kw = dict(mode="bilinear", tile=16, pin32=True)
    ref = oracle.render(cat.xyz, cat.opacity, cat.feat, cam, **kw)
    np.testing.assert_allclose(got["F"], ref["F"], rtol=1e-5, atol=1e-7)
    np.testing.assert_allclose(got["A"], ref["alpha"], rtol=1e-5, atol=1e-7)
    gr = oracle.backward(cat.xyz, cat.opacity, cat.feat, cam, cat.g_feat, cat.g_alpha, cat.g_depth, **kw)
    for a, b in ((got["d_feat"], gr["d_feat"]), (got["d_op"], gr["d_opacity"])):
        assert np.linalg.norm(a - b) / np.linalg.norm(b) < 1e-5


def test_clouds_argument_errors():
    views, cam, g = _clouds([100, 100])
    L = rast.load_library()
    c = rast.make_camera(cam)
    o = rast.make_opts()
    xyz, op, feat = _t(views[0].xyz), _t(views[0].opacity), _t(views[0].feat)
    p = rast.make_points(xyz, op, feat)
    arr = (rast.Points * 17)(*([p] * 17))
    assert L.rasterize_clouds_workspace_size(arr, 0, rast.ct.byref(c), rast.ct.byref(o)) == 0
    assert L.rasterize_clouds_workspace_size(arr, 17, rast.ct.byref(c), rast.ct.byref(o)) == 0
    feat2 = _t(np.zeros((100, 3)))
    q = rast.make_points(xyz, op, feat2)
    arr2 = (rast.Points * 2)(p, q)
    assert L.rasterize_clouds_workspace_size(arr2, 2, rast.ct.byref(c), rast.ct.byref(o)) == 0
    out = rast.make_images(torch.zeros((cam.height, cam.width, 4), device=DEV))
    ws = torch.zeros(1 << 20, dtype=torch.uint8, device=DEV)
    st = L.rasterize_clouds(arr, None, 2, rast.ct.byref(c), rast.ct.byref(out), rast.PASS_BWD, rast.ct.byref(o),
                            rast._ptr(ws), 1 << 20, None)
    assert st == rast.RAST_ERR_ARG
