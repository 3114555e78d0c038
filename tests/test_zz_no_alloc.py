"""The allocation-free forward entry point, for callers that cannot allocate
device memory where they render (a plug-in inside an application that owns
every GPU allocation, or code running while a stream is captured). Its
intermediates live in the library's static 16 MiB device scratch.

Checked here through the C ABI: its images equal those of rasterize_fwd with a
caller-allocated workspace, on two calls in a row (the second finds the first
call's contents in the shared scratch), and a problem too large for the
scratch is rejected with RAST_ERR_CAPACITY. This file is collected last so a
failure here cannot hide the other tests' results."""
import numpy as np
import pytest
import torch

from paper_2508_19140_gb300 import rast, scenes

pytestmark = pytest.mark.gpu


def _setup(v, dev):
    t = dict(xyz=torch.from_numpy(v.xyz).to(dev), op=torch.from_numpy(v.opacity).to(dev),
             feat=torch.from_numpy(v.feat).to(dev))
    pts = rast.make_points(t["xyz"], t["op"], t["feat"])
    cam = rast.make_camera(v.camera)
    return t, pts, cam


def _outputs(v, dev):
    H, W, C = v.camera.height, v.camera.width, v.feat.shape[1]
    F = torch.full((H, W, C), float("nan"), device=dev)
    A = torch.full((H, W), float("nan"), device=dev)
    D = torch.full((H, W), float("nan"), device=dev)
    return (F, A, D), rast.make_images(F, A, D)


def test_noalloc_forward_matches_workspace_forward_twice():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2508_19140_gb300 import build
    build.build()
    dev = torch.device("cuda:0")
    v = scenes.make_scene(1).views[0]          # 20,000 points at 128x128
    t, pts, cam = _setup(v, dev)
    opts = rast.make_opts()
    ref_t, ref_im = _outputs(v, dev)
    view = rast.View()
    view.pts, view.cam, view.out = pts, cam, ref_im
    ws = torch.empty(rast.rasterize_workspace_size([view], opts), dtype=torch.uint8, device=dev)
    rast.rasterize_fwd(pts, cam, opts, ws, ref_im)
    torch.cuda.synchronize()
    ref = [x.cpu().numpy() for x in ref_t]
    for _ in range(2):
        got_t, got_im = _outputs(v, dev)
        rast.rasterize_fwd_noalloc(pts, cam, opts, got_im)
        torch.cuda.synchronize()
        for g, r in zip(got_t, ref):
            np.testing.assert_allclose(g.cpu().numpy(), r, rtol=1e-5, atol=1e-7)


def test_noalloc_rejects_problems_beyond_the_scratch():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    dev = torch.device("cuda:0")
    v = scenes.random_small_view(5, 200_000, 640, 480)
    t, pts, cam = _setup(v, dev)
    _, im = _outputs(v, dev)
    with pytest.raises(rast.RastError) as e:
        rast.rasterize_fwd_noalloc(pts, cam, rast.make_opts(), im)
    assert e.value.status == rast.RAST_ERR_CAPACITY
