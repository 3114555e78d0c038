"""The allocation-free forward entry point, for callers that cannot allocate
device memory where they render: a plug-in inside an application that owns
every GPU allocation (its memory budget is fixed and it hands out no more),
or code that runs while a stream is being captured into a CUDA graph, where
an allocation is not allowed. Its intermediates live in the library's static
16 MiB device array.

Checked here through the C ABI:
  - its images equal, bit for bit, those of rasterize_fwd with a
    caller-allocated workspace, on two calls in a row of the same problem with
    a different problem (more points, more tiles, Gaussian footprints) run on
    the shared array in between, so the second call finds stale contents of
    another shape there;
  - a Gaussian view with BF16 features gives the same bits as the workspace
    path too;
  - errors the GPU raises during the pass (here: more copies than
    max_copies = 1 allows) are read back with rasterize_noalloc_get_status;
  - a problem too large for the array is rejected with RAST_ERR_CAPACITY.
This file is collected last so a failure here cannot hide the other tests'
results."""
import numpy as np
import pytest
import torch

from paper_2508_19140_gb300 import rast, scenes

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2508_19140_gb300 import build
    build.build()


def _setup(v, dev, bf16=False, gauss=False):
    t = dict(xyz=torch.from_numpy(v.xyz).to(dev), op=torch.from_numpy(v.opacity).to(dev),
             feat=torch.from_numpy(v.feat).to(dev, torch.bfloat16 if bf16 else torch.float32))
    t["scale"] = torch.from_numpy(v.scale).to(dev) if gauss and v.scale is not None else None
    pts = rast.make_points(t["xyz"], t["op"], t["feat"], t["scale"])
    cam = rast.make_camera(v.camera)
    return t, pts, cam


def _outputs(v, dev):
    H, W, C = v.camera.height, v.camera.width, v.feat.shape[1]
    F = torch.full((H, W, C), float("nan"), device=dev)
    A = torch.full((H, W), float("nan"), device=dev)
    D = torch.full((H, W), float("nan"), device=dev)
    return (F, A, D), rast.make_images(F, A, D)


def _workspace_forward(pts, cam, opts, v, dev):
    ref_t, ref_im = _outputs(v, dev)
    view = rast.View()
    view.pts, view.cam, view.out = pts, cam, ref_im
    ws = torch.full((rast.rasterize_workspace_size([view], opts),), 0xFF, dtype=torch.uint8, device=dev)
    rast.rasterize_fwd(pts, cam, opts, ws, ref_im)
    torch.cuda.synchronize()
    return [x.cpu().numpy() for x in ref_t]


def _same_bits(a, b):
    return np.array_equal(np.asarray(a).view(np.uint32), np.asarray(b).view(np.uint32))


def test_noalloc_forward_matches_workspace_forward_twice():
    dev = torch.device("cuda:0")
    v = scenes.make_scene(1).views[0]          # 20,000 points at 128x128
    t, pts, cam = _setup(v, dev)
    opts = rast.make_opts()
    ref = _workspace_forward(pts, cam, opts, v, dev)
    # another problem of another shape for the shared array in between
    w = scenes.random_small_view(41, 40000, 200, 150, c=4, gaussian=True, f=160.0)
    tw, pw, cw = _setup(w, dev, gauss=True)
    ow = rast.make_opts(mode="gaussian", max_copies=4)  # 3-sigma boxes of at most 15 px: <= 2x2 tiles
    for k in range(2):
        got_t, got_im = _outputs(v, dev)
        rast.rasterize_fwd_noalloc(pts, cam, opts, got_im)
        st, stats = rast.rasterize_noalloc_get_status()
        assert st == rast.RAST_OK, stats
        assert stats["n_points"] == len(v.xyz)
        for g, r in zip(got_t, ref):
            assert _same_bits(g.cpu().numpy(), r)
        if k == 0:
            _, im_w = _outputs(w, dev)
            rast.rasterize_fwd_noalloc(pw, cw, ow, im_w)
            st, _ = rast.rasterize_noalloc_get_status()
            assert st == rast.RAST_OK


def test_noalloc_gaussian_bf16_matches_workspace_forward():
    dev = torch.device("cuda:0")
    v = scenes.random_small_view(42, 30000, 160, 120, c=4, gaussian=True, f=140.0)
    t, pts, cam = _setup(v, dev, bf16=True, gauss=True)
    opts = rast.make_opts(mode="gaussian", max_copies=4)  # 3-sigma boxes of at most 13 px: <= 2x2 tiles
    ref = _workspace_forward(pts, cam, opts, v, dev)
    got_t, got_im = _outputs(v, dev)
    rast.rasterize_fwd_noalloc(pts, cam, opts, got_im)
    assert rast.rasterize_noalloc_get_status()[0] == rast.RAST_OK
    for g, r in zip(got_t, ref):
        assert _same_bits(g.cpu().numpy(), r)


def test_noalloc_reports_device_side_capacity_overflow():
    dev = torch.device("cuda:0")
    v = scenes.random_small_view(43, 4000, 90, 70, c=4, gaussian=True, f=80.0)
    t, pts, cam = _setup(v, dev, gauss=True)
    _, im = _outputs(v, dev)
    rast.rasterize_fwd_noalloc(pts, cam, rast.make_opts(mode="gaussian", max_copies=1), im)
    st, stats = rast.rasterize_noalloc_get_status()
    assert st == rast.RAST_ERR_CAPACITY
    assert stats["n_copies"] > stats["copy_capacity"]
    # the next call clears the error word
    _, im = _outputs(v, dev)
    rast.rasterize_fwd_noalloc(pts, cam, rast.make_opts(mode="gaussian"), im)
    assert rast.rasterize_noalloc_get_status()[0] == rast.RAST_OK


def test_noalloc_rejects_problems_beyond_the_scratch():
    dev = torch.device("cuda:0")
    v = scenes.random_small_view(5, 200_000, 640, 480)
    t, pts, cam = _setup(v, dev)
    _, im = _outputs(v, dev)
    with pytest.raises(rast.RastError) as e:
        rast.rasterize_fwd_noalloc(pts, cam, rast.make_opts(), im)
    assert e.value.status == rast.RAST_ERR_CAPACITY
