"""GPU parity of the distilled background model (Sec. 3.2 "Faster Background
Model Evaluation") against the FP64 oracle.

Bars. Directions: FP32 rounding (1e-6 absolute). Composite: the kernel maps a
direction to texel coordinates in FP32 (atan2f / acosf and a multiply by the
map width), which moves the coordinate by up to ~3e-4 texel at 2048 columns;
on the smooth (sky-like) map that changes the interpolated value by far less
than 1e-5 relative, the image bar used everywhere else. dL/dalpha follows the
same bound. The map gradient sums w (1 - alpha) g over pixels with weights
that move by the same ~3e-4 texel: normwise 1e-3 of the gradient, and exact
integer (fixed-point) accumulation makes reruns bit-identical."""

import numpy as np
import pytest
import torch

import oracle
from paper_2508_19140_gb300 import rast, scenes

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


@pytest.fixture(scope="module", autouse=True)
def _need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2508_19140_gb300 import build
    build.build()
    oracle.build()


def _cam(W, H, yaw=0.0, pitch=0.0, f=None):
    c = scenes.orbit_camera(W, H, 5.0, yaw, pitch, f=f)
    return c


def _t(a):
    return torch.from_numpy(np.ascontiguousarray(a, np.float32)).to(DEV)


def _run(cam, env_np, F, alpha, g, cached):
    env = _t(env_np)
    e = rast.make_envmap(env)
    c = rast.make_camera(cam)
    H, W, C = F.shape
    dirs = None
    if cached:
        dirs = torch.empty((H, W, 3), device=DEV)
        rast.rasterize_view_dirs(c, dirs)
    out = torch.empty((H, W, C), device=DEV)
    rast.rasterize_bg_composite(c, e, dirs, _t(F), _t(alpha), out)
    ga = _t(np.zeros((H, W)))
    dm = torch.empty_like(env)
    scratch = torch.empty(rast.rasterize_bg_scratch_size(e), dtype=torch.uint8, device=DEV)
    rast.rasterize_bg_composite_bwd(c, e, dirs, _t(alpha), _t(g), ga, dm, scratch)
    torch.cuda.synchronize()
    return out.cpu().numpy(), ga.cpu().numpy(), dm.cpu().numpy(), (None if dirs is None else dirs.cpu().numpy())


def _inputs(H, W, C, seed):
    rng = np.random.default_rng(seed)
    F = rng.uniform(0, 1, (H, W, C)).astype(np.float32)
    alpha = rng.uniform(0, 1, (H, W)).astype(np.float32)
    g = rng.standard_normal((H, W, C)).astype(np.float32)
    return F, alpha, g


VIEWS = [(0.0, 0.0), (37.0, 12.0), (180.0, 0.0), (90.0, -75.0), (-120.0, 80.0)]


@pytest.mark.parametrize("yaw,pitch", VIEWS)
@pytest.mark.parametrize("cached", [True, False])
def test_composite_and_adjoint(yaw, pitch, cached):
    H, W, C = 96, 160, 4
    cam = _cam(W, H, yaw, pitch)
    env = scenes.env_map(height=256, width=512, c=C)
    F, alpha, g = _inputs(H, W, C, seed=int(yaw) % 97)
    out, ga, dm, dirs = _run(cam, env, F, alpha, g, cached)
    if cached:
        np.testing.assert_allclose(dirs, oracle.env_dirs(cam), rtol=0, atol=1e-6)
    ref_out, _ = oracle.env_composite(env, cam, F, alpha)
    np.testing.assert_allclose(out, ref_out, rtol=1e-5, atol=1e-6)
    d_alpha, d_map = oracle.env_backward(env, cam, alpha, g)
    np.testing.assert_allclose(ga, d_alpha, rtol=1e-5, atol=1e-5)
    err = np.linalg.norm(dm - d_map) / np.linalg.norm(d_map)
    assert err < 1e-3, err
    # untouched texels stay exactly zero
    assert np.all(dm[d_map == 0] == 0)


def test_channels_8_and_noise_map_bound():
    """Noise map (worst case for the coordinate error): |delta| <= |dX| * max
    texel step with |dX| <= 5e-4 texel at 512 columns."""
    H, W, C = 64, 96, 8
    cam = _cam(W, H, 20.0, 5.0)
    env = scenes.env_map(height=128, width=512, c=C, kind="noise")
    F, alpha, g = _inputs(H, W, C, seed=5)
    out, ga, dm, _ = _run(cam, env, F, alpha, g, True)
    ref_out, _ = oracle.env_composite(env, cam, F, alpha)
    np.testing.assert_allclose(out, ref_out, rtol=0, atol=5e-4 * 2 + 1e-6)
    d_alpha, d_map = oracle.env_backward(env, cam, alpha, g)
    assert np.linalg.norm(dm - d_map) / np.linalg.norm(d_map) < 5e-3


def test_bit_identical_reruns():
    H, W, C = 120, 200, 4
    cam = _cam(W, H, 60.0, 10.0)
    env = scenes.env_map(height=128, width=256, c=C)
    F, alpha, g = _inputs(H, W, C, seed=9)
    a = _run(cam, env, F, alpha, g, True)
    b = _run(cam, env, F, alpha, g, True)
    for x, y in zip(a[:3], b[:3]):
        assert np.array_equal(x.view(np.uint32), y.view(np.uint32))


def test_full_size_paper_map():
    """1280x832 frame, the paper's 1024 x 2048 x 4 map."""
    H, W, C = 832, 1280, 4
    cam = scenes.make_scene(2).views[0].camera
    env = scenes.env_map(c=C)
    F, alpha, g = _inputs(H, W, C, seed=11)
    out, ga, dm, _ = _run(cam, env, F, alpha, g, True)
    ref_out, _ = oracle.env_composite(env, cam, F, alpha)
    np.testing.assert_allclose(out, ref_out, rtol=1e-5, atol=1e-6)
    d_alpha, d_map = oracle.env_backward(env, cam, alpha, g)
    np.testing.assert_allclose(ga, d_alpha, rtol=1e-5, atol=1e-5)
    assert np.linalg.norm(dm - d_map) / np.linalg.norm(d_map) < 1e-3


def test_argument_errors():
    env = _t(scenes.env_map(height=8, width=16, c=4))
    e = rast.make_envmap(env)
    c = rast.make_camera(_cam(16, 8))
    F = torch.zeros((8, 16, 4), device=DEV)
    A = torch.zeros((8, 16), device=DEV)
    L = rast.load_library()
    assert L.rasterize_bg_composite(None, None, None, None, None, None, None) == rast.RAST_ERR_ARG
    small = torch.empty(16, dtype=torch.uint8, device=DEV)
    st = L.rasterize_bg_composite_bwd(rast.ct.byref(c), rast.ct.byref(e), None, rast._ptr(A), rast._ptr(F),
                                      None, rast._ptr(env), rast._ptr(small), 16, None)
    assert st == rast.RAST_ERR_CAPACITY
    bad = rast.make_envmap(env)
    bad.channels = 5
    assert L.rasterize_bg_scratch_size(rast.ct.byref(bad)) == 0
