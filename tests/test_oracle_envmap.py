"""CPU pins of the background-model oracle (Sec. 3.2 "Faster Background Model
Evaluation"): closed forms, linear-reproduction of the bilinear lookup that
pins the direction -> texel mapping, wrap-around, and finite differences."""
import math

import numpy as np
import pytest

import oracle
from paper_2508_19140_gb300 import scenes


@pytest.fixture(scope="module", autouse=True)
def _build():
    oracle.build()


def _cam(W=40, H=30, f=25.0, yaw=0.0):
    c = scenes.identity_camera(W, H, f)
    if yaw:
        a = math.radians(yaw)
        c.R = np.array([[math.cos(a), 0, -math.sin(a)], [0, 1, 0], [math.sin(a), 0, math.cos(a)]], np.float32)
    return c


def _inputs(cam, C=4, seed=0):
    rng = np.random.default_rng(seed)
    F = rng.uniform(0, 1, (cam.height, cam.width, C))
    alpha = rng.uniform(0, 1, (cam.height, cam.width))
    g = rng.standard_normal((cam.height, cam.width, C))
    return F, alpha, g


def _world_dirs(cam):
    d = oracle.env_dirs(cam)
    return d @ np.asarray(cam.R, np.float64)  # rows: R^T d


def test_constant_map_closed_form():
    cam = _cam()
    F, alpha, g = _inputs(cam)
    env = np.full((16, 32, 4), 0.3)
    env[..., 1] = 0.7
    out, bg = oracle.env_composite(env, cam, F, alpha)
    np.testing.assert_allclose(bg, np.broadcast_to([0.3, 0.7, 0.3, 0.3], bg.shape), rtol=0, atol=1e-15)
    np.testing.assert_allclose(out, F + (1 - alpha)[..., None] * bg, rtol=0, atol=1e-15)
    d_alpha, d_map = oracle.env_backward(env, cam, alpha, g)
    np.testing.assert_allclose(d_alpha, -(g * bg).sum(-1), rtol=1e-14, atol=1e-14)
    # bilinear weights sum to one: the map gradient sums to sum_p (1 - alpha_p) g_p
    np.testing.assert_allclose(d_map.sum((0, 1)), ((1 - alpha)[..., None] * g).sum((0, 1)), rtol=1e-12)


def test_linear_map_pins_the_texel_mapping():
    """Bilinear interpolation reproduces a map linear in the column (row) index,
    so f_bg equals the continuous texel coordinate X (Y) of each direction."""
    cam = _cam(W=64, H=48, f=40.0, yaw=30.0)
    Hb, Wb = 64, 128
    cols = np.broadcast_to(np.arange(Wb, dtype=np.float64)[None, :, None], (Hb, Wb, 1))
    rows = np.broadcast_to(np.arange(Hb, dtype=np.float64)[:, None, None], (Hb, Wb, 1))
    dw = _world_dirs(cam)
    X = (np.arctan2(dw[..., 0], dw[..., 2]) / (2 * np.pi) + 0.5) * Wb - 0.5
    Y = np.arccos(np.clip(dw[..., 1], -1, 1)) / np.pi * Hb - 0.5
    F = np.zeros((cam.height, cam.width, 1))
    alpha = np.zeros((cam.height, cam.width))
    _, bgx = oracle.env_composite(cols, cam, F, alpha)
    _, bgy = oracle.env_composite(rows, cam, F, alpha)
    inner = (X > 0) & (X < Wb - 1)          # away from the wrap seam
    assert inner.mean() > 0.9
    np.testing.assert_allclose(bgx[..., 0][inner], X[inner], rtol=0, atol=1e-9)
    inner_y = (Y > 0) & (Y < Hb - 1)        # away from the clamped poles
    np.testing.assert_allclose(bgy[..., 0][inner_y], Y[inner_y], rtol=0, atol=1e-9)


def test_centre_pixel_looks_down_plus_z():
    cam = _cam(W=2, H=2, f=1.0)  # pixel centres at (+-1/2, +-1/2) / f about the axis
    cam.cx = cam.cy = 0.5        # pixel (0, 0) centre on the optical axis
    Hb, Wb = 8, 16
    env = np.arange(Hb * Wb, dtype=np.float64).reshape(Hb, Wb, 1)
    _, bg = oracle.env_composite(env, cam, np.zeros((2, 2, 1)), np.zeros((2, 2)))
    # d = +z: X = Wb/2 - 1/2, Y = Hb/2 - 1/2 -> mean of the four central texels
    r0, c0 = Hb // 2 - 1, Wb // 2 - 1
    want = env[r0:r0 + 2, c0:c0 + 2, 0].mean()
    assert abs(bg[0, 0, 0] - want) < 1e-12


def test_wrap_around_seam():
    """Directions just either side of lambda = +-pi blend column W_b - 1 with
    column 0 (periodic longitude)."""
    cam = _cam(W=3, H=1, f=1000.0, yaw=180.0)  # looking down -z: lambda ~ +-pi
    Hb, Wb = 4, 8
    env = np.zeros((Hb, Wb, 1))
    env[:, 0] = 1.0
    env[:, Wb - 1] = 3.0
    _, bg = oracle.env_composite(env, cam, np.zeros((1, 3, 1)), np.zeros((1, 3)))
    # every value lies between the two seam columns, both sides are used
    assert np.all(bg > 0.999) and np.all(bg < 3.001)
    assert bg.max() - bg.min() > 1e-4
    # and each one is the periodic interpolation at its texel coordinate X
    dw = _world_dirs(cam)
    X = (np.arctan2(dw[..., 0], dw[..., 2]) / (2 * np.pi) + 0.5) * Wb - 0.5
    c0 = np.floor(X)
    a = X - c0
    col = env[0, :, 0]
    want = (1 - a) * col[c0.astype(int) % Wb] + a * col[(c0.astype(int) + 1) % Wb]
    assert np.any(np.abs(X - (Wb - 1)) < 1) or np.any(X < 0)  # the seam is crossed
    np.testing.assert_allclose(bg[..., 0], want, rtol=0, atol=1e-9)


def test_cached_directions_equal_on_the_fly():
    cam = _cam(yaw=70.0)
    F, alpha, g = _inputs(cam)
    env = scenes.env_map(height=32, width=64)
    d = oracle.env_dirs(cam)
    a, _ = oracle.env_composite(env, cam, F, alpha)
    b, _ = oracle.env_composite(env, cam, F, alpha, dirs=d)
    np.testing.assert_allclose(a, b, rtol=0, atol=1e-14)


def test_adjoint_finite_differences():
    cam = _cam(W=12, H=9, f=8.0, yaw=20.0)
    rng = np.random.default_rng(3)
    F, alpha, g = _inputs(cam, C=2, seed=3)
    env = rng.uniform(0, 1, (6, 12, 2))
    loss = lambda e, a: float((oracle.env_composite(e, cam, F, a)[0] * g).sum())
    d_alpha, d_map = oracle.env_backward(env, cam, alpha, g)
    h = 1e-6
    for _ in range(12):
        i, j, c = rng.integers(6), rng.integers(12), rng.integers(2)
        e1, e2 = env.copy(), env.copy()
        e1[i, j, c] += h
        e2[i, j, c] -= h
        fd = (loss(e1, alpha) - loss(e2, alpha)) / (2 * h)
        assert abs(fd - d_map[i, j, c]) <= 1e-7 * max(1.0, abs(fd))
    for _ in range(12):
        y, x = rng.integers(9), rng.integers(12)
        a1, a2 = alpha.copy(), alpha.copy()
        a1[y, x] += h
        a2[y, x] -= h
        fd = (loss(env, a1) - loss(env, a2)) / (2 * h)
        assert abs(fd - d_alpha[y, x]) <= 1e-7 * max(1.0, abs(fd))
