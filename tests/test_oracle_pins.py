"""Pins for the CPU oracle: it is checked here against things other than itself.

* closed forms the paper fixes: bilinear weights of one point sum to one
  (Sec. 3.2, small Gaussians, first paragraph), so a lone point deposits
  exactly its opacity; Eq. 1 for two and for K stacked fragments; an on-axis
  Gaussian reduces to a radially symmetric 2D Gaussian of variance
  s^2 f^2 / z^2 + 0.16 truncated at 3 sigma (same paragraph);
* the paper's printed constants (tests/golden/paper_constants.json): 1.27
  tiles per 2x2 splat at 8x8 tiles and the sort cost model (Sec. 3.2,
  "Tiled Rendering");
* invariants: alpha in [0, 1], T never below t_min, lists sorted;
* an independent NumPy brute force on tiny inputs (tent-function weights,
  explicit matrix algebra for the 2D covariance, the O(K^2) product form of
  Eq. 1 instead of a running transmittance);
* FP64 central finite differences for the adjoint (appendix, Eq. 2), and the
  alpha = 0 case of Eq. 2 with the background sign the chain rule gives.
"""
import json
import math
import os

import numpy as np
import pytest

from paper_2508_19140_gb300 import scenes

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_constants.json")
DIL32 = float(np.float32(0.16))  # the dilation variance is an FP32 parameter


def cam_at(width, height, f, cx=None, cy=None):
    c = scenes.identity_camera(width, height, f)
    if cx is not None:
        c.cx = cx
    if cy is not None:
        c.cy = cy
    return c


def point_at_pixel(cam, u, v, z):
    """World point (identity camera) that projects to screen (u, v) at depth z."""
    return [(u - cam.cx) * z / cam.fx, (v - cam.cy) * z / cam.fy, z]


# ----------------------------------------------------------------------------- closed forms

@pytest.mark.parametrize("pin32", [True, False])
def test_single_point_deposits_its_opacity(oracle_lib, pin32):
    rng = np.random.default_rng(0)
    cam = cam_at(32, 24, 30.0)
    for _ in range(20):
        u, v = rng.uniform(3, 28), rng.uniform(3, 20)
        o = rng.uniform(0.05, 0.95)
        f = rng.uniform(0, 1, (1, 3))
        xyz = np.array([point_at_pixel(cam, u, v, 2.5)])
        r = oracle_lib.render(xyz, np.array([o]), f, cam, pin32=pin32)
        # weights sum to one -> total alpha = o, total feature = o f
        assert abs(r["alpha"].sum() - o) < 1e-12
        assert np.allclose(r["F"].sum(axis=(0, 1)), o * f[0], atol=1e-12)
        assert abs(r["depth"].sum() - o * 2.5) < 1e-5
        assert (r["n_cover"] > 0).sum() <= 4


def test_single_point_at_border_loses_weight(oracle_lib):
    cam = cam_at(16, 16, 16.0)
    xyz = np.array([point_at_pixel(cam, 0.25, 8.3, 2.0)])  # left half outside the image
    r = oracle_lib.render(xyz, np.array([0.8]), np.ones((1, 1)), cam)
    assert 0 < r["alpha"].sum() < 0.8
    # 1 - a of the x weight falls off-screen: a = (0.25 - 0.5) - floor(-0.25) = 0.75
    assert abs(r["alpha"].sum() - 0.8 * 0.75) < 1e-6


@pytest.mark.parametrize("pin32", [True, False])
def test_two_stacked_points(oracle_lib, pin32):
    cam = cam_at(16, 16, 16.0)
    u, v = 7.3, 9.6
    xyz = np.array([point_at_pixel(cam, u, v, 3.0), point_at_pixel(cam, u, v, 2.0)])
    o = np.array([0.7, 0.4])
    f = np.array([[1.0, 0.0], [0.0, 1.0]])
    r = oracle_lib.render(xyz, o, f, cam, pin32=pin32)
    a, b = (u - 0.5) - math.floor(u - 0.5), (v - 0.5) - math.floor(v - 0.5)
    i0, j0 = math.floor(u - 0.5), math.floor(v - 0.5)
    tol = 4e-6 if pin32 else 1e-12  # pin32 rounds u, v to FP32 (ulp(8) ~ 1e-6 px)
    for (px, py, w) in [(i0, j0, (1 - a) * (1 - b)), (i0 + 1, j0, a * (1 - b)),
                        (i0, j0 + 1, (1 - a) * b), (i0 + 1, j0 + 1, a * b)]:
        a1, a2 = o[1] * w, o[0] * w  # point 1 is nearer (z = 2)
        assert abs(r["alpha"][py, px] - (a1 + (1 - a1) * a2)) < tol
        assert abs(r["F"][py, px, 1] - a1) < tol
        assert abs(r["F"][py, px, 0] - (1 - a1) * a2) < tol


@pytest.mark.parametrize("pin32", [True, False])
def test_k_equal_fragments_and_termination(oracle_lib, pin32):
    cam = cam_at(8, 8, 8.0)
    K = 20
    xyz = np.array([point_at_pixel(cam, 3.5, 4.5, 2.0)] * K)  # exactly on pixel (3, 4)
    o = np.full(K, 0.5)
    r = oracle_lib.render(xyz, o, np.ones((K, 1)), cam, pin32=pin32)
    # (1 - 1/2)^k < 1e-4 first at k = 14, so 13 fragments blend
    assert r["n_cover"][4, 3] == K
    assert r["n_blend"][4, 3] == 13
    assert abs(r["alpha"][4, 3] - (1 - 0.5 ** 13)) < 1e-12
    assert r["t_final"][4, 3] >= 1e-4
    assert r["stop_pos"][4, 3] == 14
    # the three zero-weight neighbours of the 2x2 box are listed but blend nothing
    assert r["n_cover"][4, 4] == 13 or r["n_cover"][4, 4] == K
    assert r["alpha"][4, 4] == 0.0


@pytest.mark.parametrize("cov", ["ewa", "iso"])
def test_on_axis_gaussian_closed_form(oracle_lib, cov):
    f, z, s, o = 100.0, 2.0, 0.03, 0.6
    cam = cam_at(64, 64, f, cx=32.5, cy=32.5)  # optical axis through the centre of pixel 32
    xyz = np.array([[0.0, 0.0, z]])
    r = oracle_lib.render(xyz, np.array([o]), np.ones((1, 1)), cam, scale=np.array([s]),
                          mode="gaussian", gauss_cov=cov, pin32=False)
    sig2 = (s * f / z) ** 2 + DIL32
    rad = math.ceil(3 * math.sqrt(sig2))
    for py in range(64):
        for px in range(64):
            dx, dy = px - 32, py - 32
            m = (dx * dx + dy * dy) / sig2
            inside = m <= 9 and abs(dx) <= rad and abs(dy) <= rad
            want = o * math.exp(-0.5 * m) if inside else 0.0
            assert abs(r["alpha"][py, px] - want) < 1e-12, (px, py)


def test_default_scale_is_five_pixels_at_near_plane(oracle_lib):
    f = 200.0
    cam = cam_at(64, 64, f, cx=32.5, cy=32.5)
    z = float(np.float32(cam.near)) * (1 + 1e-9)  # the near plane is an FP32 parameter
    p = oracle_lib.project(np.array([[0.0, 0.0, z]]), cam, mode="gaussian", pin32=False)
    sig2 = p["cov"][0, 0] - DIL32
    assert abs(math.sqrt(sig2) - 5.0) < 1e-6
    assert p["vis"][0] == 1


# ----------------------------------------------------------------------------- paper constants

def test_copies_per_point_match_paper(oracle_lib):
    gold = json.load(open(GOLDEN))
    rng = np.random.default_rng(5)
    n, W, H = 200_000, 512, 512
    cam = cam_at(W, H, 400.0)
    # u - 1/2 spans 14 whole periods of 32 px, so the anchor is uniform modulo every T
    u = rng.uniform(32, W - 32, n)
    v = rng.uniform(32, H - 32, n)
    z = rng.uniform(2, 4, n)
    xyz = np.stack([(u - cam.cx) * z / cam.fx, (v - cam.cy) * z / cam.fy, z], 1)
    for T in (8, 16, 32):
        tiles, _ = oracle_lib.tile_lists(xyz, cam, tile=T)
        mean = len(tiles) / n
        p = 1.0 / T
        sd = math.sqrt(((1 + 3 * p) ** 2 - (1 + p) ** 4) / n)
        assert abs(mean - (1 + p) ** 2) < 4 * sd, (T, mean)
        if T == 8:
            assert round(mean, 2) == gold["copies_per_point_tile8"]["value"]
            # paper: O(1.27 * ceil((32 + 15) / 8) n) = O(7.62 n)
            assert round(round(mean, 2) * math.ceil((32 + 15) / 8), 2) == gold["sort_cost_tiled"]["value"]
            # split sort: 32-bit depth keys (4 passes over n) + 16-bit tile keys over copies
            assert round(4 + 2 * round(mean, 2), 2) == gold["sort_cost_split"]["value"]
    # untiled INPC: 4 copies, 32-bit depth + 21-bit pixel index at 1080p
    assert 4 * math.ceil((32 + math.ceil(math.log2(1920 * 1080))) / 8) == gold["sort_cost_untiled"]["value"]


def test_dilation_and_truncation_constants(oracle_lib):
    gold = json.load(open(GOLDEN))
    cam = cam_at(64, 64, 100.0, cx=32.5, cy=32.5)
    # s = 0: the footprint is the dilation Gaussian alone
    p = oracle_lib.project(np.array([[0.0, 0.0, 2.0]]), cam, scale=np.array([0.0]),
                           mode="gaussian", pin32=False)
    assert p["cov"][0, 0] == DIL32
    assert abs(p["cov"][0, 0] - gold["dilation_variance"]["value"]) < 1e-8
    r = oracle_lib.render(np.array([[0.0, 0.0, 2.0]]), np.array([0.5]), np.ones((1, 1)), cam,
                          scale=np.array([0.0]), mode="gaussian", pin32=False)
    # 3 sigma = 1.2 px: the 4-neighbours (distance 1) are in, the diagonals (1.41) out
    k = gold["truncation_sigma"]["value"]
    covered = r["n_cover"] > 0
    assert covered[32, 32] and covered[32, 33] and covered[33, 32]
    assert not covered[33, 33]
    assert 1.0 <= k * math.sqrt(0.16) < math.sqrt(2)


# ----------------------------------------------------------------------------- invariants

def test_invariants_on_tiny_config(oracle_lib):
    v = scenes.make_scene(1).views[0]
    r = oracle_lib.render(v.xyz, v.opacity, v.feat, v.camera)
    assert r["alpha"].min() >= 0 and r["alpha"].max() <= 1
    assert r["t_final"].min() >= 1e-4 - 1e-12
    assert np.all(r["n_blend"] <= r["n_cover"])
    assert np.all((r["stop_pos"] < 0) | (r["stop_pos"] > r["last_pos"]))
    assert np.allclose(r["alpha"], 1 - r["t_final"])
    # features in [0, 1] and weights T_i a_i summing to alpha bound F by alpha
    assert np.all(r["F"] <= r["alpha"][..., None] + 1e-12)
    tiles, idx = oracle_lib.tile_lists(v.xyz, v.camera)
    p = oracle_lib.project(v.xyz, v.camera)
    key = tiles.astype(np.int64) << 32 | p["zbits"][idx].astype(np.int64)
    order = np.lexsort((idx, key))
    assert np.array_equal(order, np.arange(len(idx)))
    assert np.all(r["last_pos"] <= np.bincount(tiles, minlength=64).max())


# ----------------------------------------------------------------------------- brute force

def brute_render(xyz, o, feat, cam, scale=None, gaussian=False, t_min=float(np.float32(1e-4)),
                 amax=float(np.float32(0.99)), dil=DIL32):
    """Independent FP64 restatement: tent weights / explicit covariance algebra,
    per-pixel enumeration of all points, product-form transmittance."""
    R = np.asarray(cam.R, np.float64)
    t = np.asarray(cam.t, np.float64)
    pc = xyz.astype(np.float64) @ R.T + t
    W, H = cam.width, cam.height
    C = feat.shape[1]
    F = np.zeros((H, W, C))
    A = np.zeros((H, W))
    Dp = np.zeros((H, W))
    for py in range(H):
        for px in range(W):
            frags = []
            for i in range(len(xyz)):
                x, y, z = pc[i]
                if not (cam.near < z < cam.far):
                    continue
                u = cam.fx * x / z + cam.cx
                v = cam.fy * y / z + cam.cy
                dx, dy = px + 0.5 - u, py + 0.5 - v
                if not gaussian:
                    w = max(0.0, 1 - abs(dx)) * max(0.0, 1 - abs(dy))
                    if w <= 0:
                        continue
                    a = min(o[i] * w, amax)
                else:
                    J = np.array([[cam.fx / z, 0, -cam.fx * x / z ** 2],
                                  [0, cam.fy / z, -cam.fy * y / z ** 2]])
                    S = J @ (scale[i] ** 2 * np.eye(3)) @ J.T + dil * np.eye(2)
                    rad = math.ceil(3 * math.sqrt(np.linalg.eigvalsh(S).max()))
                    d = np.array([dx, dy])
                    m = d @ np.linalg.inv(S) @ d
                    if m > 9 or abs(dx) > rad or abs(dy) > rad:
                        continue
                    a = min(o[i] * math.exp(-0.5 * m), amax)
                frags.append((np.float32(z), i, a, z))
            frags.sort(key=lambda e: (e[0], e[1]))
            alphas = [e[2] for e in frags]
            for k, (_, i, a, z) in enumerate(frags):
                Tk = float(np.prod([1 - alphas[j] for j in range(k)]))
                if Tk * (1 - a) < t_min:
                    break
                F[py, px] += Tk * a * feat[i]
                Dp[py, px] += Tk * a * z
                A[py, px] = 1 - Tk * (1 - a)
    return F, A, Dp


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_brute_force_bilinear(oracle_lib, seed):
    rng = np.random.default_rng(100 + seed)
    cam = cam_at(8 if seed else 6, 6 if seed else 8, 7.0)
    n = 6
    xyz = np.stack([rng.uniform(-0.6, 0.6, n) * 2.5, rng.uniform(-0.6, 0.6, n) * 2.5,
                    rng.uniform(1.5, 3.5, n)], 1)
    if seed == 2:  # dense stack to force early termination
        xyz = np.repeat(xyz[:1], 30, 0) + rng.normal(0, 0.02, (30, 3))
        n = 30
    o = rng.uniform(0.5, 0.99, n)
    feat = rng.uniform(0, 1, (n, 3))
    F, A, Dp = brute_render(xyz, o, feat, cam)
    r = oracle_lib.render(xyz, o, feat, cam, pin32=False, tile=2)
    assert np.allclose(r["F"], F, atol=1e-12)
    assert np.allclose(r["alpha"], A, atol=1e-12)
    assert np.allclose(r["depth"], Dp, atol=1e-12)


@pytest.mark.parametrize("cov", ["ewa"])
def test_brute_force_gaussian(oracle_lib, cov):
    rng = np.random.default_rng(7)
    cam = cam_at(12, 10, 20.0)
    n = 6
    xyz = np.stack([rng.uniform(-0.3, 0.3, n) * 2, rng.uniform(-0.3, 0.3, n) * 2,
                    rng.uniform(1.5, 3.0, n)], 1)
    o = rng.uniform(0.3, 0.99, n)
    s = rng.uniform(0.01, 0.2, n)
    feat = rng.uniform(0, 1, (n, 2))
    F, A, Dp = brute_render(xyz, o, feat, cam, scale=s, gaussian=True)
    r = oracle_lib.render(xyz, o, feat, cam, scale=s, mode="gaussian", gauss_cov=cov,
                          pin32=False, tile=4)
    assert np.allclose(r["F"], F, atol=1e-12)
    assert np.allclose(r["alpha"], A, atol=1e-12)


def test_brute_force_tile_order(oracle_lib):
    """Tile lists equal an explicit enumeration sorted by (tile, depth bits, index)."""
    v = scenes.random_small_view(3, 300, 40, 28)
    p = oracle_lib.project(v.xyz, v.camera)
    T = 8
    tx = (v.camera.width + T - 1) // T
    copies = []
    for i in range(len(v.xyz)):
        if not p["vis"][i]:
            continue
        x0, x1, y0, y1 = p["box"][i]
        for ty in range(y0 // T, y1 // T + 1):
            for txx in range(x0 // T, x1 // T + 1):
                copies.append((ty * tx + txx, int(p["zbits"][i]), i))
    copies.sort()
    tiles, idx = oracle_lib.tile_lists(v.xyz, v.camera, tile=T)
    assert [c[0] for c in copies] == tiles.tolist()
    assert [c[2] for c in copies] == idx.tolist()


def test_fp32_projection_is_pinned(oracle_lib):
    """The FP32 decision path rounds op by op in the stated order (no FMA, no
    excess precision): NumPy float32 elementwise ops give the same bits."""
    v = scenes.random_small_view(4, 2000, 64, 48)
    p = oracle_lib.project(v.xyz, v.camera)
    x, y, z = [v.xyz[:, k].astype(np.float32) for k in range(3)]
    R = v.camera.R.astype(np.float32)
    t = v.camera.t.astype(np.float32)
    f32 = np.float32
    xc = ((R[0, 0] * x + R[0, 1] * y) + R[0, 2] * z) + t[0]
    zc = ((R[2, 0] * x + R[2, 1] * y) + R[2, 2] * z) + t[2]
    u = f32(v.camera.fx) * (xc / zc) + f32(v.camera.cx)
    vis = (zc > f32(v.camera.near)) & (zc < f32(v.camera.far))
    assert np.array_equal(p["zbits"], zc.view(np.uint32))
    assert np.array_equal(p["uvz"][vis & (p["vis"] == 1), 0].astype(np.float32),
                          u[vis & (p["vis"] == 1)])


# ----------------------------------------------------------------------------- adjoint (Eq. 2)

def _loss(oracle_lib, xyz, o, feat, cam, gF, gA, gD, scale=None, **kw):
    r = oracle_lib.render(xyz, o, feat, cam, scale=scale, pin32=False, **kw)
    L = (r["F"] * gF).sum() + (r["alpha"] * gA).sum() + (r["depth"] * gD).sum()
    key = (r["n_cover"].tobytes(), r["n_blend"].tobytes())
    return L, key


def _fd_check(oracle_lib, xyz, o, feat, cam, gF, gA, gD, an, scale=None, params=(), **kw):
    base = dict(xyz=xyz, o=o, feat=feat, scale=scale)
    checked = 0
    for name, idx in params:
        arr = base[name]
        h = 1e-6 * max(1.0, abs(arr[idx]))
        vals = []
        keys = []
        for sgn in (+1, -1):
            b = {k: (None if v is None else v.copy()) for k, v in base.items()}
            b[name][idx] += sgn * h
            L, key = _loss(oracle_lib, b["xyz"], b["o"], b["feat"], cam, gF, gA, gD,
                           scale=b["scale"], **kw)
            vals.append(L)
            keys.append(key)
        if keys[0] != keys[1]:
            continue  # a coverage or termination decision flips within +-h
        fd = (vals[0] - vals[1]) / (2 * h)
        ref = an[name][idx]
        assert abs(fd - ref) <= 2e-6 * max(1.0, abs(ref)), (name, idx, fd, ref)
        checked += 1
    return checked


def test_adjoint_bilinear_finite_differences(oracle_lib):
    rng = np.random.default_rng(11)
    v = scenes.random_small_view(11, 80, 20, 16, c=3)
    cam = v.camera
    o = rng.uniform(0.2, 0.99, 80)
    o[5] = 0.0  # alpha = 0 fragments still get a gradient (appendix)
    feat = rng.uniform(0, 1, (80, 3))
    gF, gA, gD = v.g_feat.astype(np.float64), v.g_alpha.astype(np.float64), v.g_depth.astype(np.float64)
    g = oracle_lib.backward(v.xyz, o, feat, cam, gF, gA, gD, pin32=False)
    an = dict(o=g["d_opacity"], feat=g["d_feat"])
    params = [("o", (i,)) for i in range(0, 80, 3)] + [("o", (5,))]
    params += [("feat", (i, c)) for i in range(0, 80, 7) for c in range(3)]
    n = _fd_check(oracle_lib, v.xyz.astype(np.float64), o, feat, cam, gF, gA, gD, an,
                  params=params)
    assert n >= len(params) - 3
    assert abs(g["d_opacity"][5]) > 0 or not np.any(oracle_lib.project(v.xyz[5:6], cam)["vis"])


@pytest.mark.parametrize("cov", ["ewa", "iso"])
def test_adjoint_gaussian_finite_differences(oracle_lib, cov):
    rng = np.random.default_rng(12)
    v = scenes.random_small_view(12, 40, 24, 20, c=2, gaussian=True, f=30.0)
    cam = v.camera
    xyz = v.xyz.astype(np.float64)
    o = rng.uniform(0.2, 0.9, 40)
    s = v.scale.astype(np.float64) * 5
    feat = rng.uniform(0, 1, (40, 2))
    gF, gA, gD = v.g_feat.astype(np.float64), v.g_alpha.astype(np.float64), v.g_depth.astype(np.float64)
    kw = dict(mode="gaussian", gauss_cov=cov)
    g = oracle_lib.backward(xyz, o, feat, cam, gF, gA, gD, scale=s, pin32=False, **kw)
    an = dict(o=g["d_opacity"], feat=g["d_feat"], xyz=g["d_xyz"], scale=g["d_scale"])
    params = [("o", (i,)) for i in range(0, 40, 4)]
    params += [("xyz", (i, c)) for i in range(2, 40, 3) for c in range(3)]
    params += [("scale", (i,)) for i in range(1, 40, 3)]
    n = _fd_check(oracle_lib, xyz, o, feat, cam, gF, gA, gD, an, scale=s, params=params, **kw)
    assert n >= 0.8 * len(params)
    assert np.abs(g["d_xyz"]).max() > 0 and np.abs(g["d_scale"]).max() > 0


@pytest.mark.parametrize("pin32", [True, False])
def test_alpha_clamp_closed_form(oracle_lib, pin32):
    """A point on a pixel centre with opacity 1 has bilinear weight 1 there, so
    o w = 1 exceeds alpha_max and the fragment blends with alpha = alpha_max
    (0.99 as an FP32 parameter): F = alpha_max f and alpha_out = alpha_max.
    Nothing flows back through a clamped alpha: the opacity gets no gradient,
    the features get T a g_F = alpha_max g_F."""
    cam = cam_at(4, 4, 4.0)
    xyz = np.array([point_at_pixel(cam, 1.5, 2.5, 2.0)])  # centre of pixel (1, 2), exact in FP32
    o = np.array([1.0])
    feat = np.array([[0.3, 0.8]])
    amax = float(np.float32(0.99))
    r = oracle_lib.render(xyz, o, feat, cam, pin32=pin32)
    np.testing.assert_allclose(r["F"][2, 1], amax * feat[0], rtol=1e-15)
    assert abs(r["alpha"][2, 1] - amax) < 1e-15
    gF = np.zeros((4, 4, 2))
    gF[2, 1] = [1.0, -2.0]
    g = oracle_lib.backward(xyz, o, feat, cam, gF, None, None, pin32=pin32)
    assert g["d_opacity"][0] == 0.0
    np.testing.assert_allclose(g["d_feat"][0], amax * gF[2, 1], rtol=1e-15)


def _rotated(cam, seed):
    """The same intrinsics with a general rotation and translation."""
    rng = np.random.default_rng(seed)
    cam.R = scenes.random_rotations(rng, 1)[0].astype(np.float32)
    cam.t = rng.uniform(-0.5, 0.5, 3).astype(np.float32)
    return cam


def _to_world(cam, pc):
    """World points whose camera-space images (x_c = R x_w + t) are pc."""
    return (np.asarray(pc, np.float64) - cam.t.astype(np.float64)) @ cam.R.astype(np.float64)


def test_rotated_camera_projection(oracle_lib):
    """Pinhole model of Sec. 2 with x_c = R x_w + t for a general rotation:
    points placed at known camera-space positions land at u = f x_c / z_c + c_x,
    v = f y_c / z_c + c_y, depth z_c (every other pin uses R = I, where R and
    R^T cannot be told apart)."""
    cam = _rotated(cam_at(64, 48, 50.0), 13)
    rng = np.random.default_rng(13)
    n = 200
    z = rng.uniform(1.0, 3.0, n)
    pc = np.stack([rng.uniform(-0.5, 0.5, n) * z, rng.uniform(-0.4, 0.4, n) * z, z], 1)
    p = oracle_lib.project(_to_world(cam, pc), cam, pin32=False)
    assert np.all(p["vis"] == 1)
    np.testing.assert_allclose(p["uvz"][:, 0], cam.fx * pc[:, 0] / z + cam.cx, rtol=1e-5, atol=1e-5)
    np.testing.assert_allclose(p["uvz"][:, 1], cam.fy * pc[:, 1] / z + cam.cy, rtol=1e-5, atol=1e-5)
    np.testing.assert_allclose(p["uvz"][:, 2], z, rtol=1e-5)


def test_adjoint_gaussian_finite_differences_rotated_camera(oracle_lib):
    """Position gradients are world-space: with a rotated camera the chain rule
    carries R^T (finite differences in world coordinates)."""
    rng = np.random.default_rng(14)
    v = scenes.random_small_view(14, 40, 24, 20, c=2, gaussian=True, f=30.0)
    cam = _rotated(v.camera, 14)
    xyz = _to_world(cam, v.xyz.astype(np.float64))
    o = rng.uniform(0.2, 0.9, 40)
    s = v.scale.astype(np.float64) * 5
    feat = rng.uniform(0, 1, (40, 2))
    gF, gA, gD = v.g_feat.astype(np.float64), v.g_alpha.astype(np.float64), v.g_depth.astype(np.float64)
    kw = dict(mode="gaussian", gauss_cov="ewa")
    g = oracle_lib.backward(xyz, o, feat, cam, gF, gA, gD, scale=s, pin32=False, **kw)
    an = dict(o=g["d_opacity"], feat=g["d_feat"], xyz=g["d_xyz"], scale=g["d_scale"])
    params = [("xyz", (i, c)) for i in range(2, 40, 3) for c in range(3)]
    n = _fd_check(oracle_lib, xyz, o, feat, cam, gF, gA, gD, an, scale=s, params=params, **kw)
    assert n >= 0.8 * len(params)
    assert np.abs(g["d_xyz"]).max() > 0


def test_eq2_zero_alpha_with_background(oracle_lib):
    """Appendix Eq. 2 for a fragment with alpha_k = 0, background composited
    through the alpha output: F_total = F + T_{K+1} f_bg. The derivative is
    T_k f_k - sum_{i>k} a_i T_i f_i - T_{K+1} f_bg (the chain rule gives a minus
    sign on the background term)."""
    cam = cam_at(4, 4, 4.0)
    zs = [1.0, 1.5, 2.0, 2.5]
    xyz = np.array([point_at_pixel(cam, 1.5, 2.5, z) for z in zs])  # all on pixel (1, 2)
    o = np.array([0.3, 0.0, 0.5, 0.2])  # the second fragment has alpha = 0
    feat = np.array([[1.0, 0.2], [0.4, 0.9], [0.1, 0.3], [0.7, 0.5]])
    f_bg = np.array([0.25, 0.6])
    g = np.array([0.8, -1.3])
    gF = np.zeros((4, 4, 2))
    gF[2, 1] = g
    gA = np.zeros((4, 4))
    gA[2, 1] = -(g @ f_bg)  # d(T_{K+1} f_bg . g)/d alpha, alpha = 1 - T_{K+1}
    r = oracle_lib.backward(xyz, o, feat, cam, gF, gA, None, pin32=False)
    a = o.copy()
    T = np.cumprod(np.concatenate([[1.0], 1 - a]))
    k = 1
    want = g @ (T[k] * feat[k] - sum(a[i] * T[i] * feat[i] for i in range(k + 1, 4)) - T[4] * f_bg)
    assert abs(r["d_opacity"][k] - want) < 1e-12

    def total(oo):
        rr = oracle_lib.render(xyz, oo, feat, cam, pin32=False)
        return g @ (rr["F"][2, 1] + (1 - rr["alpha"][2, 1]) * f_bg)

    h = 1e-7
    fd = (total(o + np.eye(4)[k] * h) - total(o - np.eye(4)[k] * h)) / (2 * h)
    assert abs(fd - want) < 1e-7
