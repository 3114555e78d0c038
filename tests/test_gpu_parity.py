"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle, element
by element on the same seeded inputs.

Bars: records, tile rects, sorted copy lists and per-pixel last-contributor
positions are bit-exact (integer work, and FP32 values both sides compute with
the same rounded operations); images within 1e-5 relative + 1e-7 absolute
(FP32 accumulation against FP64); gradients normwise 1e-5 and elementwise
1e-4 |ref| + 1e-6 max|ref| (the replay divides by 1 - a once per fragment).
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2508_19140_gb300 import scenes

from gpu_util import Run, bf16_round, tile_offsets

pytestmark = pytest.mark.gpu

RTOL, ATOL = 1e-5, 1e-7
G_NORM, G_ELEM_R, G_ELEM_A = 1e-5, 1e-4, 1e-6


@pytest.fixture(scope="module", autouse=True)
def _need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2508_19140_gb300 import build
    build.build()
    oracle.build()


def case_view(name):
    if name == "tiny":
        return scenes.make_scene(1).views[0]
    if name == "ragged":
        return scenes.random_small_view(21, 6000, 100, 75)
    if name == "tall":
        return scenes.random_small_view(22, 3000, 37, 129, c=3)
    if name == "line":
        return scenes.random_small_view(23, 500, 161, 1, c=1)
    if name == "dense":  # deep lists: early termination everywhere
        v = scenes.random_small_view(24, 40000, 48, 40, c=8)
        return v
    if name == "gauss":
        return scenes.random_small_view(25, 4000, 90, 70, c=4, gaussian=True, f=80.0)
    if name == "gauss_tiny_sigma":
        v = scenes.random_small_view(26, 3000, 64, 48, c=2, gaussian=True, f=60.0)
        v.scale = v.scale * 0.1
        return v
    raise KeyError(name)


BILIN = ["tiny", "ragged", "tall", "line", "dense"]
GAUSS = ["gauss", "gauss_tiny_sigma"]


def oracle_kw(mode, cov="ewa"):
    return dict(mode=mode, gauss_cov=cov, tile=16, pin32=True)


def _mode(name):
    return "gaussian" if name.startswith("gauss") else "bilinear"


# ----------------------------------------------------------------------------- K1

@pytest.mark.parametrize("name", BILIN + GAUSS)
def test_records_and_rects_bit_exact(name):
    v = case_view(name)
    mode = _mode(name)
    r = Run([v], mode=mode)
    assert r.status == 0
    p = oracle.project(v.xyz, v.camera, scale=v.scale if mode == "gaussian" else None,
                       **oracle_kw(mode))
    rec = r.records()
    vis = p["vis"] == 1
    f32 = lambda a: np.asarray(a, np.float64).astype(np.float32).view(np.uint32)
    assert np.array_equal(rec[vis, 0], f32(p["uvz"][vis, 0]))
    assert np.array_equal(rec[vis, 1], f32(p["uvz"][vis, 1]))
    assert np.array_equal(rec[vis, 2], p["zbits"][vis])
    assert np.array_equal(rec[vis, 3], v.opacity[vis].view(np.uint32))
    if mode == "gaussian":
        for k in range(3):
            assert np.array_equal(rec[vis, 4 + k], f32(p["conic"][vis, k]))
    n = len(v.xyz)
    box = p["box"]
    if mode == "gaussian":
        rect = r.arr("rect", np.uint32, 2 * n).reshape(n, 2)
        tx0, ty0 = rect[:, 0] & 0xFFFF, rect[:, 0] >> 16
        tx1, ty1 = rect[:, 1] & 0xFFFF, rect[:, 1] >> 16
    else:
        # bilinear rects are packed: tx0 | ty0 << 16 | (tx1 - tx0) << 30 | (ty1 - ty0) << 31
        p4 = r.arr("rect", np.uint32, n).astype(np.int64)
        tx0, ty0 = p4 & 0xFFFF, (p4 >> 16) & 0x3FFF
        tx1, ty1 = tx0 + ((p4 >> 30) & 1), ty0 + (p4 >> 31)
        assert np.all(p4[~vis] == 0xFFFFFFFF)
    assert np.array_equal(tx0[vis], box[vis, 0] // 16) and np.array_equal(tx1[vis], box[vis, 1] // 16)
    assert np.array_equal(ty0[vis], box[vis, 2] // 16) and np.array_equal(ty1[vis], box[vis, 3] // 16)
    if mode == "gaussian":  # bilinear counts are read from the packed rect
        cnt = r.arr("count", np.uint32, n)
        assert np.all(cnt[~vis] == 0)
        assert np.array_equal(cnt[vis], (tx1 - tx0 + 1)[vis] * (ty1 - ty0 + 1)[vis])


# ----------------------------------------------------------------------------- K2-K5

@pytest.mark.parametrize("name", BILIN + GAUSS)
def test_sorted_copies_bit_exact(name):
    v = case_view(name)
    mode = _mode(name)
    r = Run([v], mode=mode)
    tiles, idx = oracle.tile_lists(v.xyz, v.camera, scale=v.scale if mode == "gaussian" else None,
                                   **oracle_kw(mode))
    keys, vals = r.sorted_copies()
    assert int(r.stats["n_copies"]) == len(tiles)
    assert np.array_equal(keys, tiles.astype(np.uint32))
    assert np.array_equal(vals, idx.astype(np.uint32))
    P = tile_offsets([v])[-1]
    ranges = r.arr("ranges", np.uint32, 2 * P).reshape(P, 2)
    cnt = np.bincount(tiles, minlength=P)
    assert np.array_equal(ranges[:, 1] - ranges[:, 0], cnt)
    nz = cnt > 0
    assert np.array_equal(ranges[nz, 0], np.searchsorted(tiles, np.arange(P)[nz]))


# ----------------------------------------------------------------------------- K6

def _check_image(r, ref, mask=None, rtol=RTOL, atol=ATOL):
    F, A, D = r.image()
    m = np.ones(A.shape, bool) if mask is None else mask
    np.testing.assert_allclose(F[m], ref["F"][m], rtol=rtol, atol=atol)
    np.testing.assert_allclose(A[m], ref["alpha"][m], rtol=rtol, atol=atol)
    np.testing.assert_allclose(D[m], ref["depth"][m], rtol=rtol, atol=atol * 10)


@pytest.mark.parametrize("name", BILIN)
def test_forward_bilinear(name):
    v = case_view(name)
    r = Run([v])
    ref = oracle.render(v.xyz, v.opacity, v.feat, v.camera, **oracle_kw("bilinear"))
    _check_image(r, ref)
    tf, last = r.pixel_state()
    assert np.array_equal(last, ref["last_pos"].astype(np.uint32))
    np.testing.assert_allclose(tf, ref["t_final"], rtol=RTOL, atol=ATOL)
    assert int(r.stats["needed_records"]) == ref["needed"]


@pytest.mark.parametrize("name", GAUSS)
@pytest.mark.parametrize("cov", ["ewa", "iso"])
def test_forward_gaussian(name, cov):
    v = case_view(name)
    r = Run([v], mode="gaussian", gauss_cov=cov)
    ref = oracle.render(v.xyz, v.opacity, v.feat, v.camera, scale=v.scale, **oracle_kw("gaussian", cov))
    # exp() may differ by an ulp between the CPU and GPU libraries: pixels whose
    # termination decision sits within that of the threshold are not comparable.
    # Every other pixel is held to the FP32 image bar (measured: at most
    # 6e-7 relative on these cases).
    ok = ref["margin"] > 1e-5
    assert ok.mean() > 0.99
    _check_image(r, ref, ok)
    tf, last = r.pixel_state()
    assert np.array_equal(last[ok], ref["last_pos"][ok].astype(np.uint32))


# ----------------------------------------------------------------------------- K7-K8

def _check_grad(got, ref, norm=G_NORM, er=G_ELEM_R, ea=G_ELEM_A, mask=None):
    g = np.asarray(got, np.float64)
    f = np.asarray(ref, np.float64)
    if mask is not None:
        g, f = g[mask], f[mask]
    den = max(np.linalg.norm(f), 1e-30)
    assert np.linalg.norm(g - f) / den <= norm, np.linalg.norm(g - f) / den
    bound = er * np.abs(f) + ea * np.abs(f).max()
    bad = np.abs(g - f) > bound
    assert not bad.any(), (np.argwhere(bad)[:5], g[bad][:5], f[bad][:5])


@pytest.mark.parametrize("name", BILIN)
def test_backward_bilinear(name):
    v = case_view(name)
    r = Run([v], backward=True)
    ref = oracle.backward(v.xyz, v.opacity, v.feat, v.camera, v.g_feat, v.g_alpha, v.g_depth,
                          **oracle_kw("bilinear"))
    g = r.grads()
    _check_grad(g["d_feat"], ref["d_feat"])
    _check_grad(g["d_opacity"], ref["d_opacity"])


@pytest.mark.parametrize("name", GAUSS)
@pytest.mark.parametrize("cov", ["ewa", "iso"])
def test_backward_gaussian(name, cov):
    v = case_view(name)
    r = Run([v], mode="gaussian", gauss_cov=cov, backward=True)
    kw = oracle_kw("gaussian", cov)
    ref_img = oracle.render(v.xyz, v.opacity, v.feat, v.camera, scale=v.scale, **kw)
    # points touching a termination-ambiguous pixel are excluded
    amb = ref_img["margin"] <= 1e-5
    p = oracle.project(v.xyz, v.camera, scale=v.scale, **kw)
    keep = np.ones(len(v.xyz), bool)
    for i in np.nonzero(p["vis"])[0]:
        x0, x1, y0, y1 = p["box"][i]
        if amb[y0:y1 + 1, x0:x1 + 1].any():
            keep[i] = False
    ref = oracle.backward(v.xyz, v.opacity, v.feat, v.camera, v.g_feat, v.g_alpha, v.g_depth,
                          scale=v.scale, **kw)
    g = r.grads()
    # FP32 chain through the 2x2 inverse and the Jacobian: looser bars
    _check_grad(g["d_feat"], ref["d_feat"], mask=keep)
    _check_grad(g["d_opacity"], ref["d_opacity"], norm=1e-4, er=1e-3, ea=1e-5, mask=keep)
    _check_grad(g["d_xyz"], ref["d_xyz"], norm=1e-4, er=1e-3, ea=1e-5, mask=keep)
    _check_grad(g["d_scale"], ref["d_scale"], norm=1e-4, er=1e-3, ea=1e-5, mask=keep)


# ----------------------------------------------------------------------------- BF16 features

def test_bf16_features_forward_and_backward():
    v = case_view("dense")
    r = Run([v], bf16=True, backward=True)
    fb = bf16_round(v.feat)
    ref_b = oracle.render(v.xyz, v.opacity, fb, v.camera, **oracle_kw("bilinear"))
    _check_image(r, ref_b)  # accumulation error only
    # Total error against FP32 features: BF16 rounds each (non-negative) feature
    # by at most its unit roundoff 2^-8 relative, and the blend weights are
    # non-negative, so |F_bf16 - F| <= 2^-8 F plus the accumulation error.
    # Elementwise, 2e-3 relative is below BF16's own unit roundoff (2^-8 =
    # 3.9e-3): a pixel dominated by one fragment carries that fragment's
    # rounding whole. Normwise over the image, where roundings of many
    # features average out, 2e-3 holds.
    ref_f = oracle.render(v.xyz, v.opacity, v.feat, v.camera, **oracle_kw("bilinear"))
    F, _, _ = r.image()
    assert np.all(np.abs(F - ref_f["F"]) <= (2.0 ** -8 + 2e-5) * np.abs(ref_f["F"]) + 1e-6)
    assert np.linalg.norm(F - ref_f["F"]) / np.linalg.norm(ref_f["F"]) <= 2e-3
    g = r.grads()
    ref = oracle.backward(v.xyz, v.opacity, fb, v.camera, v.g_feat, v.g_alpha, v.g_depth,
                          **oracle_kw("bilinear"))
    _check_grad(g["d_feat"], ref["d_feat"])
    _check_grad(g["d_opacity"], ref["d_opacity"])


# ----------------------------------------------------------------------------- batching

def test_batch_equals_single_views_bitwise():
    views = [case_view("tiny"), case_view("ragged"), case_view("tall")]
    for v in views:  # the batch needs one channel count
        v.feat = np.ascontiguousarray(np.concatenate([v.feat, v.feat], 1)[:, :4])
        v.g_feat = np.ascontiguousarray(np.concatenate([v.g_feat, v.g_feat], 2)[..., :4])
    rb = Run(views, backward=True)
    offs = tile_offsets(views)
    keys, vals = rb.sorted_copies()
    npt = np.cumsum([0] + [len(v.xyz) for v in views])
    for k, v in enumerate(views):
        rs = Run([v], backward=True)
        for a, b in zip(rb.image(k), rs.image()):
            assert np.array_equal(a, b)
        for key in ("d_feat", "d_opacity"):
            assert np.array_equal(rb.grads(k)[key], rs.grads()[key])
        ks, vs = rs.sorted_copies()
        sel = (keys >= offs[k]) & (keys < offs[k + 1])
        assert np.array_equal(keys[sel] - offs[k], ks)
        assert np.array_equal(vals[sel] - npt[k], vs)


@pytest.mark.parametrize("bf16", [False, True])
@pytest.mark.parametrize("name", ["tiny", "dense", "gauss"])
def test_deterministic_rerun(name, bf16):
    """Bit-identical results over repeated runs (no float atomics, no races)."""
    v = case_view(name)
    mode = _mode(name)
    runs = [Run([v], mode=mode, bf16=bf16, backward=True) for _ in range(3)]
    for r in runs[1:]:
        for x, y in zip(runs[0].image(), r.image()):
            assert np.array_equal(x, y)
        for key, val in runs[0].grads().items():
            assert np.array_equal(val, r.grads()[key]), key


# ----------------------------------------------------------------------------- saved record copy

@pytest.mark.parametrize("name,tile,depth", [("dense", 8, 64), ("ragged", 16, 0), ("tiny", 8, 256),
                                             ("dense", 16, 512)])
def test_saved_record_copy_gives_same_bits(name, tile, depth):
    """With RAST_FLAG_SAVE_FOR_BWD the forward writes the records it reads in
    tile-list order and the backward reads them from there instead of
    gathering them by point index: images and gradients are the same bits
    (also on a workspace pre-filled with 0xFF, and with BF16 features)."""
    from paper_2508_19140_gb300 import rast
    v = case_view(name)
    for bf16 in (False, True):
        a = Run([v], backward=True, bf16=bf16, tile=tile, blend_depth=depth)
        b = Run([v], backward=True, bf16=bf16, tile=tile, blend_depth=depth, ws_fill=0xFF,
                flags=rast.FLAG_SAVE_FOR_BWD)
        assert a.status == 0 and b.status == 0
        for x, y in zip(a.image(), b.image()):
            assert np.array_equal(x.view(np.uint32), y.view(np.uint32))
        for key, val in a.grads().items():
            assert np.array_equal(val.view(np.uint32), b.grads()[key].view(np.uint32)), key


# ----------------------------------------------------------------------------- stale workspace

@pytest.mark.parametrize("name,tile,depth", [("tiny", 16, 0), ("dense", 8, 64), ("ragged", 8, 64),
                                             ("gauss", 16, 0), ("gauss", 8, 0)])
def test_workspace_prefilled_with_ones_gives_same_bits(name, tile, depth):
    """Every workspace array a kernel reads is written earlier in the same
    call: a workspace whose bytes are all 0xFF before the call gives the same
    images, per-pixel state, copy lists and gradients, bit for bit, as a
    zeroed one."""
    v = case_view(name)
    mode = _mode(name)
    a = Run([v], mode=mode, backward=True, tile=tile, blend_depth=depth)
    b = Run([v], mode=mode, backward=True, tile=tile, blend_depth=depth, ws_fill=0xFF)
    assert a.status == 0 and b.status == 0
    for x, y in zip(a.image(), b.image()):
        assert np.array_equal(x.view(np.uint32), y.view(np.uint32))
    for x, y in zip(a.pixel_state(), b.pixel_state()):
        assert np.array_equal(x.view(np.uint32), y.view(np.uint32))
    for x, y in zip(a.sorted_copies(), b.sorted_copies()):
        assert np.array_equal(x, y)
    for key, val in a.grads().items():
        assert np.array_equal(val.view(np.uint32), b.grads()[key].view(np.uint32)), key


# ----------------------------------------------------------------------------- edge cases

def _tiny_cam(W=20, H=12, f=20.0):
    return scenes.identity_camera(W, H, f)


def _view(xyz, o, feat, cam, scale=None, seed=0):
    rng = np.random.default_rng(seed)
    H, W, C = cam.height, cam.width, feat.shape[1]
    return scenes.View(xyz=np.asarray(xyz, np.float32), opacity=np.asarray(o, np.float32),
                       feat=np.asarray(feat, np.float32), camera=cam,
                       scale=None if scale is None else np.asarray(scale, np.float32),
                       g_feat=rng.standard_normal((H, W, C)).astype(np.float32),
                       g_alpha=rng.standard_normal((H, W)).astype(np.float32),
                       g_depth=rng.standard_normal((H, W)).astype(np.float32))


def test_empty_point_set():
    cam = _tiny_cam()
    v = _view(np.zeros((0, 3)), np.zeros(0), np.zeros((0, 4)), cam)
    r = Run([v], backward=True)
    F, A, D = r.image()
    assert np.all(F == 0) and np.all(A == 0) and np.all(D == 0)
    assert r.stats["n_copies"] == 0 and r.status == 0


def test_all_points_culled():
    cam = _tiny_cam()
    xyz = [[0, 0, -1.0], [0, 0, 0.1], [100.0, 0, 1.0], [0, 0, 2e4]]
    v = _view(xyz, [0.5] * 4, np.ones((4, 2)), cam)
    r = Run([v], backward=True)
    F, A, _ = r.image()
    assert np.all(F == 0) and np.all(A == 0)
    g = r.grads()
    assert np.all(g["d_feat"] == 0) and np.all(g["d_opacity"] == 0)


def test_stacked_points_terminate_and_ties_break_by_index():
    cam = _tiny_cam()
    K = 40
    xyz = np.array([[(3.5 - cam.cx) * 2 / cam.fx, (4.5 - cam.cy) * 2 / cam.fy, 2.0]] * K)
    o = np.linspace(0.2, 0.9, K)
    feat = np.random.default_rng(1).random((K, 3))
    v = _view(xyz, o, feat, cam)
    r = Run([v], backward=True)
    ref = oracle.render(v.xyz, v.opacity, v.feat, cam, **oracle_kw("bilinear"))
    _check_image(r, ref)
    _, last = r.pixel_state()
    assert np.array_equal(last, ref["last_pos"].astype(np.uint32))
    assert ref["stop_pos"][4, 3] > 0
    g = oracle.backward(v.xyz, v.opacity, v.feat, cam, v.g_feat, v.g_alpha, v.g_depth,
                        **oracle_kw("bilinear"))
    _check_grad(r.grads()["d_opacity"], g["d_opacity"])
    keys, vals = r.sorted_copies()
    assert np.array_equal(vals, np.sort(vals))  # equal depth: ascending index


def test_alpha_clamp_and_zero_opacity():
    cam = _tiny_cam()
    rng = np.random.default_rng(3)
    n = 200
    xyz = np.stack([rng.uniform(-0.4, 0.4, n), rng.uniform(-0.2, 0.2, n), rng.uniform(1.5, 3, n)], 1)
    o = rng.choice([0.0, 0.995, 1.0, 0.5], n)
    v = _view(xyz, o, rng.random((n, 4)), cam)
    r = Run([v], backward=True)
    ref = oracle.render(v.xyz, v.opacity, v.feat, cam, **oracle_kw("bilinear"))
    _check_image(r, ref)
    g = oracle.backward(v.xyz, v.opacity, v.feat, cam, v.g_feat, v.g_alpha, v.g_depth,
                        **oracle_kw("bilinear"))
    _check_grad(r.grads()["d_opacity"], g["d_opacity"])
    assert np.any(g["d_opacity"][o == 0] != 0)  # alpha = 0 fragments still get gradients


def test_points_on_pixel_centres_and_borders():
    cam = _tiny_cam(17, 9, 10.0)
    us = np.array([0.5, 1.0, 16.5, 17.0, 8.5, -0.5, 0.0, 3.25])
    vs = np.array([0.5, 8.5, 4.0, 9.0, 0.0, 4.5, -0.25, 8.99])
    z = np.full(len(us), 2.0)
    xyz = np.stack([(us - cam.cx) * z / cam.fx, (vs - cam.cy) * z / cam.fy, z], 1)
    v = _view(xyz, np.full(len(us), 0.7), np.eye(len(us))[:, :4] + 0.1, cam)
    r = Run([v], backward=True)
    ref = oracle.render(v.xyz, v.opacity, v.feat, cam, **oracle_kw("bilinear"))
    _check_image(r, ref)
    tiles, idx = oracle.tile_lists(v.xyz, cam, **oracle_kw("bilinear"))
    keys, vals = r.sorted_copies()
    assert np.array_equal(keys, tiles) and np.array_equal(vals, idx)


def test_capacity_overflow_is_reported_not_written():
    v = case_view("gauss")
    r = Run([v], mode="gaussian", max_copies=1)
    st, stats = r.status, r.stats
    assert stats["n_copies"] > stats["copy_capacity"]
    assert st == 2  # RAST_ERR_CAPACITY
    F, A, _ = r.image()  # nothing is blended from a truncated list
    assert np.all(F == 0) and np.all(A == 0)


def test_bounded_wait_runs_out_and_is_reported():
    """Failure detection without a fault: the test hook makes the depth
    sort's first pass withhold one look-back word, so the next tile's bounded
    wait runs out. The call must return, report RAST_ERR_TIMEOUT, blend
    nothing from the partial order (empty images, zero gradients), and leave
    the context usable: a normal call right after matches the oracle."""
    from paper_2508_19140_gb300 import rast
    v = scenes.random_small_view(31, 20000, 96, 64)  # > 4096 points: several sort tiles
    r = Run([v], backward=True, flags=rast.FLAG_TEST_SORT_STALL, ws_fill=0xFF)
    assert r.status == rast.RAST_ERR_TIMEOUT
    assert r.stats["n_copies"] == 0
    F, A, D = r.image()
    assert np.all(F == 0) and np.all(A == 0) and np.all(D == 0)
    for key, val in r.grads().items():
        assert np.all(val == 0), key
    ok = Run([v], backward=True)
    assert ok.status == 0
    ref = oracle.render(v.xyz, v.opacity, v.feat, v.camera, **oracle_kw("bilinear"))
    _check_image(ok, ref)


def test_gauss_backward_bounded_wait_runs_out_and_is_reported():
    """Failure detection without a fault, Gaussian backward: with the test
    hook the second batch of every tile with more than 32 replayed records is
    never staged, so the warps' waits on its barrier (64 polls under the hook)
    run out. The call must return and report RAST_ERR_TIMEOUT, the forward
    before it must be untouched, and the context must stay usable: a normal
    forward + backward afterwards gives the same bits as one before."""
    from paper_2508_19140_gb300 import rast
    v = case_view("gauss")
    before = Run([v], mode="gaussian", backward=True)
    assert rast.rasterize_get_status(before.ws)[0] == 0
    r = Run([v], mode="gaussian", backward=True, flags=rast.FLAG_TEST_BLEND_STALL, ws_fill=0xFF)
    assert r.status == 0  # the forward ignores the hook
    assert rast.rasterize_get_status(r.ws)[0] == rast.RAST_ERR_TIMEOUT
    for a, b in zip(r.image(), before.image()):
        assert np.array_equal(a, b)
    after = Run([v], mode="gaussian", backward=True)
    assert rast.rasterize_get_status(after.ws)[0] == 0
    g0, g1 = before.grads(), after.grads()
    for key in g0:
        assert np.array_equal(g0[key], g1[key]), key


def test_wide_depth_range_uses_widest_digits():
    """near 1e-4, far 1e8: depth keys bits(z) - bits(near) of 29 bits, which the
    split sort covers with its widest digits (four 8-bit passes)."""
    cam = scenes.identity_camera(96, 64, 80.0)
    cam.near, cam.far = 1e-4, 1e8
    rng = np.random.default_rng(27)
    n = 6000
    u = rng.uniform(-2.0, cam.width + 2.0, n)
    w = rng.uniform(-2.0, cam.height + 2.0, n)
    z = np.exp(rng.uniform(np.log(2e-4), np.log(5e7), n))
    z[:20] = 2e8  # beyond far
    z[20:25] = 5e-5  # inside near
    xyz = np.stack([(u - cam.cx) * z / cam.fx, (w - cam.cy) * z / cam.fy, z], 1)
    v = _view(xyz, rng.uniform(0.05, 0.9, n), rng.random((n, 4)), cam, seed=27)
    r = Run([v], backward=True)
    assert r.status == 0
    tiles, idx = oracle.tile_lists(v.xyz, cam, **oracle_kw("bilinear"))
    keys, vals = r.sorted_copies()
    assert np.array_equal(keys, tiles) and np.array_equal(vals, idx)
    ref = oracle.render(v.xyz, v.opacity, v.feat, cam, **oracle_kw("bilinear"))
    _check_image(r, ref)
    _, last = r.pixel_state()
    assert np.array_equal(last, ref["last_pos"].astype(np.uint32))
    g = oracle.backward(v.xyz, v.opacity, v.feat, cam, v.g_feat, v.g_alpha, v.g_depth,
                        **oracle_kw("bilinear"))
    _check_grad(r.grads()["d_feat"], g["d_feat"])
    _check_grad(r.grads()["d_opacity"], g["d_opacity"])
