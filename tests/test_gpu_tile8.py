"""GPU parity with 8x8 tiles (the other compiled tile edge).

The tile edge changes the work split, not the method: every pixel still
composites its covering fragments in (depth, point index) order with the same
FP32 operations, so the images are bit-identical to the 16x16 run. The sorted
copy lists and the per-pixel last-contributor positions (1-based positions in
the pixel's tile list) depend on the tile edge and are compared with the oracle
run at tile 8; gradients against the oracle within the usual bars."""
import numpy as np
import pytest
import torch

import oracle
from paper_2508_19140_gb300 import scenes

from gpu_util import Run, tile_offsets
from test_gpu_parity import BILIN, GAUSS, case_view, _check_grad, _mode

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2508_19140_gb300 import build
    build.build()
    oracle.build()


def _kw(mode):
    return dict(mode=mode, gauss_cov="ewa", tile=8, pin32=True)


@pytest.mark.parametrize("name", BILIN + GAUSS)
def test_sorted_copies_tile8(name):
    v = case_view(name)
    mode = _mode(name)
    r = Run([v], mode=mode, tile=8)
    assert r.status == 0
    tiles, idx = oracle.tile_lists(v.xyz, v.camera, scale=v.scale if mode == "gaussian" else None,
                                   **_kw(mode))
    keys, vals = r.sorted_copies()
    assert np.array_equal(keys, tiles.astype(np.uint32))
    assert np.array_equal(vals, idx.astype(np.uint32))
    P = tile_offsets([v], T=8)[-1]
    ranges = r.arr("ranges", np.uint32, 2 * P).reshape(P, 2)
    assert np.array_equal(ranges[:, 1] - ranges[:, 0], np.bincount(tiles, minlength=P))


@pytest.mark.parametrize("name", BILIN + GAUSS)
def test_images_identical_to_tile16(name):
    v = case_view(name)
    mode = _mode(name)
    r8 = Run([v], mode=mode, tile=8)
    r16 = Run([v], mode=mode, tile=16)
    for a, b in zip(r8.image(), r16.image()):
        assert np.array_equal(a.view(np.uint32), b.view(np.uint32))
    t8, _ = r8.pixel_state()
    t16, _ = r16.pixel_state()
    assert np.array_equal(t8.view(np.uint32), t16.view(np.uint32))


@pytest.mark.parametrize("name", BILIN)
def test_forward_backward_bilinear_tile8(name):
    v = case_view(name)
    r = Run([v], backward=True, tile=8)
    kw = _kw("bilinear")
    ref = oracle.render(v.xyz, v.opacity, v.feat, v.camera, **kw)
    _, last = r.pixel_state()
    assert np.array_equal(last, ref["last_pos"].astype(np.uint32))
    assert int(r.stats["needed_records"]) == ref["needed"]
    g = oracle.backward(v.xyz, v.opacity, v.feat, v.camera, v.g_feat, v.g_alpha, v.g_depth, **kw)
    got = r.grads()
    _check_grad(got["d_feat"], g["d_feat"])
    _check_grad(got["d_opacity"], g["d_opacity"])


@pytest.mark.parametrize("name", GAUSS)
def test_forward_backward_gaussian_tile8(name):
    v = case_view(name)
    r = Run([v], mode="gaussian", backward=True, tile=8)
    kw = _kw("gaussian")
    ref = oracle.render(v.xyz, v.opacity, v.feat, v.camera, scale=v.scale, **kw)
    ok = ref["margin"] > 1e-5
    _, last = r.pixel_state()
    assert np.array_equal(last[ok], ref["last_pos"][ok].astype(np.uint32))
    p = oracle.project(v.xyz, v.camera, scale=v.scale, **kw)
    keep = np.ones(len(v.xyz), bool)
    for i in np.nonzero(p["vis"])[0]:
        x0, x1, y0, y1 = p["box"][i]
        if (~ok[y0:y1 + 1, x0:x1 + 1]).any():
            keep[i] = False
    g = oracle.backward(v.xyz, v.opacity, v.feat, v.camera, v.g_feat, v.g_alpha, v.g_depth,
                        scale=v.scale, **kw)
    got = r.grads()
    _check_grad(got["d_feat"], g["d_feat"], mask=keep)
    for key in ("d_opacity", "d_xyz", "d_scale"):
        _check_grad(got[key], g[key], norm=1e-4, er=1e-3, ea=1e-5, mask=keep)


def test_batch_tile8_bf16_deterministic():
    vs = [scenes.random_small_view(31, 6000, 100, 75), scenes.random_small_view(32, 20000, 40, 56),
          scenes.random_small_view(33, 3000, 37, 129)]
    a = Run(vs, bf16=True, backward=True, tile=8)
    b = Run(vs, bf16=True, backward=True, tile=8)
    for k in range(len(vs)):
        for x, y in zip(a.image(k), b.image(k)):
            assert np.array_equal(x.view(np.uint32), y.view(np.uint32))
        ga, gb = a.grads(k), b.grads(k)
        for key in ga:
            assert np.array_equal(ga[key].view(np.uint32), gb[key].view(np.uint32))
