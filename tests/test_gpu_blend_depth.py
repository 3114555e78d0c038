"""GPU parity across blend depths (records staged per blend batch).

The blend depth only changes how many records a tile's threads stage between
two barriers; each pixel still composites its fragments in list order with
the same FP32 operations. So the images, T_final and last-contributor
positions must be bit-identical to the default depth at the same tile edge,
and the gradients must match the oracle. Compiled depths: tile^2 x {1, 2}, and
x 4 for 8x8 tiles (bilinear)."""
import numpy as np
import pytest
import torch

import oracle
from paper_2508_19140_gb300 import scenes

from gpu_util import Run
from test_gpu_parity import BILIN, case_view, _check_grad

pytestmark = pytest.mark.gpu

DEPTHS = [(16, 512), (8, 128), (8, 256)]


@pytest.fixture(scope="module", autouse=True)
def _need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2508_19140_gb300 import build
    build.build()
    oracle.build()


def _same_bits(a, b):
    return np.array_equal(np.asarray(a).view(np.uint32), np.asarray(b).view(np.uint32))


@pytest.mark.parametrize("tile,depth", DEPTHS)
@pytest.mark.parametrize("name", BILIN)
def test_forward_bit_identical_across_depths(name, tile, depth):
    v = case_view(name)
    ref = Run([v], tile=tile)
    r = Run([v], tile=tile, blend_depth=depth)
    assert r.status == 0
    for a, b in zip(r.image(), ref.image()):
        assert _same_bits(a, b)
    for a, b in zip(r.pixel_state(), ref.pixel_state()):
        assert _same_bits(a, b)
    assert int(r.stats["needed_records"]) == int(ref.stats["needed_records"])


@pytest.mark.parametrize("tile,depth", DEPTHS)
@pytest.mark.parametrize("name", BILIN)
def test_backward_matches_oracle_across_depths(name, tile, depth):
    v = case_view(name)
    r = Run([v], backward=True, tile=tile, blend_depth=depth)
    kw = dict(mode="bilinear", tile=tile, pin32=True)
    ref = oracle.render(v.xyz, v.opacity, v.feat, v.camera, **kw)
    _, last = r.pixel_state()
    assert np.array_equal(last, ref["last_pos"].astype(np.uint32))
    g = oracle.backward(v.xyz, v.opacity, v.feat, v.camera, v.g_feat, v.g_alpha, v.g_depth, **kw)
    got = r.grads()
    _check_grad(got["d_feat"], g["d_feat"])
    _check_grad(got["d_opacity"], g["d_opacity"])


@pytest.mark.parametrize("tile,depth", DEPTHS)
def test_bf16_batch_deterministic_across_runs(tile, depth):
    vs = [scenes.random_small_view(41, 9000, 120, 80, c=8), scenes.random_small_view(42, 30000, 64, 48, c=8),
          scenes.random_small_view(43, 2000, 33, 91, c=8)]
    a = Run(vs, bf16=True, backward=True, tile=tile, blend_depth=depth)
    b = Run(vs, bf16=True, backward=True, tile=tile, blend_depth=depth)
    for k in range(len(vs)):
        for x, y in zip(a.image(k), b.image(k)):
            assert _same_bits(x, y)
        ga, gb = a.grads(k), b.grads(k)
        for key in ga:
            assert _same_bits(ga[key], gb[key])


def test_full_size_frame_tile8_depth256():
    """4,194,304 clustered points at 1280x832: sampled pixels and points."""
    v = scenes.make_scene(2).views[0]
    r = Run([v], backward=True, tile=8, blend_depth=256)
    assert r.status == 0
    kw = dict(mode="bilinear", tile=8, pin32=True)
    W, H = v.camera.width, v.camera.height
    rng = np.random.default_rng(5)
    pix = rng.choice(W * H, 2000, replace=False)
    ref = oracle.render(v.xyz, v.opacity, v.feat, v.camera, pix=pix, **kw)
    F, A, _ = r.image()
    np.testing.assert_allclose(F.reshape(-1, F.shape[-1])[pix], ref["F"], rtol=1e-5, atol=1e-7)
    np.testing.assert_allclose(A.reshape(-1)[pix], ref["alpha"], rtol=1e-5, atol=1e-7)
    _, last = r.pixel_state()
    assert np.array_equal(last.reshape(-1)[pix], ref["last_pos"].astype(np.uint32))
    pm = np.zeros(len(v.xyz), np.uint8)
    pm[rng.choice(len(v.xyz), 1500, replace=False)] = 1
    g = oracle.backward(v.xyz, v.opacity, v.feat, v.camera, v.g_feat, v.g_alpha, v.g_depth, pmask=pm, **kw)
    got = r.grads()
    sel = pm == 1
    for key in ("d_feat", "d_opacity"):
        a, b = got[key][sel].astype(np.float64), g[key][sel]
        assert np.linalg.norm(a - b) / np.linalg.norm(b) < 1e-5
