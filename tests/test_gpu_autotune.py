"""The autotuner on the GPU: it times every compiled (tile, blend depth)
candidate on the caller's views, picks one of them, caches it, and the
rasterizer run with the tuned split gives the same images as the default."""
import numpy as np
import pytest
import torch

from paper_2508_19140_gb300 import autotune, rast, scenes

from gpu_util import Run

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2508_19140_gb300 import build
    build.build()


@pytest.mark.parametrize("mode", ["bilinear", "gaussian"])
def test_autotune_on_views(mode, tmp_path):
    g = mode == "gaussian"
    vs = [scenes.random_small_view(51, 20000, 160, 120, c=4, gaussian=g, f=120.0 if g else None),
          scenes.random_small_view(52, 8000, 96, 64, c=4, gaussian=g, f=80.0 if g else None)]
    base = Run(vs, mode=mode, backward=True)
    opts = base.opts
    cache = str(tmp_path / "tune.json")
    r = autotune.autotune(base.cviews, opts, rast.PASS_FWD | rast.PASS_BWD, cache_file=cache)
    cands = rast.rasterize_tune_candidates(mode)
    assert (r.tile, r.blend_depth) in cands and not r.from_cache
    assert {c[:2] for c in r.timings_ms} == set(cands) and not r.save_copy
    assert all(ms is not None and ms > 0 for ms in r.timings_ms.values())
    r2 = autotune.autotune(base.cviews, opts, rast.PASS_FWD | rast.PASS_BWD, cache_file=cache)
    assert r2.from_cache and (r2.tile, r2.blend_depth) == (r.tile, r.blend_depth)
    tuned = Run(vs, mode=mode, tile=r.tile, blend_depth=r.blend_depth)
    ref = Run(vs, mode=mode)
    for k in range(len(vs)):
        for a, b in zip(tuned.image(k), ref.image(k)):
            assert np.array_equal(a.view(np.uint32), b.view(np.uint32))


def test_autotune_with_record_copy_allowed(tmp_path):
    """A training step whose caller allows the forward's record copy: every
    compiled pair is timed without and with it, the winner runs, and its
    images and gradients are bit-identical to the default split's."""
    vs = [scenes.random_small_view(53, 30000, 192, 128, c=4)]
    base = Run(vs, backward=True, flags=rast.FLAG_SAVE_FOR_BWD)
    r = autotune.autotune(base.cviews, base.opts, rast.PASS_FWD | rast.PASS_BWD, use_cache=False)
    cands = rast.rasterize_tune_candidates("bilinear")
    assert set(r.timings_ms) == {(t, d, s) for t, d in cands for s in (False, True)}
    flags = rast.FLAG_SAVE_FOR_BWD if r.save_copy else 0
    tuned = Run(vs, backward=True, tile=r.tile, blend_depth=r.blend_depth, flags=flags)
    ref = Run(vs, backward=True)
    for a, b in zip(tuned.image(), ref.image()):
        assert np.array_equal(a.view(np.uint32), b.view(np.uint32))
