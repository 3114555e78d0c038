"""Host logic of the autotuner (no GPU): candidate list from the C ABI,
selection, cache keys and the JSON cache. The timer is a stand-in."""
import json

import pytest

from paper_2508_19140_gb300 import autotune, rast


@pytest.fixture(scope="module")
def lib():
    from paper_2508_19140_gb300 import build
    build.build()
    return rast.load_library()


def _views(sizes, C=8, bf16=True):
    out = []
    for (w, h, n) in sizes:
        v = rast.View()
        v.cam.width, v.cam.height = w, h
        v.pts.n, v.pts.channels = n, C
        v.pts.feat_dtype = rast.BF16 if bf16 else rast.F32
        # placeholder addresses: only the planner (no device access) sees them
        v.pts.xyz = v.pts.opacity = v.pts.feat = v.out.feat = v.grad.g_feat = 256
        v.cam.fx = v.cam.fy = 100.0
        v.cam.near_z, v.cam.far_z = 0.1, 100.0
        out.append(v)
    return out


def test_candidates_from_library(lib):
    assert rast.rasterize_tune_candidates("bilinear") == [(16, 256), (16, 512), (8, 64), (8, 128), (8, 256)]
    assert rast.rasterize_tune_candidates("gaussian") == [(16, 256), (8, 64)]
    assert lib.rasterize_tune_candidates(7, None, None, 0) == -1
    # every candidate is accepted by the workspace planner
    vs = _views([(64, 48, 100)], C=4, bf16=False)
    for mode in ("bilinear", "gaussian"):
        for t, d in rast.rasterize_tune_candidates(mode):
            assert rast.rasterize_workspace_size(vs, rast.make_opts(mode=mode, tile=t, blend_depth=d)) > 0


def test_select_min_and_ties_to_default():
    assert autotune.select({(16, 256): 3.0, (8, 64): 2.0, (8, 128): 2.5}) == (8, 64)
    assert autotune.select({(16, 256): 2.0, (8, 64): 2.0}) == (16, 256)
    assert autotune.select({(16, 256): 2.0, (8, 64): 1.99}) == (16, 256)   # within 1 %: keep the earlier
    assert autotune.select({(16, 256): 2.0, (8, 64): 1.9}) == (8, 64)
    assert autotune.select({(16, 256): None, (8, 64): 4.0}) == (8, 64)
    assert autotune.select({(16, 256): None}) is None


def test_keys_bucket_workloads(lib):
    o = rast.make_opts()
    k1 = autotune.tune_key("GB300", o, _views([(1280, 832, 4 << 20)]), 3)
    k2 = autotune.tune_key("GB300", o, _views([(1300, 820, 4200000)]), 3)
    assert k1 == k2
    assert k1 != autotune.tune_key("GB300", o, _views([(1280, 832, 16 << 20)]), 3)
    assert k1 != autotune.tune_key("GB300", o, _views([(1280, 832, 4 << 20)], C=4), 3)
    assert k1 != autotune.tune_key("GB300", o, _views([(1280, 832, 4 << 20)]), 1)
    assert k1 != autotune.tune_key("B200", o, _views([(1280, 832, 4 << 20)]), 3)
    assert k1 != autotune.tune_key("GB300", rast.make_opts(mode="gaussian"), _views([(1280, 832, 4 << 20)]), 3)


def test_autotune_times_each_candidate_and_caches(lib, tmp_path):
    cache = str(tmp_path / "tune.json")
    vs = _views([(640, 480, 1 << 20), (1920, 1080, 1 << 24)])
    o = rast.make_opts()
    seen = []
    fake = {(16, 256): 5.0, (16, 512): 6.0, (8, 64): 4.0, (8, 128): 4.5, (8, 256): 7.0}

    def timer(opts):
        seen.append((opts.tile, opts.blend_depth))
        return fake[(opts.tile, opts.blend_depth)]

    r = autotune.autotune(vs, o, 3, device_name="GB300", timer=timer, cache_file=cache)
    assert (r.tile, r.blend_depth, r.from_cache, r.save_copy) == (8, 64, False, False)
    assert seen == list(fake)
    assert (o.tile, o.blend_depth) == (16, 0)  # caller's opts untouched
    d = json.load(open(cache))
    assert d[r.key]["tile"] == 8 and d[r.key]["blend_depth"] == 64

    def boom(opts):
        raise AssertionError("cache hit must not time")

    r2 = autotune.autotune(vs, o, 3, device_name="GB300", timer=boom, cache_file=cache)
    assert (r2.tile, r2.blend_depth, r2.from_cache) == (8, 64, True)
    o2 = autotune.with_split(o, r2.tile, r2.blend_depth)
    assert (o2.tile, o2.blend_depth, o2.mode, o2.t_min) == (8, 64, o.mode, o.t_min)


def test_corrupt_cache_is_ignored(lib, tmp_path):
    cache = tmp_path / "tune.json"
    cache.write_text("{not json")
    vs = _views([(64, 64, 1000)])
    r = autotune.autotune(vs, rast.make_opts(mode="gaussian"), 1, device_name="X",
                          timer=lambda o: 1.0 if o.tile == 8 else 2.0, cache_file=str(cache))
    assert (r.tile, r.blend_depth) == (8, 64)
    assert json.load(open(cache))[r.key]["tile"] == 8


def test_no_candidate_runs(lib, tmp_path):
    with pytest.raises(RuntimeError):
        autotune.autotune(_views([(64, 64, 10)]), rast.make_opts(), 1, device_name="X",
                          timer=lambda o: None, cache_file=str(tmp_path / "t.json"))


def test_record_copy_is_a_tuned_choice_when_allowed(lib, tmp_path):
    """With RAST_FLAG_SAVE_FOR_BWD in the caller's opts and a backward pass,
    every pair is timed without and then with the record copy; the flag of
    the winner is what with_split applies. Without the caller's flag, or for
    a forward-only pass, the copy is never tried."""
    cache = str(tmp_path / "tune.json")
    vs = _views([(1280, 832, 4 << 20)], C=4, bf16=False)
    o = rast.make_opts(flags=rast.FLAG_SAVE_FOR_BWD)
    seen = []

    def timer(opts):
        save = bool(opts.flags & rast.FLAG_SAVE_FOR_BWD)
        seen.append((opts.tile, opts.blend_depth, save))
        return 2.0 if (opts.tile, opts.blend_depth, save) == (8, 64, True) else 3.0

    r = autotune.autotune(vs, o, 3, device_name="GB300", timer=timer, cache_file=cache)
    pairs = rast.rasterize_tune_candidates("bilinear")
    assert seen == [(t, d, False) for t, d in pairs] + [(t, d, True) for t, d in pairs]
    assert (r.tile, r.blend_depth, r.save_copy) == (8, 64, True)
    o2 = autotune.with_split(o, r.tile, r.blend_depth, r.save_copy)
    assert o2.flags & rast.FLAG_SAVE_FOR_BWD
    assert not autotune.with_split(o, 8, 64, False).flags & rast.FLAG_SAVE_FOR_BWD
    r2 = autotune.autotune(vs, o, 3, device_name="GB300", timer=None, cache_file=cache)
    assert (r2.from_cache, r2.save_copy) == (True, True)
    seen.clear()
    autotune.autotune(vs, rast.make_opts(), 3, device_name="X", timer=timer, use_cache=False)
    assert all(not s for _, _, s in seen)
    seen.clear()
    autotune.autotune(vs, o, 1, device_name="X", timer=timer, use_cache=False)
    assert all(s for _, _, s in seen) and len(seen) == len(pairs)
