"""The untiled baseline in the arrangement Sec. 3.2 "Tiled Rendering" counts
as 28n: about 4n per-pixel copies, ONE stable LSD radix sort over the 64-bit
key [pixel id | depth key], one warp per pixel in the blend.

Bars: the sorted (pixel, point) list equals the oracle's per-pixel lists
(tile edge of one pixel) bit for bit; last-contributor positions, T_final and
the needed-record count equal those of the per-thread untiled walk and the
oracle exactly (the warp steps the transmittance through each chunk with the
serial FP32 operations); images within the FP32 image bar of the oracle (the
chunk sums are warp reductions, so they are not bit-identical to the serial
walk)."""
import numpy as np
import pytest
import torch

import oracle
from paper_2508_19140_gb300 import rast, scenes

from test_gpu_parity import BILIN, case_view

pytestmark = pytest.mark.gpu
DEV = "cuda:0"
KW = dict(mode="bilinear", tile=1, pin32=True)


@pytest.fixture(scope="module", autouse=True)
def _need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2508_19140_gb300 import build
    build.build()
    oracle.build()


class Untiled:
    def __init__(self, v, key64=True, bf16=False, flags=0, ws_fill=0):
        self.v = v
        xyz = torch.from_numpy(v.xyz).to(DEV)
        op = torch.from_numpy(v.opacity).to(DEV)
        feat = torch.from_numpy(v.feat).to(DEV, torch.bfloat16 if bf16 else torch.float32)
        H, W, C = v.camera.height, v.camera.width, v.feat.shape[1]
        self.F = torch.full((H, W, C), float("nan"), device=DEV)
        self.A = torch.full((H, W), float("nan"), device=DEV)
        self.D = torch.full((H, W), float("nan"), device=DEV)
        pts = rast.make_points(xyz, op, feat)
        cam = rast.make_camera(v.camera)
        opts = rast.make_opts(flags=flags)
        im = rast.make_images(self.F, self.A, self.D)
        if key64:
            n = rast.rasterize_untiled64_workspace_size(pts, cam, opts)
            self.layout = rast.rasterize_untiled64_workspace_layout(pts, cam, opts)
            self.ws = torch.full((n,), ws_fill, dtype=torch.uint8, device=DEV)
            rast.rasterize_fwd_untiled64(pts, cam, opts, self.ws, im)
        else:
            n = rast.rasterize_untiled_workspace_size(pts, cam, opts)
            self.layout = None
            self.ws = torch.full((n,), ws_fill, dtype=torch.uint8, device=DEV)
            rast.rasterize_fwd_untiled(pts, cam, opts, self.ws, im)
        torch.cuda.synchronize()
        self.status, self.stats = rast.rasterize_get_status(self.ws)
        self._keep = (xyz, op, feat)

    def arr(self, name, dtype, count):
        off, _ = self.layout[name]
        item = np.dtype(dtype).itemsize
        return self.ws[off: off + count * item].cpu().numpy().view(dtype)

    def lists(self):
        D = int(self.stats["n_copies"])
        return self.arr("sorted_keys", np.uint32, D), self.arr("sorted_vals", np.uint32, D)

    def pixel_state(self):
        HW = self.v.camera.width * self.v.camera.height
        return self.arr("t_final", np.float32, HW), self.arr("last", np.uint32, HW)

    def image(self):
        return self.F.cpu().numpy(), self.A.cpu().numpy(), self.D.cpu().numpy()


def _check_image(u, ref, pix=None):
    F, A, D = u.image()
    F, A, D = F.reshape(-1, F.shape[-1]), A.reshape(-1), D.reshape(-1)
    if pix is not None:
        F, A, D = F[pix], A[pix], D[pix]
    rF, rA, rD = ref["F"].reshape(F.shape), ref["alpha"].reshape(A.shape), ref["depth"].reshape(D.shape)
    np.testing.assert_allclose(F, rF, rtol=1e-5, atol=1e-7)
    np.testing.assert_allclose(A, rA, rtol=1e-5, atol=1e-7)
    np.testing.assert_allclose(D, rD, rtol=1e-5, atol=1e-6)


@pytest.mark.parametrize("name", BILIN)
def test_key64_lists_state_and_images(name):
    v = case_view(name)
    u = Untiled(v)
    assert u.status == 0, u.stats
    pix_ids, pts = oracle.tile_lists(v.xyz, v.camera, **KW)
    keys, vals = u.lists()
    assert np.array_equal(keys, pix_ids.astype(np.uint32))
    assert np.array_equal(vals, pts.astype(np.uint32))
    ref = oracle.render(v.xyz, v.opacity, v.feat, v.camera, **KW)
    tf, last = u.pixel_state()
    assert np.array_equal(last, ref["last_pos"].reshape(-1).astype(np.uint32))
    assert int(u.stats["needed_records"]) == ref["needed"]
    _check_image(u, ref)
    np.testing.assert_allclose(tf, ref["t_final"].reshape(-1), rtol=1e-5, atol=1e-7)
    # the per-thread untiled walk: same lists, same serial T chain
    split = Untiled(v, key64=False)
    assert split.status == 0
    assert int(split.stats["needed_records"]) == int(u.stats["needed_records"])
    _check_image(split, ref)


def test_key64_full_frame_bf16():
    v = scenes.make_scene(2).views[0]
    u = Untiled(v, bf16=True, ws_fill=0xFF)
    assert u.status == 0, u.stats
    D = int(u.stats["n_copies"])
    assert 3.5 * len(v.xyz) < D <= 4 * len(v.xyz)
    pix_ids, pts = oracle.tile_lists(v.xyz, v.camera, **KW)
    keys, vals = u.lists()
    assert np.array_equal(keys, pix_ids.astype(np.uint32))
    assert np.array_equal(vals, pts.astype(np.uint32))
    rng = np.random.default_rng(3)
    W, H = v.camera.width, v.camera.height
    pix = rng.choice(W * H, 2000, replace=False)
    fb = torch.from_numpy(v.feat).to(torch.bfloat16).float().numpy()
    ref = oracle.render(v.xyz, v.opacity, fb, v.camera, pix=pix, **KW)
    _check_image(u, ref, pix)
    _, last = u.pixel_state()
    assert np.array_equal(last[pix], ref["last_pos"].astype(np.uint32))


def test_key64_bounded_wait_runs_out_and_is_reported():
    v = scenes.random_small_view(33, 20000, 96, 64)
    u = Untiled(v, flags=rast.FLAG_TEST_SORT_STALL, ws_fill=0xFF)
    assert u.status == rast.RAST_ERR_TIMEOUT
    F, A, D = u.image()
    assert np.all(F == 0) and np.all(A == 0) and np.all(D == 0)


def test_key64_rejects_gaussian():
    v = case_view("gauss")
    pts = rast.make_points(torch.from_numpy(v.xyz).to(DEV), torch.from_numpy(v.opacity).to(DEV),
                           torch.from_numpy(v.feat).to(DEV), torch.from_numpy(v.scale).to(DEV))
    cam = rast.make_camera(v.camera)
    L = rast.load_library()
    o = rast.make_opts(mode="gaussian")
    assert L.rasterize_untiled64_workspace_size(rast.ct.byref(pts), rast.ct.byref(cam), rast.ct.byref(o)) == 0
