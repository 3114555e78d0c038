"""The differentiable wrapper (``rast.rasterize`` / ``rast.rasterize_views``, a
torch.autograd.Function over the C ABI's forward and backward passes): the
gradients that reach the leaf tensors through ``loss.backward()`` must equal the
oracle's adjoint of the same loss (appendix, corrected Eq. 2), for bilinear and
Gaussian splats, several views in one call, upstream gradients on some outputs
only, and BF16 features; an FP32 directional finite difference of the loss
checks the wiring end to end."""
import numpy as np
import pytest
import torch

import oracle
from paper_2508_19140_gb300 import rast, scenes

from gpu_util import bf16_round

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


@pytest.fixture(scope="module", autouse=True)
def _need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2508_19140_gb300 import build
    build.build()
    oracle.build()


def _t(a, dtype=torch.float32, grad=False):
    t = torch.from_numpy(np.ascontiguousarray(a)).to(DEV, dtype)
    return t.requires_grad_(grad)


def _check(got, ref, norm=1e-5, er=1e-4, ea=1e-6, mask=None):
    g = np.asarray(got, np.float64)
    f = np.asarray(ref, np.float64)
    if mask is not None:
        g, f = g[mask], f[mask]
    assert np.linalg.norm(g - f) <= norm * max(np.linalg.norm(f), 1e-30)
    bad = np.abs(g - f) > er * np.abs(f) + ea * np.abs(f).max()
    assert not bad.any(), (np.argwhere(bad)[:5], g[bad][:5], f[bad][:5])


def _loss(out, v, use_alpha=True, use_depth=True):
    F, A, D = out
    L = (F.double() * _t(v.g_feat, torch.float64)).sum()
    if use_alpha:
        L = L + (A.double() * _t(v.g_alpha, torch.float64)).sum()
    if use_depth:
        L = L + (D.double() * _t(v.g_depth, torch.float64)).sum()
    return L


KW_B = dict(mode="bilinear", tile=16, pin32=True)


def test_bilinear_grads_reach_leaves():
    v = scenes.random_small_view(31, 5000, 100, 75, c=4)
    xyz, op, feat = _t(v.xyz, grad=True), _t(v.opacity, grad=True), _t(v.feat, grad=True)
    out = rast.rasterize(xyz, op, feat, v.camera)
    ref_img = oracle.render(v.xyz, v.opacity, v.feat, v.camera, **KW_B)
    np.testing.assert_allclose(out[0].detach().cpu().numpy(), ref_img["F"], rtol=1e-5, atol=1e-7)
    _loss(out, v).backward()
    ref = oracle.backward(v.xyz, v.opacity, v.feat, v.camera, v.g_feat, v.g_alpha, v.g_depth, **KW_B)
    _check(op.grad.cpu().numpy(), ref["d_opacity"])
    _check(feat.grad.cpu().numpy(), ref["d_feat"])
    assert xyz.grad is None  # a bilinear splat passes no gradient to positions


def test_gaussian_grads_reach_leaves():
    v = scenes.random_small_view(25, 4000, 90, 70, c=4, gaussian=True, f=80.0)
    kw = dict(mode="gaussian", gauss_cov="ewa", tile=16, pin32=True)
    xyz, op = _t(v.xyz, grad=True), _t(v.opacity, grad=True)
    feat, scale = _t(v.feat, grad=True), _t(v.scale, grad=True)
    out = rast.rasterize(xyz, op, feat, v.camera, scale=scale, mode="gaussian")
    _loss(out, v).backward()
    ref = oracle.backward(v.xyz, v.opacity, v.feat, v.camera, v.g_feat, v.g_alpha, v.g_depth,
                          scale=v.scale, **kw)
    # points touching a pixel whose termination is ambiguous in FP32 are left out
    img = oracle.render(v.xyz, v.opacity, v.feat, v.camera, scale=v.scale, **kw)
    amb = img["margin"] <= 1e-5
    p = oracle.project(v.xyz, v.camera, scale=v.scale, **kw)
    keep = np.ones(len(v.xyz), bool)
    for i in np.nonzero(p["vis"])[0]:
        x0, x1, y0, y1 = p["box"][i]
        keep[i] = not amb[y0:y1 + 1, x0:x1 + 1].any()
    _check(feat.grad.cpu().numpy(), ref["d_feat"], mask=keep)
    loose = dict(norm=1e-4, er=1e-3, ea=1e-5, mask=keep)
    _check(op.grad.cpu().numpy(), ref["d_opacity"], **loose)
    _check(xyz.grad.cpu().numpy(), ref["d_xyz"], **loose)
    _check(scale.grad.cpu().numpy(), ref["d_scale"], **loose)


def test_views_of_uneven_size_in_one_call():
    vs = [scenes.random_small_view(41, 3000, 64, 48, c=3),
          scenes.random_small_view(42, 9000, 130, 90, c=3),
          scenes.random_small_view(43, 700, 33, 17, c=3)]
    leaves = [(_t(v.xyz), _t(v.opacity, grad=True), _t(v.feat, grad=True)) for v in vs]
    outs = rast.rasterize_views([(x, o, f, v.camera) for (x, o, f), v in zip(leaves, vs)])
    sum(_loss(o, v) for o, v in zip(outs, vs)).backward()
    for (x, o, f), v in zip(leaves, vs):
        ref = oracle.backward(v.xyz, v.opacity, v.feat, v.camera, v.g_feat, v.g_alpha, v.g_depth, **KW_B)
        _check(o.grad.cpu().numpy(), ref["d_opacity"])
        _check(f.grad.cpu().numpy(), ref["d_feat"])


def test_upstream_gradient_on_features_only():
    v = scenes.random_small_view(44, 4000, 80, 60, c=2)
    op, feat = _t(v.opacity, grad=True), _t(v.feat, grad=True)
    F, A, D = rast.rasterize(_t(v.xyz), op, feat, v.camera)
    (F.double() * _t(v.g_feat, torch.float64)).sum().backward()  # alpha and depth unused
    ref = oracle.backward(v.xyz, v.opacity, v.feat, v.camera, v.g_feat, None, None, **KW_B)
    _check(op.grad.cpu().numpy(), ref["d_opacity"])
    _check(feat.grad.cpu().numpy(), ref["d_feat"])


def test_bf16_features_get_bf16_gradients():
    v = scenes.random_small_view(45, 6000, 96, 64, c=8)
    op, feat = _t(v.opacity, grad=True), _t(v.feat, torch.bfloat16, grad=True)
    out = rast.rasterize(_t(v.xyz), op, feat, v.camera)
    _loss(out, v).backward()
    assert feat.grad.dtype == torch.bfloat16
    fb = bf16_round(v.feat)
    ref = oracle.backward(v.xyz, v.opacity, fb, v.camera, v.g_feat, v.g_alpha, v.g_depth, **KW_B)
    _check(op.grad.cpu().numpy(), ref["d_opacity"])
    # dL/df is computed in FP32 and rounded once to BF16 (8 significant bits)
    _check(feat.grad.float().cpu().numpy(), ref["d_feat"], norm=4e-3, er=8e-3, ea=1e-6)


def test_directional_finite_difference():
    """Central difference of the loss along a random direction in (opacity,
    features), FP32 forward, FP64 loss; opacities kept low so that no alpha is
    clamped and no pixel terminates inside the step."""
    v = scenes.random_small_view(46, 2500, 64, 48, c=3)
    rng = np.random.default_rng(46)
    v.opacity = (0.05 + 0.4 * rng.random(len(v.xyz))).astype(np.float32)
    img = oracle.render(v.xyz, v.opacity, v.feat, v.camera, **KW_B)
    assert img["alpha"].max() < 1 - 1e-2  # transmittance stays far above the cutoff
    xyz = _t(v.xyz)
    op, feat = _t(v.opacity, grad=True), _t(v.feat, grad=True)
    _loss(rast.rasterize(xyz, op, feat, v.camera), v).backward()
    d_op = rng.uniform(-1, 1, len(v.xyz))
    d_f = rng.uniform(-1, 1, v.feat.shape)
    analytic = float((op.grad.double().cpu().numpy() * d_op).sum() + (feat.grad.double().cpu().numpy() * d_f).sum())
    h = 1e-2

    def L(s):
        o = _t(v.opacity + s * h * d_op)
        f = _t(v.feat + s * h * d_f)
        with torch.no_grad():
            return float(_loss(rast.rasterize(xyz, o, f, v.camera), v))

    fd = (L(1) - L(-1)) / (2 * h)
    assert abs(fd - analytic) <= 2e-3 * abs(analytic), (fd, analytic)
