"""Seeded synthetic workloads for the tiled point rasterizer.

This module only draws inputs: point clouds, per-point attributes, cameras and
upstream gradients. It holds none of the rasterizer's arithmetic, so both the
CUDA path and the CPU oracle may consume what it produces.

The five workloads stand in for the paper's Mip-NeRF360 / Tanks and Temples
scenes (Sec. 4: 1, 1.5 and 2 MP images; Sec. 2: 8 M training samples per
iteration, 33 M pre-extracted points, four features per point). Every array
comes from ``numpy.random.default_rng(1000 + config_id)`` unless a seed is
given.

Camera convention: x_c = R @ x_w + t, camera looks down +z, pixel (i, j) has
its centre at (i + 0.5, j + 0.5), u = fx * x_c / z_c + cx.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

NEAR = 0.2
FAR = 1.0e4


@dataclass
class Camera:
    fx: float
    fy: float
    cx: float
    cy: float
    R: np.ndarray  # (3, 3) float32, row-major, world -> camera
    t: np.ndarray  # (3,) float32
    width: int
    height: int
    near: float = NEAR
    far: float = FAR


@dataclass
class View:
    """One view: its own point cloud, camera and upstream gradients."""
    xyz: np.ndarray            # (N, 3) float32
    opacity: np.ndarray        # (N,) float32
    feat: np.ndarray           # (N, C) float32 (rounded to bf16 later if asked)
    camera: Camera
    scale: np.ndarray | None = None    # (N,) float32, Gaussian mode only
    g_feat: np.ndarray | None = None   # (H, W, C) float32 upstream dL/dF
    g_alpha: np.ndarray | None = None  # (H, W) float32
    g_depth: np.ndarray | None = None  # (H, W) float32


@dataclass
class Scene:
    config_id: int
    name: str
    mode: str                  # "bilinear" or "gaussian"
    feat_dtype: str            # "f32" or "bf16"
    views: list = field(default_factory=list)
    backward: bool = True


def look_at(eye, target=(0.0, 0.0, 0.0), up=(0.0, -1.0, 0.0)):
    """World->camera rotation and translation for a camera at ``eye``
    looking at ``target`` (camera +z forward, +x right, +y down)."""
    eye = np.asarray(eye, np.float64)
    fwd = np.asarray(target, np.float64) - eye
    fwd /= np.linalg.norm(fwd)
    right = np.cross(fwd, np.asarray(up, np.float64))
    right /= np.linalg.norm(right)
    down = np.cross(fwd, right)
    R = np.stack([right, down, fwd]).astype(np.float32)
    t = (-R.astype(np.float64) @ eye).astype(np.float32)
    return R, t


def orbit_camera(width, height, distance, yaw_deg, pitch_deg, f=None):
    yaw, pitch = math.radians(yaw_deg), math.radians(pitch_deg)
    eye = (distance * math.sin(yaw) * math.cos(pitch),
           -distance * math.sin(pitch),
           -distance * math.cos(yaw) * math.cos(pitch))
    R, t = look_at(eye)
    if f is None:
        f = 0.866 * width  # 60 degree horizontal field of view
    return Camera(fx=float(f), fy=float(f), cx=width / 2.0, cy=height / 2.0,
                  R=R, t=t, width=int(width), height=int(height))


def identity_camera(width, height, f):
    return Camera(fx=float(f), fy=float(f), cx=width / 2.0, cy=height / 2.0,
                  R=np.eye(3, dtype=np.float32), t=np.zeros(3, np.float32),
                  width=int(width), height=int(height))


def random_rotations(rng, k):
    q, r = np.linalg.qr(rng.standard_normal((k, 3, 3)))
    q *= np.sign(np.diagonal(r, axis1=1, axis2=2))[:, None, :]
    return q


def clustered_points(rng, n, n_clusters=64, bg_frac=0.10, extent=2.0):
    """Mixture of anisotropic 3D Gaussian clusters plus a uniform background."""
    n_bg = int(round(n * bg_frac))
    n_cl = n - n_bg
    centres = rng.uniform(-1.5, 1.5, (n_clusters, 3))
    sig = rng.uniform(0.02, 0.3, (n_clusters, 3))
    rot = random_rotations(rng, n_clusters)
    which = rng.integers(0, n_clusters, n_cl)
    local = rng.standard_normal((n_cl, 3), dtype=np.float32) * sig[which].astype(np.float32)
    pts = np.einsum("nij,nj->ni", rot[which].astype(np.float32), local) + centres[which].astype(np.float32)
    bg = rng.uniform(-extent, extent, (n_bg, 3)).astype(np.float32)
    xyz = np.concatenate([pts.astype(np.float32), bg], axis=0)
    perm = rng.permutation(n)
    return np.ascontiguousarray(xyz[perm])


def _attrs(rng, n, c, beta=True):
    if beta:
        o = rng.beta(2.0, 2.0, n).astype(np.float32)
    else:
        o = rng.uniform(0.05, 0.95, n).astype(np.float32)
    f = rng.random((n, c), dtype=np.float32)
    return o, f


def _grads(rng, cam, c):
    h, w = cam.height, cam.width
    return (rng.standard_normal((h, w, c), dtype=np.float32),
            rng.standard_normal((h, w), dtype=np.float32),
            rng.standard_normal((h, w), dtype=np.float32))


def tiny_scene(seed=1001, n=20000, width=128, height=128, f=128.0, c=4):
    """Config 1: points uniform in a unit cube at z in [2, 4], identity camera."""
    rng = np.random.default_rng(seed)
    xyz = np.stack([rng.uniform(-0.5, 0.5, n), rng.uniform(-0.5, 0.5, n),
                    rng.uniform(2.0, 4.0, n)], axis=1).astype(np.float32)
    o, feat = _attrs(rng, n, c, beta=False)
    cam = identity_camera(width, height, f)
    gf, ga, gd = _grads(rng, cam, c)
    return View(xyz=xyz, opacity=o, feat=feat, camera=cam, g_feat=gf, g_alpha=ga, g_depth=gd)


def clustered_view(rng, n, width, height, distance, yaw, pitch, c, f=None):
    xyz = clustered_points(rng, n)
    o, feat = _attrs(rng, n, c, beta=True)
    cam = orbit_camera(width, height, distance, yaw, pitch, f)
    gf, ga, gd = _grads(rng, cam, c)
    return View(xyz=xyz, opacity=o, feat=feat, camera=cam, g_feat=gf, g_alpha=ga, g_depth=gd)


def gaussian_view(rng, n, width=1920, height=1080, distance=5.0, c=4, f=1000.0,
                  zmin=1.9, zmax=10.0):
    """Config 4: clustered points rejection-sampled to z_c in [zmin, zmax],
    world scale ~ logU(1e-3, 1e-2)."""
    cam = orbit_camera(width, height, distance, 20.0, 10.0, f)
    R = cam.R.astype(np.float64)
    t = cam.t.astype(np.float64)
    keep = []
    have = 0
    while have < n:
        cand = clustered_points(rng, max(n // 2, 1024))
        zc = cand.astype(np.float64) @ R[2] + t[2]
        ok = cand[(zc >= zmin) & (zc <= zmax)]
        keep.append(ok)
        have += len(ok)
    xyz = np.ascontiguousarray(np.concatenate(keep)[:n])
    o, feat = _attrs(rng, n, c, beta=True)
    scale = np.exp(rng.uniform(math.log(1e-3), math.log(1e-2), n)).astype(np.float32)
    gf, ga, gd = _grads(rng, cam, c)
    return View(xyz=xyz, opacity=o, feat=feat, camera=cam, scale=scale,
                g_feat=gf, g_alpha=ga, g_depth=gd)


BATCH_VIEWS = [(640, 480, 1 << 20), (800, 600, 1 << 21), (1024, 768, 1 << 22),
               (1280, 720, 1 << 22), (1280, 832, 1 << 23), (1600, 900, 1 << 23),
               (1920, 1080, 1 << 24), (1920, 1080, 1 << 24)]


def make_scene(config_id: int, seed: int | None = None, scale_points: float = 1.0) -> Scene:
    """Build one of the five synthetic workloads.

    ``scale_points`` shrinks the point counts (never the images) for quick runs;
    1.0 gives the full workload.
    """
    if seed is None:
        seed = 1000 + config_id
    rng = np.random.default_rng(seed)

    def npts(n):
        return max(1, int(n * scale_points))

    if config_id == 1:
        v = tiny_scene(seed=seed, n=npts(20000))
        # the tiny workload is a plain forward (its views still carry upstream
        # gradients for the backward parity tests)
        return Scene(1, "tiny-128x128-20k-bilinear-f32", "bilinear", "f32", [v], backward=False)
    if config_id == 2:
        v = clustered_view(rng, npts(1 << 22), 1280, 832, 6.0, 30.0, 15.0, 4)
        return Scene(2, "train-4M-1280x832-bilinear-f32", "bilinear", "f32", [v], backward=True)
    if config_id == 3:
        v = clustered_view(rng, npts(1 << 25), 1920, 1080, 6.0, 0.0, 0.0, 4)
        return Scene(3, "infer-32M-1920x1080-bilinear-f32", "bilinear", "f32", [v], backward=False)
    if config_id == 4:
        v = gaussian_view(rng, npts(1 << 24))
        return Scene(4, "gauss-16M-1920x1080-ewa-bf16", "gaussian", "bf16", [v], backward=True)
    if config_id == 5:
        views = []
        for k, (w, h, n) in enumerate(BATCH_VIEWS):
            views.append(clustered_view(rng, npts(n), w, h, 6.0, 45.0 * k, 15.0, 8))
        return Scene(5, "batch-8views-1M-16M-bilinear-bf16", "bilinear", "bf16", views, backward=True)
    raise ValueError(f"unknown config {config_id}")


def random_small_view(seed, n, width, height, c=4, gaussian=False, f=None,
                      zrange=(1.5, 4.0)):
    """Small random view for parity tests: points spread over the frustum,
    including some off-screen and some behind the near plane."""
    rng = np.random.default_rng(seed)
    if f is None:
        f = 0.9 * width
    z = rng.uniform(zrange[0], zrange[1], n)
    x = (rng.uniform(-0.6, 0.6, n) * width / f) * z
    y = (rng.uniform(-0.6, 0.6, n) * height / f) * z
    xyz = np.stack([x, y, z], 1).astype(np.float32)
    # a few culled points: behind the camera, inside the near plane, beyond far
    k = max(1, n // 50)
    xyz[:k, 2] = -1.0
    xyz[k:2 * k, 2] = 0.1
    o, feat = _attrs(rng, n, c, beta=True)
    cam = identity_camera(width, height, f)
    scale = None
    if gaussian:
        scale = np.exp(rng.uniform(math.log(2e-3), math.log(2e-2), n)).astype(np.float32)
    gf, ga, gd = _grads(rng, cam, c)
    return View(xyz=xyz, opacity=o, feat=feat, camera=cam, scale=scale,
                g_feat=gf, g_alpha=ga, g_depth=gd)


def env_map(seed=2001, height=1024, width=2048, c=4, kind="smooth"):
    """Synthetic stand-in for the distilled spherical background map
    (H_b x W_b x C FP32; the paper's map is 1024 x 2048 x 4).

    kind="smooth": a low-frequency field (sky-like: a vertical gradient plus a
    few long-wavelength waves in longitude and polar angle), values in
    (0.05, 0.95); kind="noise": i.i.d. U(0, 1) texels (worst case for
    interpolation error)."""
    rng = np.random.default_rng(seed)
    if kind == "noise":
        return rng.uniform(0.0, 1.0, (height, width, c)).astype(np.float32)
    lam = (np.arange(width) + 0.5) / width * 2.0 * np.pi - np.pi
    th = (np.arange(height) + 0.5) / height * np.pi
    L, TH = np.meshgrid(lam, th)
    out = np.empty((height, width, c), np.float64)
    for ch in range(c):
        k = rng.integers(1, 4, 3)
        ph = rng.uniform(0, 2 * np.pi, 3)
        v = 0.5 + 0.25 * np.cos(TH + ph[0])
        v += 0.1 * np.cos(k[0] * L + ph[1]) * np.sin(TH)
        v += 0.05 * np.cos(k[1] * L + k[2] * TH + ph[2])
        out[..., ch] = v
    return np.clip(out, 0.05, 0.95).astype(np.float32)
