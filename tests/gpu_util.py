"""Helpers for the GPU parity tests: run a view through the C ABI (via the
thin binding) and read the workspace arrays the kernels produced."""
import numpy as np
import torch

from paper_2508_19140_gb300 import rast

DEV = "cuda:0"


def to_dev(a, dtype=torch.float32):
    return None if a is None else torch.from_numpy(np.ascontiguousarray(a)).to(DEV, dtype)


class Run:
    """Forward (and optionally backward) of one or several views."""

    def __init__(self, views, mode="bilinear", bf16=False, gauss_cov="ewa", backward=False,
                 g_alpha=True, g_depth=True, ws_fill=0, **opt_kw):
        self.views = views
        self.opts = rast.make_opts(mode=mode, gauss_cov=gauss_cov, **opt_kw)
        self.gauss = mode == "gaussian"
        self.tensors = []
        cviews = []
        for v in views:
            xyz = to_dev(v.xyz)
            op = to_dev(v.opacity)
            feat = to_dev(v.feat, torch.bfloat16 if bf16 else torch.float32)
            scale = to_dev(v.scale) if self.gauss and v.scale is not None else None
            H, W, C = v.camera.height, v.camera.width, v.feat.shape[1]
            F = torch.full((H, W, C), float("nan"), device=DEV)
            A = torch.full((H, W), float("nan"), device=DEV)
            Dp = torch.full((H, W), float("nan"), device=DEV)
            cv = rast.View()
            cv.pts = rast.make_points(xyz, op, feat, scale)
            cv.cam = rast.make_camera(v.camera)
            cv.out = rast.make_images(F, A, Dp)
            t = dict(xyz=xyz, op=op, feat=feat, scale=scale, F=F, A=A, D=Dp)
            if backward:
                n = v.xyz.shape[0]
                t["gF"] = to_dev(v.g_feat)
                t["gA"] = to_dev(v.g_alpha) if g_alpha else None
                t["gD"] = to_dev(v.g_depth) if g_depth else None
                t["d_feat"] = torch.full((n, C), float("nan"), device=DEV)
                t["d_op"] = torch.full((n,), float("nan"), device=DEV)
                t["d_xyz"] = torch.full((n, 3), float("nan"), device=DEV) if self.gauss else None
                t["d_scale"] = (torch.full((n,), float("nan"), device=DEV)
                                if self.gauss and scale is not None else None)
                cv.grad = rast.make_grads(t["gF"], t["gA"], t["gD"], t["d_feat"], t["d_op"],
                                          t["d_xyz"], t["d_scale"])
            self.tensors.append(t)
            cviews.append(cv)
        self.cviews = cviews
        self.ws_bytes = rast.rasterize_workspace_size(cviews, self.opts)
        # ws_fill: byte the workspace holds before the first call (0xFF checks
        # that no kernel reads anything it did not write in this call).
        self.ws = torch.full((self.ws_bytes,), ws_fill, dtype=torch.uint8, device=DEV)
        self.layout = rast.rasterize_workspace_layout(cviews, self.opts)
        rast.rasterize_batch(cviews, rast.PASS_FWD, self.opts, self.ws)
        self.status, self.stats = rast.rasterize_get_status(self.ws)
        if backward:
            rast.rasterize_batch(cviews, rast.PASS_BWD, self.opts, self.ws)
        torch.cuda.synchronize()

    def arr(self, name, dtype, count=None):
        off, nbytes = self.layout[name]
        item = np.dtype(dtype).itemsize
        n = nbytes // item if count is None else count
        return self.ws[off: off + n * item].cpu().numpy().view(dtype)

    def image(self, k=0):
        t = self.tensors[k]
        return t["F"].cpu().numpy(), t["A"].cpu().numpy(), t["D"].cpu().numpy()

    def grads(self, k=0):
        t = self.tensors[k]
        out = dict(d_feat=t["d_feat"].cpu().numpy(), d_opacity=t["d_op"].cpu().numpy())
        if t.get("d_xyz") is not None:
            out["d_xyz"] = t["d_xyz"].cpu().numpy()
        if t.get("d_scale") is not None:
            out["d_scale"] = t["d_scale"].cpu().numpy()
        return out

    def pixel_state(self, k=0):
        """(T_final, last) of view k."""
        off = sum(v.camera.width * v.camera.height for v in self.views[:k])
        n = self.views[k].camera.width * self.views[k].camera.height
        tf = self.arr("t_final", np.float32)[off: off + n]
        last = self.arr("last", np.uint32)[off: off + n]
        shp = (self.views[k].camera.height, self.views[k].camera.width)
        return tf.reshape(shp), last.reshape(shp)

    def sorted_copies(self):
        D = int(self.stats["n_copies"])
        keys = self.arr("sorted_keys", np.uint32, D)
        vals = self.arr("sorted_vals", np.uint32, D)
        return keys, vals

    def records(self):
        n = sum(v.xyz.shape[0] for v in self.views)
        words = self.layout["records"][1] // 4 // max(n, 1)
        return self.arr("records", np.uint32, n * words).reshape(n, words)


def tile_offsets(views, T=16):
    offs = [0]
    for v in views:
        offs.append(offs[-1] + ((v.camera.width + T - 1) // T) * ((v.camera.height + T - 1) // T))
    return offs


def bf16_round(a):
    """Round-to-nearest-even FP32 -> BF16 -> FP32 (what torch's .to(bfloat16) does)."""
    return torch.from_numpy(np.ascontiguousarray(a, np.float32)).to(torch.bfloat16).float().numpy()
