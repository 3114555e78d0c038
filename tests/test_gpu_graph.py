"""GPU parity of the batched path as the benchmark times it: one CUDA graph
that holds a whole rasterize_batch forward + backward over several views of
uneven size and point count (BF16 features, C = 8, 8x8 tiles, blend depth 64).

The graph is captured once and replayed twice; every replay must reproduce the
eager call's images, per-pixel state and gradients bit for bit (the graph
replays the same kernels on the same buffers, with no host work in between),
and the images and gradients must equal the FP64 oracle fed the same BF16
features within the parity tolerances. Outputs are poisoned with NaN before
each replay so a stage the graph failed to record would show."""
import numpy as np
import pytest
import torch

import oracle
from paper_2508_19140_gb300 import rast, scenes

from gpu_util import DEV, bf16_round, to_dev

pytestmark = pytest.mark.gpu

TILE, DEPTH, C = 8, 64, 8


@pytest.fixture(scope="module", autouse=True)
def _need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2508_19140_gb300 import build
    build.build()
    oracle.build()


def _views():
    shapes = [(3000, 72, 40), (9000, 130, 90), (500, 33, 17), (6000, 96, 64)]
    return [scenes.random_small_view(60 + k, n, W, H, c=C) for k, (n, W, H) in enumerate(shapes)]


class Batch:
    """Device tensors and C-ABI views of a batch; outputs kept addressable so
    a captured graph writes into them on every replay."""

    def __init__(self, views, opts):
        self.views, self.opts = views, opts
        self.t, self.cv = [], []
        for v in views:
            n = len(v.xyz)
            H, W = v.camera.height, v.camera.width
            t = dict(xyz=to_dev(v.xyz), op=to_dev(v.opacity), feat=to_dev(v.feat, torch.bfloat16),
                     gF=to_dev(v.g_feat), gA=to_dev(v.g_alpha), gD=to_dev(v.g_depth),
                     F=torch.empty((H, W, C), device=DEV), A=torch.empty((H, W), device=DEV),
                     D=torch.empty((H, W), device=DEV), d_feat=torch.empty((n, C), device=DEV),
                     d_op=torch.empty((n,), device=DEV))
            cv = rast.View()
            cv.pts = rast.make_points(t["xyz"], t["op"], t["feat"])
            cv.cam = rast.make_camera(v.camera)
            cv.out = rast.make_images(t["F"], t["A"], t["D"])
            cv.grad = rast.make_grads(t["gF"], t["gA"], t["gD"], t["d_feat"], t["d_op"])
            self.t.append(t)
            self.cv.append(cv)
        self.ws = torch.empty(rast.rasterize_workspace_size(self.cv, opts), dtype=torch.uint8, device=DEV)
        self.layout = rast.rasterize_workspace_layout(self.cv, opts)

    def poison(self):
        for t in self.t:
            for k in ("F", "A", "D", "d_feat", "d_op"):
                t[k].fill_(float("nan"))

    def outputs(self):
        out = []
        for t in self.t:
            out.append({k: t[k].cpu().numpy().copy() for k in ("F", "A", "D", "d_feat", "d_op")})
        state = {}
        for name in ("t_final", "last"):
            off, nb = self.layout[name]
            state[name] = self.ws[off: off + nb].cpu().numpy().copy()
        return out, state


def _same(a, b):
    return np.array_equal(np.asarray(a).view(np.uint32), np.asarray(b).view(np.uint32))


def test_graph_replay_bit_identical_to_eager_and_matches_oracle():
    views = _views()
    opts = rast.make_opts(tile=TILE, blend_depth=DEPTH)
    both = rast.PASS_FWD | rast.PASS_BWD

    eager = Batch(views, opts)
    eager.poison()
    rast.rasterize_batch(eager.cv, both, opts, eager.ws)
    st, stats = rast.rasterize_get_status(eager.ws)
    assert st == rast.RAST_OK, stats
    ref_out, ref_state = eager.outputs()

    g = Batch(views, opts)
    stream = torch.cuda.Stream(DEV)
    stream.wait_stream(torch.cuda.current_stream(DEV))
    with torch.cuda.stream(stream):
        rast.rasterize_batch(g.cv, both, opts, g.ws, stream)  # warm-up outside capture
    torch.cuda.current_stream(DEV).wait_stream(stream)
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=stream):
        rast.rasterize_batch(g.cv, both, opts, g.ws, torch.cuda.current_stream(DEV))
    torch.cuda.synchronize()
    for _ in range(2):
        g.poison()
        graph.replay()
        torch.cuda.synchronize()
        st, _ = rast.rasterize_get_status(g.ws)
        assert st == rast.RAST_OK
        out, state = g.outputs()
        for k in range(len(views)):
            for key in ref_out[k]:
                assert _same(out[k][key], ref_out[k][key]), (k, key)
        for key in ref_state:
            assert np.array_equal(state[key], ref_state[key]), key

    kw = dict(mode="bilinear", tile=TILE, pin32=True)
    for k, v in enumerate(views):
        fb = bf16_round(v.feat)
        ref = oracle.render(v.xyz, v.opacity, fb, v.camera, **kw)
        np.testing.assert_allclose(out[k]["F"], ref["F"], rtol=1e-5, atol=1e-7)
        np.testing.assert_allclose(out[k]["A"], ref["alpha"], rtol=1e-5, atol=1e-7)
        np.testing.assert_allclose(out[k]["D"], ref["depth"], rtol=1e-5, atol=1e-6)
        gr = oracle.backward(v.xyz, v.opacity, fb, v.camera, v.g_feat, v.g_alpha, v.g_depth, **kw)
        for key, want in (("d_feat", gr["d_feat"]), ("d_op", gr["d_opacity"])):
            got = out[k][key].astype(np.float64)
            assert np.linalg.norm(got - want) / max(np.linalg.norm(want), 1e-30) <= 1e-5, (k, key)
            assert np.all(np.abs(got - want) <= 1e-4 * np.abs(want) + 1e-6 * np.abs(want).max()), (k, key)
