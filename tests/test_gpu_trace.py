"""The per-tile trace the bilinear blend kernels leave in the workspace
("tile_trace": per tile and pass, the globaltimer at the CTA's start and end,
its clock64 cycles and the SM it ran on): every tile of a forward + backward
pair has a complete, ordered record, and the backward ran after the forward."""
import numpy as np
import pytest
import torch

from paper_2508_19140_gb300 import scenes

from gpu_util import Run, tile_offsets

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2508_19140_gb300 import build
    build.build()


@pytest.mark.parametrize("tile,depth", [(16, 0), (8, 64)])
def test_every_tile_has_an_ordered_trace(tile, depth):
    views = [scenes.random_small_view(71, 6000, 100, 75, c=4), scenes.random_small_view(72, 2000, 37, 29, c=4)]
    r = Run(views, backward=True, tile=tile, blend_depth=depth)
    assert r.status == 0
    P = tile_offsets(views, tile)[-1]
    tr = r.arr("tile_trace", np.uint64, P * 2 * 4).reshape(P, 2, 4)
    start, end, cycles, sm = tr[..., 0], tr[..., 1], tr[..., 2], tr[..., 3]
    n_sm = torch.cuda.get_device_properties(0).multi_processor_count
    assert np.all(start > 0) and np.all(end >= start)
    assert np.all(cycles > 0) and np.all(sm < n_sm)
    assert end[:, 0].max() <= start[:, 1].min()  # the backward launch follows the forward
