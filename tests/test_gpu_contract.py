"""GPU parity of the fused spherical contraction (Sec. 3.4) against the FP64
oracle: IEEE-rounded FP32 operations, so each coordinate is within a few ulp
(4e-7 relative + 1e-30 absolute)."""
import numpy as np
import pytest
import torch

import oracle
from paper_2508_19140_gb300 import rast

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


@pytest.fixture(scope="module", autouse=True)
def _need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2508_19140_gb300 import build
    build.build()
    oracle.build()


def _points(n, seed):
    rng = np.random.default_rng(seed)
    d = rng.standard_normal((n, 3))
    d /= np.maximum(np.linalg.norm(d, axis=1, keepdims=True), 1e-30)
    r = np.exp(rng.uniform(-4, 12, n))
    return (d * r[:, None]).astype(np.float32)


@pytest.mark.parametrize("n", [0, 1, 3, 4, 7, 1000, 1 << 20, (1 << 20) + 5])
def test_contract_matches_oracle(n):
    x = _points(n, n)
    xd = torch.from_numpy(x).to(DEV)
    out = torch.empty_like(xd)
    rast.rasterize_contract(xd, out)
    got = out.cpu().numpy()
    ref = oracle.contract(x.astype(np.float64)) if n else np.zeros((0, 3))
    np.testing.assert_allclose(got, ref, rtol=4e-7, atol=1e-30)
    if n:
        assert np.all(np.linalg.norm(got.astype(np.float64), axis=1) < 2.0 + 1e-6)


def test_in_place_unaligned_and_edges():
    x = np.array([[0, 0, 0], [1, 0, 0], [0.6, 0.8, 0], [3e38, 0, 0], [-1e-30, 2, -2], [0.5, 0.5, 0.5]],
                 np.float32)
    big = torch.zeros((x.shape[0] * 3 + 1,), device=DEV)
    view = big[1:].view(-1, 3)               # 4-byte offset: scalar path
    view.copy_(torch.from_numpy(x).to(DEV))
    rast.rasterize_contract(view, view)
    got = view.cpu().numpy()
    ref = oracle.contract(x.astype(np.float64))
    np.testing.assert_allclose(got, ref, rtol=4e-7, atol=1e-30)
    assert np.array_equal(got[:2], x[:2])    # on or inside the unit sphere: unchanged
