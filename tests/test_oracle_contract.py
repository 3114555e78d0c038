"""CPU pins of the contraction oracle (Mip-NeRF 360 spherical contraction,
applied to the sampled positions; fused into one kernel in Sec. 3.4)."""
import numpy as np
import pytest

import oracle


@pytest.fixture(scope="module", autouse=True)
def _build():
    oracle.build()


def test_identity_inside_unit_ball():
    rng = np.random.default_rng(0)
    x = rng.uniform(-1, 1, (1000, 3))
    x = x[np.linalg.norm(x, axis=1) <= 1]
    assert np.array_equal(oracle.contract(x), x)


def test_radial_closed_form_outside():
    rng = np.random.default_rng(1)
    d = rng.standard_normal((500, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    r = np.exp(rng.uniform(0, 8, 500))           # radii 1 .. e^8
    y = oracle.contract(d * r[:, None])
    # direction kept, radius 2 - 1/r
    np.testing.assert_allclose(np.linalg.norm(y, axis=1), 2 - 1 / r, rtol=1e-13)
    np.testing.assert_allclose(y / np.linalg.norm(y, axis=1, keepdims=True), d, atol=1e-13)


def test_continuous_at_the_sphere_and_bounded():
    e = np.array([[1.0, 0, 0], [0, 1 + 1e-12, 0], [0, 0, -(1 - 1e-12)]])
    np.testing.assert_allclose(np.linalg.norm(oracle.contract(e), axis=1), 1.0, atol=2e-12)
    far = oracle.contract(np.array([[1e30, 0, 0], [0, -1e15, 1e15]]))
    assert np.all(np.linalg.norm(far, axis=1) < 2.0)
    assert np.array_equal(oracle.contract(np.zeros((1, 3))), np.zeros((1, 3)))
