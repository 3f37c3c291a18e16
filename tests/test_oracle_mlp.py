"""Pins for the CPU reference of the learned cost model."""
import numpy as np
import pytest

import graphgen
import oracle as O
from oracle import mlp


@pytest.mark.parametrize("H", [1, 4, 16])
def test_gradient_matches_finite_differences(H):
    rng = np.random.default_rng(H)
    p = rng.normal(0, 0.5, mlp.n_params(H))
    X = rng.normal(0, 1, (37, 8))
    t = rng.normal(0, 1, 37)
    loss, g = mlp.loss_grad(p, X, t, H)
    eps = 1e-6
    num = np.zeros_like(p)
    for i in range(len(p)):
        e = np.zeros_like(p)
        e[i] = eps
        num[i] = (mlp.loss_grad(p + e, X, t, H)[0] - mlp.loss_grad(p - e, X, t, H)[0]) / (2 * eps)
    assert np.allclose(g, num, rtol=1e-5, atol=1e-7)
    assert loss == pytest.approx(np.mean((mlp.forward(p, X, H) - t) ** 2))


def test_linear_regime_closed_form():
    """With positive weights and inputs the ReLUs pass everything: the network
    is the product of its affine maps."""
    H = 3
    rng = np.random.default_rng(0)
    p = np.abs(rng.normal(0, 1, mlp.n_params(H)))
    X = np.abs(rng.normal(0, 1, (5, 8)))
    W1, b1, W2, b2, w3, b3 = mlp.unpack(p, H)
    expect = ((X @ W1.T + b1) @ W2.T + b2) @ w3 + b3
    assert np.allclose(mlp.forward(p, X, H), expect)


def test_features_small_graph():
    # triangle 0-1-2 plus pendant 3 on vertex 0, isolated 4
    g = O.Graph(5, np.array([0, 1, 2, 0], np.int32), np.array([1, 2, 0, 3], np.int32))
    F = mlp.features(g)
    assert np.allclose(F[:, 0], np.log1p([3, 2, 2, 1, 0]))
    assert np.allclose(F[:, 1], [2, 2, 2, 1, 0])
    assert np.allclose(F[:, 2], np.log1p([1, 1, 1, 0, 0]))
    assert F[0, 7] == pytest.approx(2 * 1 / (3 * 2)) and F[1, 7] == pytest.approx(1.0) and F[3, 7] == 0
    assert F[3, 3] == pytest.approx(np.log1p(3)) and F[3, 4] == pytest.approx(0.0)
    assert F[4].tolist()[3:7] == [0, 0, 0, 0]
    # vertex 1's neighbours 0 (degree 3) and 2 (degree 2, higher id): both rank above it
    assert F[1, 6] == pytest.approx(np.log1p(2))


def test_features_er_shapes():
    u, v = graphgen.er(200, 0.05, 3)
    g = O.Graph(200, u, v)
    F = mlp.features(g)
    assert F.shape == (200, 8) and np.isfinite(F).all()
    assert (F[:, 7] >= 0).all() and (F[:, 7] <= 1).all()


def test_light_features_closed_forms():
    """One-pass features on a star K_{1,4} (centre 0) and a triangle."""
    import oracle as O
    from oracle import mlp
    g = O.Graph(5, np.zeros(4, np.int32), np.arange(1, 5, dtype=np.int32))
    F = mlp.features_light(g)
    # centre: d = 4, every neighbour has degree 1 (lower degree rank)
    assert np.allclose(F[0], [np.log1p(4), np.log1p(1), 0, np.log1p(1), 0, np.log1p(4 * 1 / 2), 0, np.log1p(4)])
    # leaf: d = 1, its one neighbour has degree 4 (higher)
    assert np.allclose(F[1], [np.log1p(1), np.log1p(4), 0, np.log1p(4), np.log1p(1), np.log1p(0.5), 1.0,
                              np.log1p(4)])
    t = O.Graph(3, np.array([0, 1, 0], np.int32), np.array([1, 2, 2], np.int32))
    Ft = mlp.features_light(t)
    # equal degrees: the higher id ranks higher, so vertex 0 has 2 higher neighbours, vertex 2 none
    assert np.allclose(Ft[:, 4], np.log1p([2, 1, 0])) and np.allclose(Ft[:, 6], [1.0, 0.5, 0.0])
    assert np.allclose(Ft[:, 5], np.log1p(2.0))
