"""Pins for the Gate-SDF MLP: hand-computed nets, softplus limits, a float64 library run."""
import math

import numpy as np
import pytest

from oracle import mlp


def test_softplus_limits_and_values():
    b = 100.0
    assert abs(mlp.softplus(np.float64(0.0), b) - math.log(2.0) / b) < 1e-15
    assert mlp.softplus(np.float64(5.0), b) == 5.0 + math.log1p(math.exp(-500.0)) / b
    assert 0.0 < mlp.softplus(np.float64(-5.0), b) < 1e-200
    x = np.linspace(-0.05, 0.05, 11)
    np.testing.assert_allclose(mlp.softplus(x, b), np.log1p(np.exp(b * x)) / b, rtol=1e-14)
    np.testing.assert_allclose(mlp.softplus_grad(x, b), 1.0 / (1.0 + np.exp(-b * x)), rtol=1e-14)


def test_one_hidden_unit_by_hand():
    # in=2 -> 1 hidden unit -> 1 output, beta = 1 so the numbers are easy
    layers = [(np.array([[1.0, 2.0]]), np.array([0.5])), (np.array([[3.0]]), np.array([-1.0]))]
    x = np.array([[0.25, -0.5]])         # pre-activation 0.25 - 1 + 0.5 = -0.25
    expect = 3.0 * math.log(1.0 + math.exp(-0.25)) - 1.0
    assert abs(mlp.forward(layers, x, beta=1.0)[0] - expect) < 1e-15
    g = mlp.input_gradient(layers, x, beta=1.0)
    sig = 1.0 / (1.0 + math.exp(0.25))
    np.testing.assert_allclose(g[0], [3.0 * sig * 1.0, 3.0 * sig * 2.0], rtol=1e-14)


def _random_net(rng, dims):
    return [(rng.normal(0, 1 / math.sqrt(a), (b, a)), rng.normal(0, 0.1, b)) for a, b in zip(dims[:-1], dims[1:])]


def test_forward_matches_torch_float64():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(0)
    dims = [67, 128, 128, 128, 128, 1]
    layers = _random_net(rng, dims)
    x = rng.normal(0, 1, (300, 67))
    h = torch.tensor(x, dtype=torch.float64)
    for i, (W, b) in enumerate(layers):
        h = torch.nn.functional.linear(h, torch.tensor(W), torch.tensor(b))
        if i < len(layers) - 1:
            h = torch.nn.functional.softplus(h, beta=100.0, threshold=1e9)
    np.testing.assert_allclose(mlp.forward(layers, x), h[:, 0].numpy(), rtol=1e-12, atol=1e-12)


def test_sdf_concatenates_point_then_latent():
    rng = np.random.default_rng(1)
    layers = _random_net(rng, [5, 4, 1])
    pg = rng.normal(size=(7, 3))
    z = rng.normal(size=2)
    x = np.concatenate([pg, np.tile(z, (7, 1))], axis=1)
    np.testing.assert_array_equal(mlp.sdf(layers, pg, z), mlp.forward(layers, x))


def test_input_gradient_central_differences():
    rng = np.random.default_rng(2)
    layers = _random_net(rng, [6, 16, 16, 1])
    x = rng.normal(0, 0.05, (20, 6))
    g = mlp.input_gradient(layers, x)
    e = 1e-6
    fd = np.stack([(mlp.forward(layers, x + e * np.eye(6)[i]) - mlp.forward(layers, x - e * np.eye(6)[i])) / (2 * e)
                   for i in range(6)], axis=1)
    np.testing.assert_allclose(g, fd, rtol=1e-5, atol=1e-7)


def test_positional_encoding_closed_forms():
    from oracle import mlp as M
    p = np.array([[0.25, -0.5, 1.0]])
    f = M.positional_encoding(p, 2)
    assert f.shape == (1, 15)
    np.testing.assert_allclose(f[0, 0:3], p[0])
    np.testing.assert_allclose(f[0, 3:6], [np.sin(np.pi / 4), -1.0, 0.0], atol=1e-15)       # sin(pi p)
    np.testing.assert_allclose(f[0, 6:9], [np.cos(np.pi / 4), 0.0, -1.0], atol=1e-15)       # cos(pi p)
    np.testing.assert_allclose(f[0, 9:12], [1.0, 0.0, 0.0], atol=1e-15)                     # sin(2 pi p)
    np.testing.assert_allclose(f[0, 12:15], [0.0, -1.0, 1.0], atol=1e-15)                   # cos(2 pi p)
    np.testing.assert_array_equal(M.positional_encoding(p, 0), p)


def test_sdf_with_positional_encoding_is_the_mlp_of_the_encoded_point():
    import workloads as W
    from oracle import mlp as M
    layers = W.xavier_mlp(5, in_dim=3 + 6 * 3 + 64)
    rng = np.random.default_rng(1)
    pg, z = rng.normal(size=(7, 3)), rng.normal(size=64)
    x = np.concatenate([M.positional_encoding(pg, 3), np.tile(z, (7, 1))], axis=1)
    np.testing.assert_allclose(M.sdf(layers, pg, z, pe_levels=3), M.forward(layers, x), rtol=1e-15)
