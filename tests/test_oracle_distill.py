"""Pins for the distillation oracle: gradients by finite differences, tangents
against the reverse-mode input gradient, Adam's closed-form steps, surface areas."""
import math

import numpy as np

from oracle import distill, mlp


def _net(rng, hidden=8, latent=4):
    dims = [3 + latent, hidden, hidden, hidden, hidden, 1]
    return [(rng.normal(0, 1 / math.sqrt(a), (b, a)), rng.normal(0, 0.3, b)) for a, b in zip(dims[:-1], dims[1:])]


def test_tangents_equal_reverse_mode_input_gradient():
    rng = np.random.default_rng(0)
    layers = _net(rng)
    P = rng.normal(0, 0.5, (9, 3))
    z = rng.normal(0, 1, 4)
    s, g, _ = distill.forward_tangents(layers, P, z, beta=7.0)
    x = np.concatenate([P, np.tile(z, (9, 1))], axis=1)
    np.testing.assert_allclose(s, mlp.forward(layers, x, beta=7.0), rtol=1e-13)
    np.testing.assert_allclose(g, mlp.input_gradient(layers, x, beta=7.0)[:, :3], rtol=1e-12, atol=1e-14)


def test_parameter_gradients_match_central_differences():
    rng = np.random.default_rng(1)
    beta = 5.0                               # smooth enough for differences of the Eikonal term
    layers = _net(rng)
    P = rng.normal(0, 0.7, (11, 3))
    z = rng.normal(0, 1, 4)
    s0, _, _ = distill.forward_tangents(layers, P, z, beta)
    target = s0 + np.where(rng.random(11) < 0.5, -1.0, 1.0)   # away from the L1 kink
    loss, grads = distill.loss_and_grads(layers, P, z, target, lam_e=0.3, beta=beta)

    def L(ls):
        s, g, _ = distill.forward_tangents(ls, P, z, beta)
        return distill.loss_value(s, g, target, 0.3)

    assert abs(L(layers) - loss) < 1e-14
    e = 1e-6
    for li, (W, b) in enumerate(layers):
        for which, arr in ((0, W), (1, b)):
            idx = [tuple(rng.integers(0, n) for n in arr.shape) for _ in range(6)]
            for ix in idx:
                plus = [(w.copy(), c.copy()) for w, c in layers]
                minus = [(w.copy(), c.copy()) for w, c in layers]
                plus[li][which][ix] += e
                minus[li][which][ix] -= e
                fd = (L(plus) - L(minus)) / (2 * e)
                got = grads[li][which][ix]
                assert abs(got - fd) <= 1e-6 * max(1.0, abs(fd)), (li, which, ix, got, fd)


def test_adam_first_steps_closed_form():
    g = np.array([0.3, -2.0, 1e-3])
    p, m, v = distill.adam_update(np.zeros(3), g, np.zeros(3), np.zeros(3), t=1, lr=0.01)
    np.testing.assert_allclose(p, -0.01 * g / (np.abs(g) + 1e-8), rtol=1e-12)
    # constant gradient: the bias-corrected moments are g and g^2 at every step
    p2, _, _ = distill.adam_update(p, g, m, v, t=2, lr=0.01)
    np.testing.assert_allclose(p2 - p, -0.01 * g / (np.abs(g) + 1e-8), rtol=1e-12)


def test_surface_areas_and_targets():
    a = distill.surface_areas()
    assert abs(a["faces"] - 2.5) < 1e-12 and abs(a["outer"] - 1.2) < 1e-12 and abs(a["inner"] - 0.8) < 1e-12
    np.testing.assert_allclose(distill.targets(np.array([[0.0, 0.0, 0.0], [0.0, 0.6, 0.0]])), [0.5, -0.1], atol=1e-12)
