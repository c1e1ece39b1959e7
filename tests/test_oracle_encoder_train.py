"""Pins for the denoising training of the depth encoder in the oracle: the pooled target by hand,
every gradient against central differences of the loss, and Adam's first step in closed form."""
import numpy as np
import pytest

import workloads as W
from oracle import encoder_train as T


def test_pooled_target_blocks():
    img = np.arange(2 * 10 * 17, dtype=np.float64).reshape(2, 10, 17)
    t = T.pooled_target(img, 2.0)
    assert t.shape == (2, 2, 3)
    assert abs(t[0, 0, 0] - img[0, :8, :8].mean() / 2) < 1e-12
    assert abs(t[1, 1, 2] - img[1, 8:, 16:].mean() / 2) < 1e-12      # 2 x 1 edge block


def _setup(seed=0):
    rng = np.random.default_rng(seed)
    enc = [(W.astype(np.float64), b.astype(np.float64)) for W, b in W.encoder_weights(11)]
    dec = (rng.normal(0, 0.2, (6, 64)), rng.normal(0, 0.1, 6))
    clean = rng.uniform(0.5, 10.0, (2, 13, 17))
    noisy = clean + rng.normal(0, 0.3, clean.shape)
    return noisy, clean, enc, dec


def test_gradients_match_central_differences():
    noisy, clean, enc, dec = _setup()
    L, g_enc, g_dec = T.gradients(noisy, clean, 10.0, enc, dec)
    assert abs(L - T.loss(noisy, clean, 10.0, enc, dec)) < 1e-14
    rng = np.random.default_rng(1)
    h = 1e-6

    def fd(get, setter, idx):
        base = get()
        old = base[idx]
        base[idx] = old + h
        setter(base)
        lp = T.loss(noisy, clean, 10.0, enc, dec)
        base[idx] = old - h
        setter(base)
        lm = T.loss(noisy, clean, 10.0, enc, dec)
        base[idx] = old
        setter(base)
        return (lp - lm) / (2 * h)

    for li in range(5):
        for which in (0, 1):
            arr = enc[li][which]
            grad = g_enc[li][which]
            scale = np.max(np.abs(grad)) + 1e-12
            for _ in range(6):
                idx = tuple(rng.integers(s) for s in arr.shape)
                num = fd(lambda: enc[li][which], lambda a: None, idx)
                assert abs(num - grad[idx]) <= 1e-5 * scale + 1e-9, (li, which, idx, num, grad[idx])
    for which in (0, 1):
        arr = dec[which]
        for _ in range(6):
            idx = tuple(rng.integers(s) for s in arr.shape)
            num = fd(lambda: dec[which], lambda a: None, idx)
            assert abs(num - g_dec[which][idx]) <= 1e-5 * (np.max(np.abs(g_dec[which])) + 1e-12) + 1e-9


def test_adam_first_step_is_lr_sign():
    p = [np.array([1.0, -2.0, 3.0])]
    g = [np.array([0.5, -1e-3, 0.0])]
    out, m, v = T.adam_step(p, g, [np.zeros(3)], [np.zeros(3)], 1, 0.01)
    np.testing.assert_allclose(out[0], [0.99, -1.99, 3.0], rtol=0, atol=1e-7)
