"""Pins for the uniform mapping, Box-Muller and the noise keying."""
import math

import numpy as np
import pytest

from oracle import noise


def test_uniform_mapping_endpoints():
    u = noise.words_to_uniform(np.array([0, 255, 256, 0xFFFFFFFF], dtype=np.uint32))
    np.testing.assert_array_equal(u, [2.0 ** -25, 2.0 ** -25, 3 * 2.0 ** -25, 1.0 - 2.0 ** -25])
    assert np.all((u > 0) & (u < 1))


@pytest.mark.parametrize("ua,ub,expect", [
    (math.exp(-0.5), 0.0, (1.0, 0.0)),
    (math.exp(-0.5), 0.25, (0.0, 1.0)),
    (math.exp(-0.5), 0.5, (-1.0, 0.0)),
    (math.exp(-2.0), 0.75, (0.0, -2.0)),
    (math.exp(-4.5), 0.125, (3.0 / math.sqrt(2), 3.0 / math.sqrt(2))),
])
def test_box_muller_closed_forms(ua, ub, expect):
    n0, n1 = noise.box_muller(np.float64(ua), np.float64(ub))
    assert abs(n0 - expect[0]) < 1e-12 and abs(n1 - expect[1]) < 1e-12


def test_normals_statistics():
    from scipy import stats
    n = noise.standard_normals(noise.philox_words(1024, 256, seed=11, step=3, drone_id=1))
    flat = n.reshape(-1, 4)
    N = flat.shape[0]
    for c in range(4):
        x = flat[:, c]
        assert abs(x.mean()) < 5 / math.sqrt(N)
        assert abs(x.var() - 1.0) < 5 * math.sqrt(2.0 / N)
        assert stats.kstest(x, "norm").pvalue > 1e-4
    corr = np.corrcoef(flat.T)
    assert np.max(np.abs(corr - np.eye(4))) < 5 / math.sqrt(N)


def test_noise_scaling_and_layout():
    d = noise.control_noise(64, 8, seed=0, step=0, drone_id=0, sigma_thrust=2.0, sigma_rate=1.5)
    n = noise.standard_normals(noise.philox_words(64, 8, 0, 0, 0))
    np.testing.assert_array_equal(d[..., 0], 2.0 * n[..., 0])
    np.testing.assert_array_equal(d[..., 1:], 1.5 * n[..., 1:])
    assert d.shape == (64, 8, 4)


def test_noise_keying_distinct_and_reproducible():
    a = noise.philox_words(16, 4, seed=5, step=0, drone_id=0)
    b = noise.philox_words(16, 4, seed=5, step=1, drone_id=0)
    c = noise.philox_words(16, 4, seed=5, step=0, drone_id=1)
    d = noise.philox_words(16, 4, seed=6, step=0, drone_id=0)
    e = noise.philox_words(16, 4, seed=5, step=0, drone_id=0)
    np.testing.assert_array_equal(a, e)
    for other in (b, c, d):
        assert not np.any(np.all(a == other, axis=-1))
    # step is taken modulo 2**32
    np.testing.assert_array_equal(noise.philox_words(4, 2, 5, 2**32 + 1, 0), noise.philox_words(4, 2, 5, 1, 0))
    # blocks are distinct over (k, h)
    assert np.unique(a.reshape(-1, 4), axis=0).shape[0] == 64
