"""Pins for the rollout dynamics: closed forms, equilibria and a library rotation."""
import math

import numpy as np
import pytest

from oracle import dynamics as D

M, G, DT = 0.8, 9.81, 0.02


def _state(p=(0, 0, 0), v=(0, 0, 0), q=(1, 0, 0, 0)):
    return (np.array([p], dtype=np.float64), np.array([v], dtype=np.float64), np.array([q], dtype=np.float64))


def test_quaternion_convention_matches_scipy_rotation():
    from scipy.spatial.transform import Rotation
    rng = np.random.default_rng(0)
    q = rng.normal(size=(50, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    v = rng.normal(size=(50, 3))
    R = Rotation.from_quat(np.concatenate([q[:, 1:], q[:, :1]], axis=1))   # scipy: (x, y, z, w)
    np.testing.assert_allclose(D.quat_rotate(q, v), R.apply(v), atol=1e-12)
    np.testing.assert_allclose(D.body_z_axis(q), R.apply(np.array([0.0, 0.0, 1.0])), atol=1e-12)
    # Hamilton product composes rotations: R(a b) = R(a) R(b)
    a, b = q[:25], q[25:]
    Ra = Rotation.from_quat(np.concatenate([a[:, 1:], a[:, :1]], axis=1))
    Rb = Rotation.from_quat(np.concatenate([b[:, 1:], b[:, :1]], axis=1))
    np.testing.assert_allclose(D.quat_rotate(D.quat_mul(a, b), v[:25]), (Ra * Rb).apply(v[:25]), atol=1e-12)


def test_hover_is_an_equilibrium():
    p, v, q = _state(p=(1.0, -2.0, 3.0))
    u = np.array([[M * G, 0.0, 0.0, 0.0]])
    for _ in range(50):
        p, v, q, w = D.rk4_step(p, v, q, u, DT, M, G)
    np.testing.assert_allclose(p, [[1.0, -2.0, 3.0]], atol=1e-13)
    np.testing.assert_allclose(v, 0.0, atol=1e-13)
    np.testing.assert_allclose(q, [[1, 0, 0, 0]], atol=1e-15)


def test_free_fall_is_exact():
    # T = 0: p(t) = p0 + v0 t - g t^2 / 2 e_z, a polynomial RK4 integrates exactly
    p0, v0 = np.array([0.5, 1.0, 10.0]), np.array([2.0, -1.0, 3.0])
    p, v, q = _state(p=p0, v=v0)
    u = np.zeros((1, 4))
    n = 37
    for _ in range(n):
        p, v, q, _ = D.rk4_step(p, v, q, u, DT, M, G)
    t = n * DT
    np.testing.assert_allclose(p[0], p0 + v0 * t - 0.5 * G * t * t * np.array([0, 0, 1]), atol=1e-12)
    np.testing.assert_allclose(v[0], v0 - G * t * np.array([0, 0, 1]), atol=1e-12)


@pytest.mark.parametrize("angle", [0.3, -1.1, 2.5])
def test_constant_tilt_thrust(angle):
    # attitude a fixed rotation about world x by `angle`: thrust direction (0, -sin a, cos a)
    q0 = (math.cos(angle / 2), math.sin(angle / 2), 0.0, 0.0)
    p, v, q = _state(q=q0)
    T = 13.0
    u = np.array([[T, 0.0, 0.0, 0.0]])
    n = 25
    for _ in range(n):
        p, v, q, _ = D.rk4_step(p, v, q, u, DT, M, G)
    a = (T / M) * np.array([0.0, -math.sin(angle), math.cos(angle)]) - np.array([0, 0, G])
    t = n * DT
    np.testing.assert_allclose(p[0], 0.5 * a * t * t, atol=1e-12)
    np.testing.assert_allclose(v[0], a * t, atol=1e-12)


def test_constant_rate_matches_quaternion_exponential():
    w = np.array([1.3, -2.1, 0.7])
    q0 = np.array([0.9, 0.1, -0.3, 0.2])
    q0 /= np.linalg.norm(q0)
    p, v, q = _state(q=q0)
    u = np.array([[M * G, *w]])
    n = 60
    for _ in range(n):
        p, v, q, wout = D.rk4_step(p, v, q, u, DT, M, G)
        assert abs(np.linalg.norm(q) - 1.0) < 1e-15
    t = n * DT
    ang = np.linalg.norm(w) * t
    exp_w = np.concatenate([[math.cos(ang / 2)], math.sin(ang / 2) * w / np.linalg.norm(w)])
    expect = D.quat_mul(q0[None], exp_w[None])[0]
    np.testing.assert_allclose(q[0], expect, atol=1e-10)
    np.testing.assert_array_equal(wout[0], w)


def test_rollout_positions_are_post_step_states():
    rng = np.random.default_rng(1)
    U = np.concatenate([rng.uniform(0, 20, (3, 4, 1)), rng.uniform(-3, 3, (3, 4, 3))], axis=2)
    state = np.array([0, 0, 1, 0.5, 0, 0, 1, 0, 0, 0, 0, 0, 0], dtype=np.float64)
    pos = D.rollout(state, U, DT, M, G)
    assert pos.shape == (3, 4, 3)
    s = state.copy()
    for h in range(4):
        s = D.plant_step(s, U[1, h], DT, M, G)
        np.testing.assert_allclose(pos[1, h], s[0:3], atol=1e-14)
