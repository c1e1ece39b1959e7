"""Pins of the rotor-thrust-rate model (Sec. IV-A, oracle.rotor) against closed forms,
invariants and special cases."""
import numpy as np

import workloads as W
from oracle import mppi as O
from oracle import rotor as R


def _prm(**over):
    d = dict(W.params(8, 10), dynamics="rotor")
    d.update(over)
    return O.Params(**d)


def _step(state, u, prm, n=1):
    s = np.asarray(state, dtype=np.float64)
    for _ in range(n):
        s = R.plant_step(s, u, prm)
    return s


def test_layout_torques_closed_form():
    x, y, k = R.rotor_layout(0.2, 0.01)
    d = 0.2 / np.sqrt(2.0)
    assert np.allclose(x, [d, -d, -d, d]) and np.allclose(y, [-d, -d, d, d]) and np.allclose(k, [0.01, -0.01, 0.01, -0.01])
    # equal thrusts: no torque; (a, a, b, b): pure roll 2 d (b - a); (a, b, b, a): pitch 2 d (a - b)... sign of -x
    assert np.allclose(R.torque(np.full(4, 3.0), 0.2, 0.01), 0.0)
    assert np.allclose(R.torque(np.array([1.0, 1.0, 2.0, 2.0]), 0.2, 0.01), [2 * d, 0.0, 0.0])
    assert np.allclose(R.torque(np.array([2.0, 1.0, 1.0, 2.0]), 0.2, 0.01), [0.0, -2 * d, 0.0])
    assert np.allclose(R.torque(np.array([2.0, 1.0, 2.0, 1.0]), 0.2, 0.01), [0.0, 0.0, 0.02])


def test_hover_is_an_equilibrium():
    # zero net force and torque up to the rounding of the torque sums (~1e-16)
    prm = _prm()
    s0 = R.hover_state([1.0, -2.0, 3.0], prm)
    np.testing.assert_allclose(_step(s0, np.zeros(4), prm, 20), s0, rtol=0, atol=1e-13)


def test_equal_thrust_ramp_gives_the_cubic_climb():
    # level, at rest, every rotor ramping at c N/s: z'' = (4 (T0 + c t)) / m - g, a cubic in t,
    # which RK4 integrates exactly
    prm = _prm()
    c, n = 3.0, 10
    s = R.hover_state([0.0, 0.0, 0.0], prm)
    T0 = s[13]
    out = _step(s, np.full(4, c), prm, n)
    t = n * prm.dt
    z = (4 * T0 / prm.mass - prm.gravity) * t * t / 2 + (4 * c / prm.mass) * t ** 3 / 6
    assert abs(out[2] - z) < 1e-12 and abs(out[5] - (4 * c / prm.mass) * t * t / 2) < 1e-12
    np.testing.assert_allclose(out[13:17], T0 + c * t, atol=1e-12)
    np.testing.assert_allclose(out[6:10], [1.0, 0.0, 0.0, 0.0], atol=1e-13)


def test_pure_yaw_torque_spins_up_linearly():
    prm = _prm()
    a, b = 2.5, 1.5
    s = R.hover_state([0.0, 0.0, 0.0], prm)
    s[13:17] = [a, b, a, b]
    n = 8
    out = _step(s, np.zeros(4), prm, n)
    t = n * prm.dt
    alpha = 2 * prm.kappa * (a - b) / prm.inertia[2]
    assert abs(out[12] - alpha * t) < 1e-12 and abs(out[10]) < 1e-15 and abs(out[11]) < 1e-15
    psi = alpha * t * t / 2
    np.testing.assert_allclose(out[6:10], [np.cos(psi / 2), 0.0, 0.0, np.sin(psi / 2)], atol=1e-9)


def test_torque_free_rotation_conserves_energy_and_momentum():
    prm = _prm(gravity=0.0)
    s = R.hover_state([0.0, 0.0, 0.0], prm)
    s[13:17] = 0.0
    s[10:13] = [3.0, -1.0, 2.0]
    J = np.array(prm.inertia)
    e0, l0 = 0.5 * np.sum(J * s[10:13] ** 2), np.linalg.norm(J * s[10:13])
    out = _step(s, np.zeros(4), prm, 25)
    w = out[10:13]
    assert abs(0.5 * np.sum(J * w ** 2) - e0) < 1e-8 and abs(np.linalg.norm(J * w) - l0) < 1e-8
    assert not np.allclose(w, s[10:13])                      # the gyroscopic term does act


def test_thrusts_are_clamped_to_their_bounds():
    prm = _prm()
    s = R.hover_state([0.0, 0.0, 0.0], prm)
    out = _step(s, np.full(4, -1000.0), prm)
    np.testing.assert_array_equal(out[13:17], 0.0)
    out = _step(s, np.full(4, 1e6), prm)
    np.testing.assert_array_equal(out[13:17], prm.rotor_thrust_max)


def test_rotor_step_clips_rates_and_keeps_hover_at_hover():
    prm = _prm(K=32, H=6, sigma_tdot=0.0)
    poses = np.array([[5.0, 0.0, 0.0, 1.0, 0.0, 0.0, 0.0]])
    s = R.hover_state([0.0, 0.0, 0.0], prm)
    out = O.mppi_step(s, np.zeros((6, 4)), poses, prm, 0)
    np.testing.assert_array_equal(out["U_new"], 0.0)
    nxt, nom = O.receding_horizon(s, out["U_new"], prm)
    np.testing.assert_allclose(nxt, s, rtol=0, atol=1e-13)
    np.testing.assert_array_equal(nom, 0.0)
    noisy = O.mppi_step(s, np.full((6, 4), 9.5), poses, O.Params(**dict(prm.__dict__, sigma_tdot=5.0)), 0)
    assert np.all(np.abs(noisy["U"]) <= prm.tdot_max)
