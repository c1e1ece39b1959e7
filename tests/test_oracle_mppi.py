"""Pins for the MPPI step: temperature limits, degenerate cases, closed-form costs."""
import math

import numpy as np
import pytest

import workloads as W
from oracle import mppi, noise


def _prm(**over):
    return mppi.Params(**W.params(over.pop("K", 8), over.pop("H", 5), **over))


def test_weights_sum_to_one_and_shift_invariance():
    rng = np.random.default_rng(0)
    J = rng.normal(50, 5, 100)
    w = mppi.softmax_weights(J, 0.1)
    assert abs(w.sum() - 1.0) < 1e-14
    np.testing.assert_allclose(mppi.softmax_weights(J + 1234.5, 0.1), w, rtol=1e-10)
    # the plain (unshifted) definition of Eq. 5 at moderate costs
    Js = rng.normal(0, 0.05, 100)
    e = np.exp(-Js / 0.1)
    np.testing.assert_allclose(mppi.softmax_weights(Js, 0.1), e / e.sum(), rtol=1e-13)


def test_lambda_to_zero_selects_argmin_rollout():
    prm = _prm(K=32, H=6, lam=1e-6)
    w = W.hover_gate()
    out = mppi.mppi_step(w["state"], W.hover_nominal(6), w["poses"], prm, step=0)
    k = int(np.argmin(out["J"]))
    assert np.sort(out["J"])[1] - out["J"][k] > 1e-3          # a strict winner
    np.testing.assert_allclose(out["U_new"], out["U"][k], atol=1e-12)


def test_lambda_to_infinity_gives_mean_of_samples():
    prm = _prm(K=64, H=4, lam=1e9)
    w = W.hover_gate()
    out = mppi.mppi_step(w["state"], W.hover_nominal(4), w["poses"], prm, step=2)
    np.testing.assert_allclose(out["U_new"], out["U"].mean(axis=0), atol=1e-7)
    # with no clipping active, that is U* + mean noise
    assert np.all(out["U"][..., 0] > 0) and np.all(np.abs(out["U"][..., 1:]) < 8)
    np.testing.assert_allclose(out["U_new"], W.hover_nominal(4) + out["delta"].mean(axis=0), atol=1e-7)


def test_zero_noise_keeps_hover_and_uniform_weights():
    prm = _prm(K=16, H=5, sigma_thrust=0.0, sigma_rate=0.0)
    w = W.hover_gate()
    out = mppi.mppi_step(w["state"], W.hover_nominal(5), w["poses"], prm, step=0)
    np.testing.assert_allclose(out["weights"], 1.0 / 16, rtol=1e-14)
    np.testing.assert_allclose(out["U_new"], W.hover_nominal(5), rtol=1e-14)
    # 5 m in front of the gate no state is within d_safe; hover moves nothing; u = u_hover
    np.testing.assert_allclose(out["J"], 0.0, atol=1e-12)


def test_single_rollout_has_weight_one():
    prm = _prm(K=1, H=3)
    w = W.hover_gate()
    out = mppi.mppi_step(w["state"], W.hover_nominal(3), w["poses"], prm, step=0)
    assert out["weights"][0] == 1.0
    np.testing.assert_array_equal(out["U_new"], out["U"][0])


def test_collision_cost_closed_form_hovering_near_top_bar():
    # hovering at (0, 0, 0.35): the top bar's inner face z = 0.5 is 0.15 away
    H = 7
    prm = _prm(K=4, H=H, sigma_thrust=0.0, sigma_rate=0.0, w_col=100.0, d_safe=0.3)
    state = W.hover_state([0.0, 0.0, 0.35]).astype(np.float64)
    state[2] = 0.35                                  # exact inputs: the float32 copy of 0.35 is not 0.35
    nominal = np.tile(prm.u_hover(), (H, 1))
    out = mppi.mppi_step(state, nominal, W.origin_gate(), prm, step=0)
    np.testing.assert_allclose(out["sdf"], 0.15, atol=1e-12)
    np.testing.assert_allclose(out["J_col"], 100.0 * H * 0.15 ** 2, rtol=1e-10)


def test_progress_cost_free_fall_along_gate_normal():
    # gate pitched so its normal is +z; zero thrust: free fall of g T^2 / 2 against the normal
    H, dt, g = 10, 0.02, 9.81
    prm = _prm(K=2, H=H, sigma_thrust=0.0, sigma_rate=0.0, thrust_max=0.0)
    pitch = -math.pi / 2
    pose = np.array([[0.0, 0.0, 50.0, math.cos(pitch / 2), 0.0, math.sin(pitch / 2), 0.0]])
    state = W.hover_state([0.0, 0.0, 0.0])
    out = mppi.mppi_step(state, np.zeros((H, 4)), pose, prm, step=0)
    T = H * dt
    np.testing.assert_allclose(out["J_prog"], 0.5 * g * T * T, rtol=1e-10)
    np.testing.assert_allclose(out["J_ctl"], 1e-3 * H * (0.8 * g) ** 2, rtol=1e-12)


def test_target_gate_selection():
    poses = np.array([[5.0, 0, 0, 1, 0, 0, 0], [12.0, 0, 0, 1, 0, 0, 0]])
    assert mppi.target_gate(W.hover_state([0, 0, 0]), poses) == 0
    assert mppi.target_gate(W.hover_state([6, 0, 0]), poses) == 1
    assert mppi.target_gate(W.hover_state([13, 0, 0]), poses) == 1
    assert mppi.target_gate(W.hover_state([0, 0, 0]), np.zeros((0, 7))) == -1


def test_clipping_bounds():
    prm = _prm(K=4096, H=2, sigma_thrust=50.0, sigma_rate=50.0)
    out = mppi.mppi_step(W.hover_state([-5, 0, 0]), W.hover_nominal(2), W.origin_gate(), prm, step=0)
    U = out["U"]
    assert U[..., 0].min() == 0.0 and U[..., 0].max() == 30.0
    assert U[..., 1:].min() == -8.0 and U[..., 1:].max() == 8.0


def test_shift_and_receding_horizon_at_hover():
    prm = _prm(K=8, H=4, sigma_thrust=0.0, sigma_rate=0.0)
    state = W.hover_state([-5.0, 0.0, 0.0]).astype(np.float64)
    hover = np.tile(prm.u_hover(), (4, 1))
    recs, st, nom = mppi.closed_loop(state, hover, W.origin_gate(), prm, 5)
    np.testing.assert_allclose(st, state, atol=1e-12)
    np.testing.assert_allclose(nom, hover, rtol=1e-14)
    U_new = np.arange(16, dtype=np.float64).reshape(4, 4)
    sh = mppi.shift_nominal(U_new, prm)
    np.testing.assert_array_equal(sh[:3], U_new[1:])
    np.testing.assert_allclose(sh[3], [0.8 * 9.81, 0, 0, 0])


def test_mlp_sdf_uses_each_gates_latent():
    w = W.two_gate_mlp()
    pos = np.random.default_rng(0).uniform(0, 12, (5, 3, 3))
    s = mppi.min_gate_sdf(pos, w["poses"], w["latents"], w["layers"])
    from oracle import gate_sdf, mlp
    for g in range(2):
        pg = gate_sdf.to_gate_frame(pos.reshape(-1, 3), w["poses"][g])
        sg = mlp.sdf(w["layers"], pg, w["latents"][g]).reshape(5, 3)
        assert np.all(s <= sg + 1e-15)
