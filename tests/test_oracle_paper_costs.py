"""Pins of the paper-cost form of the oracle (Sec. IV-B, Eq. 2, 6-9) against closed forms."""
import numpy as np
import pytest

import workloads as W
from oracle import dynamics as D
from oracle import gate_sdf as GS
from oracle import mppi as O

pytestmark = pytest.mark.filterwarnings("ignore")


def _prm(**over):
    d = dict(W.params(4, 3), cost_mode="paper", d_safe=1.0)
    d.update(over)
    return O.Params(**d)


def _gate(x=5.0, y=0.0, z=0.0):
    return np.array([[x, y, z, 1.0, 0.0, 0.0, 0.0]])


def _ident(K, H):
    att = np.zeros((K, H, 4))
    att[..., 0] = 1.0
    return att


def test_yaw_angle_closed_forms():
    for psi in (-2.5, -0.3, 0.0, 0.7, 3.0):
        q = [np.cos(psi / 2), 0.0, 0.0, np.sin(psi / 2)]
        assert abs(D.yaw_angle(q) - psi) < 1e-12
    # a pure pitch or roll keeps the heading at 0
    assert abs(D.yaw_angle([np.cos(0.2), 0.0, np.sin(0.2), 0.0])) < 1e-12
    assert abs(D.yaw_angle([np.cos(0.2), np.sin(0.2), 0.0, 0.0])) < 1e-12


def test_visibility_cost_facing_beside_and_behind():
    state = W.hover_state([0.0, 0.0, 0.0])
    prm = _prm(q_gate=0.0, q_sdf=0.0, q_vis=1.0)
    pos = np.zeros((3, 4, 3))                                    # three rollouts, four steps at the origin
    att = _ident(3, 4)
    for k, psi in enumerate((0.0, np.pi / 2, np.pi)):            # gate ahead, to the right of the heading, behind
        att[k, :, 0], att[k, :, 3] = np.cos(psi / 2), np.sin(psi / 2)
    c = O.paper_costs(state, pos, att, _gate(), prm)
    np.testing.assert_allclose(c["J_ctl"], [0.0, 4.0, 8.0], atol=1e-12)   # 4 x (1 - cos 0 / 90 / 180 deg)


def test_gate_progress_telescopes_and_free_fall_closed_form():
    state = W.hover_state([0.0, 0.0, 0.0])
    prm = _prm(q_vis=0.0, q_sdf=0.0, q_gate=1.0)
    rng = np.random.default_rng(0)
    pos = rng.normal(size=(5, 7, 3))
    wp = _gate(3.0, -1.0, 2.0)
    c = O.paper_costs(state, pos, _ident(5, 7), wp, prm)
    direct = np.sum((pos[:, -1] - wp[0, :3]) ** 2, axis=1) - np.sum(wp[0, :3] ** 2)
    np.testing.assert_allclose(c["J_prog"], direct, rtol=1e-12)
    # free fall from rest for T = H dt below a waypoint 2 m above: |2 + g T^2 / 2|^2 - 4
    H, dt, g = 10, 0.02, 9.81
    U = np.zeros((1, H, 4))
    p, att = D.rollout_states(state, U, dt, 0.8, g)
    T = H * dt
    c = O.paper_costs(state, p, att, _gate(0.0, 0.0, 2.0), _prm(q_vis=0.0, q_sdf=0.0, H=H))
    assert abs(c["J_prog"][0] - ((2.0 + 0.5 * g * T * T) ** 2 - 4.0)) < 1e-9


def test_sdf_hinge_on_the_guidance_field():
    state = W.hover_state([-5.0, 0.0, 0.0])
    prm = _prm(q_gate=0.0, q_vis=0.0, q_sdf=1.0, d_safe=1.0, guide_tan_alpha=0.5)
    # on the gate axis at x = -2: s = 0.5 + 2 * 0.5 - 0 = 1.5 (no cost); at x = -0.4, y = 0.3:
    # s = 0.5 + 0.2 - 0.3 = 0.4 -> cost 0.6; at the gate plane off axis (0, 0.9, 0): s = -0.4 -> 1.4
    pos = np.array([[[-2.0, 0.0, 0.0], [-0.4, 0.3, 0.0], [0.0, 0.9, 0.0]]])
    c = O.paper_costs(state, pos, _ident(1, 3), _gate(0.0), prm)
    np.testing.assert_allclose(c["sdf"][0], [1.5, 0.4, -0.4], atol=1e-12)
    assert abs(c["J_col"][0] - (0.0 + 0.6 + 1.4)) < 1e-12
    # the guidance field in a yawed gate frame matches Eq. 2 of the transformed point
    pose = np.array([1.0, 2.0, 0.0] + list(W.yaw_pitch_quat(0.6, 0.0)))
    pg = GS.to_gate_frame(pos.reshape(-1, 3), pose)
    c2 = O.paper_costs(state, pos, _ident(1, 3), pose[None], prm)
    np.testing.assert_allclose(c2["sdf"].reshape(-1), 0.5 + 0.5 * np.abs(pg[:, 0]) - np.max(np.abs(pg[:, 1:]), axis=1))


def test_paper_step_targets_the_first_uncrossed_gate_and_lambda_limits():
    poses = np.concatenate([_gate(-1.0), _gate(4.0), _gate(9.0)])   # the first one is behind the start
    state = W.hover_state([0.0, 0.0, 0.0])
    prm = _prm(K=64, H=8)
    out = O.mppi_step(state, W.hover_nominal(8), poses, prm, 0)
    pos = out["positions"]
    d2 = np.sum((pos[:, -1] - poses[1, :3]) ** 2, axis=1) - 16.0
    np.testing.assert_allclose(out["J_prog"], d2, rtol=1e-9, atol=1e-9)
    small = O.mppi_step(state, W.hover_nominal(8), poses, O.Params(**dict(prm.__dict__, lam=1e-9)), 0)
    k = int(np.argmin(small["J"]))
    np.testing.assert_allclose(small["U_new"], small["U"][k], atol=1e-12)
