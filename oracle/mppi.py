"""One MPPI control step with Gate-SDF costs (Sec. IV, Eq. 5-10), and a closed loop.

Test infrastructure only (see ``oracle/__init__.py``).

Per control step (Sec. IV-A, Eq. 5):

1. draw delta U^m ~ N(0, Sigma) for every rollout m and horizon step
   (``oracle.noise``), and form U^m = clip(U* + delta U^m) with the thrust in
   [T_min, T_max] and each body rate in [-w_max, w_max];
2. roll out every U^m from the current state with the dynamics model
   (``oracle.dynamics``), giving positions p_1 .. p_H;
3. evaluate the cost of every rollout in the configured form of Eq. 8-10:
       J = J_col + J_prog + J_ctl
       J_col  = w_col * sum_{h=1..H} max(0, d_safe - s(p_h))^2
                with s(p) = min over gates of the gate's SDF (analytic frame
                or the Gate-SDF MLP queried at the gate-frame point),
       J_prog = -n_tgt . (p_H - p_0), the signed distance travelled along the
                target gate's normal (Eq. 6's per-step differences summed,
                in the configured linear form),
       J_ctl  = w_u * sum_{h=0..H-1} |U^m_h - u_hover|^2,  u_hover = (m g, 0, 0, 0);
4. weights w_m = exp(-J_m / lambda) / sum_i exp(-J_i / lambda), evaluated as
   exp(-(J_m - rho) / lambda) / eta with rho = min J (Eq. 5);
   or, with ``cost_mode = "paper"``, the paper's own terms (``paper_costs``, Eq. 6-9:
   waypoint progress, perception alignment, linear SDF hinge on the target gate's
   guidance SDF of Eq. 2 or its network);
5. U*_new = sum_m w_m U^m (Eq. 5; U^m the clipped sequences that were rolled out);
6. receding horizon: apply U*_new[0] to the plant for one step and start the
   next cycle from U*_new shifted left by one with u_hover appended.

Readings where the paper is silent are listed in the module docstrings of
``noise``, ``dynamics`` and ``gate_sdf`` and in ``target_gate`` below.
"""

from dataclasses import dataclass

import numpy as np

from . import dynamics, gate_sdf, mlp, noise, rotor


@dataclass
class Params:
    K: int = 256
    H: int = 20
    dt: float = 0.02
    mass: float = 0.8
    gravity: float = 9.81
    thrust_min: float = 0.0
    thrust_max: float = 30.0
    rate_max: float = 8.0
    sigma_thrust: float = 2.0
    sigma_rate: float = 1.5
    lam: float = 0.1
    w_col: float = 100.0
    d_safe: float = 0.3
    w_u: float = 1e-3
    seed: int = 0
    drone_id: int = 0
    # "configured": w_col max(0, d_safe - s)^2 + progress along the gate normal + control cost;
    # "paper": Q_gate J_gate + Q_vis J_vis + Q_sdf J_sdf (Eq. 6-9) on the target gate's
    # guidance SDF (Eq. 2, analytic) or its Gate-SDF network
    cost_mode: str = "configured"
    q_gate: float = 1.0
    q_vis: float = 1.0
    q_sdf: float = 10.0
    guide_tan_alpha: float = 0.5773502691896257      # tan(30 deg), the cone angle of Eq. 2
    # "ctbr": collective thrust + body rates; "rotor": the paper's rotor-thrust rates
    # (``oracle.rotor``) with the bounds of its Table I and the airframe readings below
    dynamics: str = "ctbr"
    tdot_max: float = 10.0
    rotor_thrust_max: float = 10.0
    sigma_tdot: float = 5.0
    arm_length: float = 0.15
    kappa: float = 0.016
    inertia: tuple = (0.003, 0.003, 0.005)
    # positional-encoding levels of the Gate-SDF decoder's query point (0: the raw point)
    pe_levels: int = 0

    def u_hover(self):
        if self.dynamics == "rotor":
            return np.zeros(4)
        return np.array([self.mass * self.gravity, 0.0, 0.0, 0.0])


def clip_controls(U, prm):
    if prm.dynamics == "rotor":
        return np.clip(U, -prm.tdot_max, prm.tdot_max)
    lo = np.array([prm.thrust_min, -prm.rate_max, -prm.rate_max, -prm.rate_max])
    hi = np.array([prm.thrust_max, prm.rate_max, prm.rate_max, prm.rate_max])
    return np.minimum(np.maximum(U, lo), hi)


def target_gate(state, poses):
    """Index of the first gate whose plane the current position has not crossed.

    A gate g counts as crossed once n_g . (p - t_g) >= 0; if every gate is
    crossed the last gate stays the target.  Returns -1 when there are no gates.
    """
    poses = np.asarray(poses, dtype=np.float64).reshape(-1, 7)
    if poses.shape[0] == 0:
        return -1
    p = np.asarray(state, dtype=np.float64)[0:3]
    for g in range(poses.shape[0]):
        if np.dot(gate_sdf.gate_normal(poses[g]), p - poses[g, 0:3]) < 0.0:
            return g
    return poses.shape[0] - 1


def min_gate_sdf(positions, poses, latents=None, layers=None, pe_levels=0):
    """s(p) = min over gates of the gate SDF at world points positions [..., 3].

    With ``layers`` the Gate-SDF MLP is queried at the gate-frame point with
    that gate's latent; without, the exact frame SDF is used.  +inf with no gates.
    """
    poses = np.asarray(poses, dtype=np.float64).reshape(-1, 7)
    shape = positions.shape[:-1]
    best = np.full(shape, np.inf)
    flat = positions.reshape(-1, 3)
    for g in range(poses.shape[0]):
        pg = gate_sdf.to_gate_frame(flat, poses[g])
        if layers is None:
            s = gate_sdf.frame_sdf(pg)
        else:
            s = mlp.sdf(layers, pg, latents[g], pe_levels=pe_levels)
        best = np.minimum(best, s.reshape(shape))
    return best


def rollout_costs(state, U, positions, poses, prm, latents=None, layers=None):
    """Cost terms of every rollout: dict of J_col, J_prog, J_ctl, J (each [K]) and sdf [K, H]."""
    p0 = np.asarray(state, dtype=np.float64)[0:3]
    s = min_gate_sdf(positions, poses, latents, layers, prm.pe_levels)
    J_col = prm.w_col * np.sum(np.maximum(0.0, prm.d_safe - s) ** 2, axis=1)
    g = target_gate(state, poses)
    if g < 0:
        J_prog = np.zeros(U.shape[0])
    else:
        n = gate_sdf.gate_normal(np.asarray(poses, dtype=np.float64).reshape(-1, 7)[g])
        J_prog = -((positions[:, -1, :] - p0) @ n)
    du = U - prm.u_hover()
    J_ctl = prm.w_u * np.sum(du * du, axis=(1, 2))
    return dict(sdf=s, J_col=J_col, J_prog=J_prog, J_ctl=J_ctl, J=J_col + J_prog + J_ctl)


def paper_costs(state, positions, attitudes, poses, prm, latents=None, layers=None):
    """The paper's task costs (Sec. IV-B) for every rollout, at the post-step states 1 .. H:

    J_gate = sum_k (|p_{k+1} - p_wp|^2 - |p_k - p_wp|^2)            (Eq. 6)
    J_vis  = sum_k (1 - cos(psi_k - psi_gate,k))                      (Eq. 7)
    J_sdf  = sum_k max(0, d_safe - s_k)                                (Eq. 8)
    J      = Q_gate J_gate + Q_vis J_vis + Q_sdf J_sdf                 (Eq. 9)

    The waypoint p_wp is the target gate's centre; psi_k is the yaw of the rollout's
    attitude, psi_gate,k the bearing from p_k to p_wp in the horizontal plane; s_k is the
    guidance SDF of Eq. 2 of the target gate (c = the opening's half-width, cone angle
    atan(guide_tan_alpha)) or, with ``layers``, the Gate-SDF network at the target gate.
    Returns the three weighted terms, their sum and s [K, H].
    """
    K, H, _ = positions.shape
    poses = np.asarray(poses, dtype=np.float64).reshape(-1, 7)
    g = target_gate(state, poses)
    if g < 0:
        z = np.zeros(K)
        return dict(sdf=np.full((K, H), np.inf), J_col=z, J_prog=z.copy(), J_ctl=z.copy(), J=z.copy())
    wp = poses[g, 0:3]
    p0 = np.asarray(state, dtype=np.float64)[0:3]
    p_all = np.concatenate([np.broadcast_to(p0, (K, 1, 3)), positions], axis=1)      # p_0 .. p_H
    d2 = np.sum((p_all - wp) ** 2, axis=-1)
    J_gate = np.sum(d2[:, 1:] - d2[:, :-1], axis=1)
    psi = dynamics.yaw_angle(attitudes)
    psi_gate = np.arctan2(wp[1] - positions[..., 1], wp[0] - positions[..., 0])
    J_vis = np.sum(1.0 - np.cos(psi - psi_gate), axis=1)
    pg = gate_sdf.to_gate_frame(positions.reshape(-1, 3), poses[g])
    if layers is None:
        s = gate_sdf.guide_sdf(pg, c=gate_sdf.GATE_INNER_HALF, alpha=np.arctan(prm.guide_tan_alpha))
    else:
        s = mlp.sdf(layers, pg, latents[g], pe_levels=prm.pe_levels)
    s = s.reshape(K, H)
    J_sdf = np.sum(np.maximum(0.0, prm.d_safe - s), axis=1)
    parts = dict(J_col=prm.q_sdf * J_sdf, J_prog=prm.q_gate * J_gate, J_ctl=prm.q_vis * J_vis)
    return dict(sdf=s, J=parts["J_col"] + parts["J_prog"] + parts["J_ctl"], **parts)


def softmax_weights(J, lam):
    """Eq. 5 weights with max-subtraction: rho = min J."""
    J = np.asarray(J, dtype=np.float64)
    rho = np.min(J)
    wt = np.exp(-(J - rho) / lam)
    return wt / np.sum(wt)


def weighted_update(w, U):
    """Eq. 5: U*_new[h] = sum_m w_m U^m[h]."""
    return np.einsum("k,khc->hc", w, U)


def shift_nominal(U_new, prm):
    """Warm start for the next cycle: drop the applied first action, append u_hover."""
    return np.concatenate([U_new[1:], prm.u_hover()[None, :]], axis=0)


def mppi_step(state, nominal, poses, prm, step, latents=None, layers=None):
    """One control step from state [13] and nominal U* [H, 4]; returns every intermediate."""
    state = np.asarray(state, dtype=np.float64)
    nominal = np.asarray(nominal, dtype=np.float64)
    rot = prm.dynamics == "rotor"
    delta = noise.control_noise(prm.K, prm.H, prm.seed, step, prm.drone_id,
                                prm.sigma_tdot if rot else prm.sigma_thrust, prm.sigma_tdot if rot else prm.sigma_rate)
    U = clip_controls(nominal[None, :, :] + delta, prm)
    if rot:
        positions, attitudes = rotor.rollout(state, U, prm)
    else:
        positions, attitudes = dynamics.rollout_states(state, U, prm.dt, prm.mass, prm.gravity)
    if prm.cost_mode == "paper":
        costs = paper_costs(state, positions, attitudes, poses, prm, latents, layers)
    else:
        costs = rollout_costs(state, U, positions, poses, prm, latents, layers)
    w = softmax_weights(costs["J"], prm.lam)
    U_new = weighted_update(w, U)
    out = dict(delta=delta, U=U, positions=positions, weights=w, U_new=U_new)
    out.update(costs)
    return out


def receding_horizon(state, U_new, prm):
    """Apply U*_new[0] to the plant; return (next state, next nominal)."""
    if prm.dynamics == "rotor":
        nxt = rotor.plant_step(state, U_new[0], prm)
    else:
        nxt = dynamics.plant_step(state, U_new[0], prm.dt, prm.mass, prm.gravity)
    return nxt, shift_nominal(U_new, prm)


def closed_loop(state, nominal, poses, prm, n_steps, latents=None, layers=None, first_step=0):
    """Free-running closed loop of n_steps control steps; returns per-step records."""
    records = []
    for i in range(n_steps):
        out = mppi_step(state, nominal, poses, prm, first_step + i, latents, layers)
        nxt, nominal = receding_horizon(state, out["U_new"], prm)
        records.append(dict(state=state, U_new=out["U_new"], J=out["J"]))
        state = nxt
    return records, state, nominal
