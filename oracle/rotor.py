"""The paper's rotor-thrust-rate quadrotor model (Sec. IV-A) and its RK4 integration.

Test infrastructure only (see ``oracle/__init__.py``).

The paper's command is the derivative of the four rotor thrusts,
u = [dT_1/dt, dT_2/dt, dT_3/dt, dT_4/dt] (after Romero et al.), so the state adds
the rotor thrusts to [p, v, q, w]: x = [p, v, q, w, T_1..T_4] (17 numbers).  The paper
bounds the thrust rates and the rotor thrusts (Table I: [-10, 10] and [0, 10] N) but
gives no airframe constants.  Readings used on both sides of the parity check:

* X layout: rotor i sits at body (x_i, y_i) = d (1, -1), (-1, -1), (-1, 1), (1, 1) with
  d = l / sqrt(2) and arm length l; its reaction torque about body z is kappa_i T_i with
  kappa_i = kappa (+1, -1, +1, -1);
* the torque of the thrusts is tau = sum_i (y_i T_i, -x_i T_i, kappa_i T_i), the
  inertia J = diag(Jx, Jy, Jz);
* dp/dt = v,  dv/dt = (sum_i T_i / m) R(q) e_z - g e_z,  dq/dt = 1/2 q (x) (0, w),
  dw/dt = J^-1 (tau - w x (J w)),  dT_i/dt = u_i;
* R(q) e_z in the unit-quaternion form at every RK4 stage, as in ``dynamics``;
* one classical RK4 step per dt with u held, then q renormalised and every T_i clamped
  to [0, T_max].
"""

import numpy as np

from .dynamics import body_z_axis, quat_mul


def rotor_layout(arm_length, kappa):
    """Body-frame rotor positions x [4], y [4] and reaction-torque coefficients [4]."""
    d = arm_length / np.sqrt(2.0)
    x = d * np.array([1.0, -1.0, -1.0, 1.0])
    y = d * np.array([-1.0, -1.0, 1.0, 1.0])
    k = kappa * np.array([1.0, -1.0, 1.0, -1.0])
    return x, y, k


def torque(T, arm_length, kappa):
    """Body torque of rotor thrusts T [..., 4]."""
    x, y, k = rotor_layout(arm_length, kappa)
    return np.stack([T @ y, -(T @ x), T @ k], axis=-1)


def derivatives(p, v, q, w, T, u, prm):
    """f(x, u) of the rotor model: (dp, dv, dq, dw, dT)."""
    mass, g = prm.mass, prm.gravity
    J = np.asarray(prm.inertia, dtype=np.float64)
    acc = (np.sum(T, axis=-1) / mass)[..., None] * body_z_axis(q)
    acc[..., 2] -= g
    zero = np.zeros(w.shape[:-1] + (1,))
    dq = 0.5 * quat_mul(q, np.concatenate([zero, w], axis=-1))
    tau = torque(T, prm.arm_length, prm.kappa)
    dw = (tau - np.cross(w, J * w)) / J
    return v, acc, dq, dw, np.asarray(u, dtype=np.float64)


def rk4_step(p, v, q, w, T, u, prm):
    """One RK4 step of length dt with u [..., 4] held; q renormalised, T clamped."""
    dt = prm.dt
    x = (p, v, q, w, T)
    k1 = derivatives(*x, u, prm)
    k2 = derivatives(*[a + 0.5 * dt * b for a, b in zip(x, k1)], u, prm)
    k3 = derivatives(*[a + 0.5 * dt * b for a, b in zip(x, k2)], u, prm)
    k4 = derivatives(*[a + dt * b for a, b in zip(x, k3)], u, prm)
    p1, v1, q1, w1, T1 = [a + (dt / 6.0) * (b + 2.0 * c + 2.0 * d + e) for a, b, c, d, e in zip(x, k1, k2, k3, k4)]
    q1 = q1 / np.linalg.norm(q1, axis=-1, keepdims=True)
    T1 = np.clip(T1, 0.0, prm.rotor_thrust_max)
    return p1, v1, q1, w1, T1


def unpack(state):
    s = np.asarray(state, dtype=np.float64)
    return s[..., 0:3], s[..., 3:6], s[..., 6:10], s[..., 10:13], s[..., 13:17]


def rollout(state, U, prm):
    """Roll out thrust-rate sequences U [K, H, 4] from one 17-number state.

    Returns (positions [K, H, 3], attitudes [K, H, 4]) of the post-step states 1 .. H.
    """
    K, H, _ = U.shape
    p, v, q, w, T = (np.broadcast_to(a, (K, a.shape[-1])).copy() for a in unpack(state))
    pos = np.empty((K, H, 3))
    att = np.empty((K, H, 4))
    for h in range(H):
        p, v, q, w, T = rk4_step(p, v, q, w, T, U[:, h, :], prm)
        pos[:, h] = p
        att[:, h] = q
    return pos, att


def plant_step(state, u, prm):
    """The true (noiseless) plant: one RK4 step of the rotor model from a 17-number state."""
    p, v, q, w, T = rk4_step(*unpack(state), np.asarray(u, dtype=np.float64), prm)
    return np.concatenate([p, v, q, w, T])


def hover_state(position, prm):
    """At rest, level, every rotor carrying m g / 4."""
    s = np.zeros(17)
    s[0:3] = position
    s[6] = 1.0
    s[13:17] = prm.mass * prm.gravity / 4.0
    return s
