"""Quadrotor rollout model x_dot = f(x, u) and its RK4 integration (Sec. IV-A).

Test infrastructure only (see ``oracle/__init__.py``).

State x = [p, v, q, w] (position, linear velocity, unit quaternion, body
rates; 3 + 3 + 4 + 3 = 13 numbers), as the paper lists it.  The paper's
command is the rotor-thrust rate vector; the rollouts here use the
collective-thrust + body-rate command u = [T, wx, wy, wz] instead.
Readings used on both sides of the parity check:

* world frame z-up, gravity g along -z; thrust acts along +z of the body;
* quaternions are (w, x, y, z), Hamilton product, rotating body -> world;
* the body-rate command is tracked ideally: during a step the body rate
  equals the (clipped) command and dw/dt = 0, so the state's w carries the
  last command;
* dp/dt = v,  dv/dt = (T / m) R(q) e_z - g e_z,  dq/dt = 1/2 q (x) (0, w),
  with R(q) e_z taken from the unit-quaternion rotation matrix
  (2(xz + wy), 2(yz - wx), 1 - 2(x^2 + y^2)) -- also at the RK4 stage
  points, where q is not exactly unit;
* one classical RK4 step per dt with the command held constant, then q is
  renormalised to unit length.
"""

import numpy as np


def quat_mul(a, b):
    """Hamilton product a (x) b of quaternions [..., 4] = (w, x, y, z)."""
    aw, ax, ay, az = (a[..., i] for i in range(4))
    bw, bx, by, bz = (b[..., i] for i in range(4))
    return np.stack([
        aw * bw - ax * bx - ay * by - az * bz,
        aw * bx + ax * bw + ay * bz - az * by,
        aw * by - ax * bz + ay * bw + az * bx,
        aw * bz + ax * by - ay * bx + az * bw,
    ], axis=-1)


def quat_conj(q):
    return q * np.array([1.0, -1.0, -1.0, -1.0])


def quat_rotate(q, v):
    """Rotate vectors v [..., 3] by unit quaternions q [..., 4]: q (x) (0, v) (x) q*."""
    zero = np.zeros(v.shape[:-1] + (1,))
    qv = np.concatenate([zero, v], axis=-1)
    return quat_mul(quat_mul(q, qv), quat_conj(q))[..., 1:]


def body_z_axis(q):
    """Third column of the rotation matrix of q: the body +z axis in world coordinates."""
    w, x, y, z = (q[..., i] for i in range(4))
    return np.stack([2.0 * (x * z + w * y), 2.0 * (y * z - w * x), 1.0 - 2.0 * (x * x + y * y)], axis=-1)


def derivatives(p, v, q, thrust, omega, mass, gravity):
    """f(x, u): (dp/dt, dv/dt, dq/dt) for thrust [...] and body rates omega [..., 3]."""
    acc = (thrust / mass)[..., None] * body_z_axis(q)
    acc[..., 2] -= gravity
    zero = np.zeros(omega.shape[:-1] + (1,))
    qdot = 0.5 * quat_mul(q, np.concatenate([zero, omega], axis=-1))
    return v, acc, qdot


def rk4_step(p, v, q, u, dt, mass, gravity):
    """Advance (p, v, q) by one RK4 step of length dt under command u [..., 4].

    Returns (p, v, q, w) after the step, with q renormalised and the body
    rate w equal to the commanded rate.
    """
    thrust = u[..., 0]
    omega = u[..., 1:4]
    k1 = derivatives(p, v, q, thrust, omega, mass, gravity)
    s2 = [x + 0.5 * dt * d for x, d in zip((p, v, q), k1)]
    k2 = derivatives(*s2, thrust, omega, mass, gravity)
    s3 = [x + 0.5 * dt * d for x, d in zip((p, v, q), k2)]
    k3 = derivatives(*s3, thrust, omega, mass, gravity)
    s4 = [x + dt * d for x, d in zip((p, v, q), k3)]
    k4 = derivatives(*s4, thrust, omega, mass, gravity)
    out = [x + (dt / 6.0) * (a + 2.0 * b + 2.0 * c + d)
           for x, a, b, c, d in zip((p, v, q), k1, k2, k3, k4)]
    p1, v1, q1 = out
    q1 = q1 / np.linalg.norm(q1, axis=-1, keepdims=True)
    return p1, v1, q1, omega.copy()


def unpack_state(x):
    x = np.asarray(x, dtype=np.float64)
    return x[..., 0:3], x[..., 3:6], x[..., 6:10], x[..., 10:13]


def pack_state(p, v, q, w):
    return np.concatenate([p, v, q, w], axis=-1)


def rollout_states(state, U, dt, mass, gravity):
    """Roll out command sequences U [K, H, 4] from one state [13].

    Returns (positions [K, H, 3], attitudes [K, H, 4]) of the post-step states 1 .. H.
    """
    K, H, _ = U.shape
    p0, v0, q0, _ = unpack_state(state)
    p = np.broadcast_to(p0, (K, 3)).copy()
    v = np.broadcast_to(v0, (K, 3)).copy()
    q = np.broadcast_to(q0, (K, 4)).copy()
    pos = np.empty((K, H, 3))
    att = np.empty((K, H, 4))
    for h in range(H):
        p, v, q, _ = rk4_step(p, v, q, U[:, h, :], dt, mass, gravity)
        pos[:, h, :] = p
        att[:, h, :] = q
    return pos, att


def rollout(state, U, dt, mass, gravity):
    """Positions [K, H, 3] of the post-step states p_1 .. p_H (see rollout_states)."""
    return rollout_states(state, U, dt, mass, gravity)[0]


def yaw_angle(q):
    """Heading of the body x axis about world z: atan2 of the first column of R(q)
    projected on the horizontal plane, (2 (xy + wz), 1 - 2 (y^2 + z^2))."""
    q = np.asarray(q, dtype=np.float64)
    w, x, y, z = q[..., 0], q[..., 1], q[..., 2], q[..., 3]
    return np.arctan2(2.0 * (x * y + w * z), 1.0 - 2.0 * (y * y + z * z))


def plant_step(state, u, dt, mass, gravity):
    """The true (noiseless) plant: one RK4 step of the same model from state [13]."""
    p, v, q, _ = unpack_state(state)
    p1, v1, q1, w1 = rk4_step(p, v, q, np.asarray(u, dtype=np.float64), dt, mass, gravity)
    return pack_state(p1, v1, q1, w1)
