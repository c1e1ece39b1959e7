"""Seeded synthetic inputs shared by the oracle checks, the tests and the bench.

This module holds no arithmetic of the control method: it only draws and
packages inputs (gate poses, latent codes, MLP weights, start states and the
controller parameters of each workload).  It imports neither the oracle nor
the CUDA package, and neither of them imports it.

Workloads (stand-ins for the paper's simulated race tracks, whose layouts,
depth images and trained networks are not available):

* ``hover_gate``   K=256,  H=20, one gate at the origin facing +x, analytic
                   frame SDF, start hovering 5 m in front of it (10 steps).
* ``two_gate_mlp`` K=4096, H=50, two gates at seeded poses 6-10 m apart with
                   yaw in [-60, 60] deg and pitch in [-30, 30] deg, Gate-SDF MLP
                   with Xavier-uniform weights and N(0, 1) latents (100 steps).
* ``four_gate_mlp`` K=16384, H=64, four such gates.
* ``depth_views``  64 camera poses approaching the two-gate track, rendered at
                   640 x 480 by a pinhole camera of about 80 x 64 degrees (a stereo
                   depth sensor's field of view; the paper's sensor and images are
                   not available), with depth noise and dropout.
"""

import math

import numpy as np

LATENT_DIM = 64
HIDDEN = 128
N_HIDDEN_LAYERS = 4

BASE_PARAMS = dict(
    dt=0.02, mass=0.8, gravity=9.81,
    thrust_min=0.0, thrust_max=30.0, rate_max=8.0,
    sigma_thrust=2.0, sigma_rate=1.5, lam=0.1,
    w_col=100.0, d_safe=0.3, w_u=1e-3,
    seed=0, drone_id=0,
)


def params(K, H, **over):
    d = dict(BASE_PARAMS)
    d.update(K=K, H=H)
    d.update(over)
    return d


def paper_params(K, H, **over):
    """Parameters of the paper's cost form (Eq. 6-9): d_safe = 1.0 m (its table of MPPI
    parameters), weights Q_gate = 1, Q_vis = 1, Q_sdf = 10 and a 30 degree guidance cone."""
    d = params(K, H, cost_mode="paper", d_safe=1.0, q_gate=1.0, q_vis=1.0, q_sdf=10.0,
               guide_tan_alpha=math.tan(math.radians(30.0)))
    d.update(over)
    return d


def rotor_params(K, H, **over):
    """Parameters of the paper's rotor-thrust-rate model: its Table I bounds (thrust rates in
    [-10, 10] N/s, rotor thrusts in [0, 10] N) and the airframe readings (arm 0.15 m, reaction
    torque 0.016 m per newton, inertia diag(0.003, 0.003, 0.005) kg m^2), noise 5 N/s."""
    d = params(K, H, dynamics="rotor", tdot_max=10.0, rotor_thrust_max=10.0, sigma_tdot=5.0,
               arm_length=0.15, kappa=0.016, inertia=(0.003, 0.003, 0.005))
    d.update(over)
    return d


def rotor_state(position, mass=0.8, gravity=9.81, yaw=0.0, rates=(0.0, 0.0, 0.0), thrust_offsets=(0.0, 0.0, 0.0, 0.0)):
    """A 17-number rotor-model state: at rest at `position` with heading `yaw`, body rates
    `rates`, every rotor carrying m g / 4 plus its offset (float32)."""
    s = np.zeros(17, dtype=np.float32)
    s[0:3] = position
    s[6], s[9] = math.cos(0.5 * yaw), math.sin(0.5 * yaw)
    s[10:13] = rates
    s[13:17] = 0.25 * mass * gravity + np.asarray(thrust_offsets, dtype=np.float32)
    return s


def yaw_pitch_quat(yaw, pitch):
    """Unit quaternion (w, x, y, z) of a yaw about world z followed by a pitch about the
    yawed y axis, written out in closed form from the half-angle sines and cosines."""
    cy, sy = math.cos(0.5 * yaw), math.sin(0.5 * yaw)
    cp, sp = math.cos(0.5 * pitch), math.sin(0.5 * pitch)
    return [cy * cp, -sy * sp, cy * sp, sy * cp]


def gate_track(n_gates, seed=3, start=(0.0, 0.0, 0.0), spacing=(6.0, 10.0),
               max_yaw_deg=60.0, max_pitch_deg=30.0):
    """Gate poses [n, 7] = (t, q): gate i at t_{i-1} + d_i e_x with d_i ~ U(spacing)."""
    rng = np.random.default_rng(seed)
    poses = np.zeros((n_gates, 7), dtype=np.float32)
    t = np.array(start, dtype=np.float64)
    for i in range(n_gates):
        t = t + np.array([rng.uniform(*spacing), 0.0, 0.0])
        yaw = math.radians(rng.uniform(-max_yaw_deg, max_yaw_deg))
        pitch = math.radians(rng.uniform(-max_pitch_deg, max_pitch_deg))
        poses[i, 0:3] = t
        poses[i, 3:7] = yaw_pitch_quat(yaw, pitch)
    return poses


def origin_gate():
    """One gate at the origin, unrotated (normal +x)."""
    return np.array([[0.0, 0.0, 0.0, 1.0, 0.0, 0.0, 0.0]], dtype=np.float32)


def latents(n_gates, dim=LATENT_DIM, seed=2):
    return np.random.default_rng(seed).standard_normal((n_gates, dim)).astype(np.float32)


def xavier_mlp(seed=1, in_dim=3 + LATENT_DIM, hidden=HIDDEN, n_hidden=N_HIDDEN_LAYERS):
    """Xavier-uniform weights U(-a, a), a = sqrt(6 / (fan_in + fan_out)); zero biases.

    Returns [(W [out, in], b [out])] for in -> hidden x n_hidden -> 1, float32.
    """
    rng = np.random.default_rng(seed)
    dims = [in_dim] + [hidden] * n_hidden + [1]
    layers = []
    for fi, fo in zip(dims[:-1], dims[1:]):
        a = math.sqrt(6.0 / (fi + fo))
        W = rng.uniform(-a, a, size=(fo, fi)).astype(np.float32)
        layers.append((W, np.zeros(fo, dtype=np.float32)))
    return layers


def hover_state(position):
    s = np.zeros(13, dtype=np.float32)
    s[0:3] = position
    s[6] = 1.0
    return s


def hover_nominal(H, mass=BASE_PARAMS["mass"], gravity=BASE_PARAMS["gravity"]):
    U = np.zeros((H, 4), dtype=np.float32)
    U[:, 0] = np.float32(mass * gravity)
    return U


def perturbed_states(n, seed, base):
    """n start states near ``base``: position jitter, velocity, a small random attitude."""
    rng = np.random.default_rng(seed)
    out = np.repeat(np.asarray(base, dtype=np.float32)[None, :], n, axis=0)
    out[:, 0:3] += rng.normal(0.0, 0.5, (n, 3)).astype(np.float32)
    out[:, 3:6] = rng.normal(0.0, 1.0, (n, 3)).astype(np.float32)
    q = rng.normal(0.0, 1.0, (n, 4))
    q[:, 0] += 6.0
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    out[:, 6:10] = q.astype(np.float32)
    out[:, 10:13] = rng.normal(0.0, 0.5, (n, 3)).astype(np.float32)
    return out


def hover_gate():
    """K=256, H=20, one gate at the origin facing +x, analytic SDF, start 5 m in front."""
    prm = params(256, 20)
    return dict(name="hover_gate_K256_H20_G1_analytic", params=prm, poses=origin_gate(),
                latents=np.zeros((1, LATENT_DIM), dtype=np.float32), layers=None,
                state=hover_state([-5.0, 0.0, 0.0]), nominal=hover_nominal(20), steps=10)


def two_gate_mlp():
    """K=4096, H=50, two seeded gates, Gate-SDF MLP (Xavier seed 1, latents seed 2)."""
    prm = params(4096, 50)
    return dict(name="two_gate_mlp_K4096_H50_G2", params=prm, poses=gate_track(2),
                latents=latents(2), layers=xavier_mlp(1),
                state=hover_state([0.0, 0.0, 0.0]), nominal=hover_nominal(50), steps=100)


def four_gate_mlp():
    """K=16384, H=64, four seeded gates, Gate-SDF MLP."""
    prm = params(16384, 64)
    return dict(name="four_gate_mlp_K16384_H64_G4", params=prm, poses=gate_track(4),
                latents=latents(4), layers=xavier_mlp(1),
                state=hover_state([0.0, 0.0, 0.0]), nominal=hover_nominal(64), steps=3)


def serving_fleet(n_drones, seed=4, Ks=(1024, 2048, 4096, 8192), Hs=(30, 50, 80), max_gates=4):
    """Drones of the serving workload: per drone K, H and the number of gates in view
    (1..max_gates) drawn uniformly, its own seeded gate poses and latents, and a start
    state near the origin.  Returns a list of dicts (params, poses, latents, state, drone_id)."""
    rng = np.random.default_rng(seed)
    fleet = []
    for d in range(n_drones):
        K = int(rng.choice(Ks))
        H = int(rng.choice(Hs))
        G = int(rng.integers(1, max_gates + 1))
        prm = params(K, H, drone_id=d)
        fleet.append(dict(drone_id=d, params=prm, G=G, poses=gate_track(G, seed=1000 + d),
                          latents=latents(G, seed=2000 + d), state=perturbed_states(1, 3000 + d, hover_state([0, 0, 0]))[0]))
    return fleet


def poisson_arrivals(n_drones, rate_hz, duration_s, seed=5):
    """Request times of n_drones independent Poisson processes (exponential gaps):
    a time-sorted list of (t, drone_id)."""
    rng = np.random.default_rng(seed)
    out = []
    for d in range(n_drones):
        t = rng.exponential(1.0 / rate_hz)
        while t < duration_s:
            out.append((t, d))
            t += rng.exponential(1.0 / rate_hz)
    out.sort()
    return out


def camera_views(n_views, gate_poses, seed=6, dist=(2.0, 9.0), lateral=1.5, vertical=0.8,
                 yaw_jitter_deg=15.0, pitch_jitter_deg=10.0):
    """Camera poses [n, 7] approaching the gates: each in front of a random gate (on the side
    its normal points away from), at a distance ~ U(dist) along the normal, offset sideways
    and vertically, heading towards the gate centre with yaw / pitch jitter.  The camera looks
    along its +x axis (y left, z up)."""
    rng = np.random.default_rng(seed)
    gate_poses = np.asarray(gate_poses, dtype=np.float64).reshape(-1, 7)
    out = np.zeros((n_views, 7), dtype=np.float32)
    for i in range(n_views):
        g = gate_poses[rng.integers(len(gate_poses))]
        w, x, y, z = g[3:7] / np.linalg.norm(g[3:7])
        normal = np.array([1 - 2 * (y * y + z * z), 2 * (x * y + w * z), 2 * (x * z - w * y)])
        side = np.cross([0.0, 0.0, 1.0], normal)
        side /= max(np.linalg.norm(side), 1e-9)
        pos = (g[0:3] - rng.uniform(*dist) * normal + rng.uniform(-lateral, lateral) * side
               + np.array([0.0, 0.0, rng.uniform(-vertical, vertical)]))
        to_gate = g[0:3] - pos
        yaw = math.atan2(to_gate[1], to_gate[0]) + math.radians(rng.uniform(-yaw_jitter_deg, yaw_jitter_deg))
        elev = math.atan2(to_gate[2], math.hypot(to_gate[0], to_gate[1]))
        pitch = -elev + math.radians(rng.uniform(-pitch_jitter_deg, pitch_jitter_deg))
        out[i, 0:3] = pos
        out[i, 3:7] = yaw_pitch_quat(yaw, pitch)
    return out


DEPTH_CAMERA = dict(width=640, height=480, fx=385.0, fy=385.0, cx=320.0, cy=240.0, max_range=10.0)


def depth_views():
    """64 views of the two-gate track at 640 x 480, with depth noise sigma = 0.005 z^2 and 2 %
    dropout (readings of the paper's unspecified sensor noise)."""
    gates = gate_track(2)
    return dict(name="depth_views_N64_640x480_G2", camera=dict(DEPTH_CAMERA), gates=gates,
                cams=camera_views(64, gates), noise_depth_coeff=0.005, dropout=0.02, seed=9, frame=0)


ENCODER_CHANNELS = (16, 32, 64, 64)


def encoder_weights(seed=7, channels=ENCODER_CHANNELS, latent=LATENT_DIM):
    """Weights of the depth encoder: 4 convolutions 3x3 (He-uniform U(-a, a), a = sqrt(6 / fan_in),
    biases U(-0.05, 0.05)) and the linear head (Xavier-uniform, zero bias).
    Returns [(W [co, ci, 3, 3], b [co])] x 4 + [(W [64, 64], b [64])], float32."""
    rng = np.random.default_rng(seed)
    layers = []
    ci = 1
    for co in channels:
        a = math.sqrt(6.0 / (9 * ci))
        layers.append((rng.uniform(-a, a, size=(co, ci, 3, 3)).astype(np.float32),
                       rng.uniform(-0.05, 0.05, size=co).astype(np.float32)))
        ci = co
    a = math.sqrt(6.0 / (ci + latent))
    layers.append((rng.uniform(-a, a, size=(latent, ci)).astype(np.float32), np.zeros(latent, dtype=np.float32)))
    return layers
