"""Sampled control perturbations delta u ~ N(0, Sigma) (Sec. IV-A, Eq. 5).

Test infrastructure only (see ``oracle/__init__.py``).

The paper draws Gaussian noise around the previous optimal sequence but does
not say how.  Reading used on both sides of the parity check:

* one Philox4x32-10 block per (rollout k, horizon step h), keyed by the
  64-bit seed (k0 = low word, k1 = high word), counter
  (k, h, step mod 2**32, drone_id), where ``step`` counts the control steps
  this controller has taken (0 for the first);
* each 32-bit word x becomes a uniform on the open interval (0, 1) as
  u = (floor(x / 2**8) + 1/2) * 2**-24;
* Box-Muller (G. E. P. Box and M. E. Muller, Ann. Math. Stat. 29, 1958) turns
  the uniform pairs (u0, u1) and (u2, u3) into four independent standard
  normals n0..n3: with r = sqrt(-2 ln ua) and theta = 2 pi ub, the pair is
  (r cos theta, r sin theta);
* Sigma is diagonal: delta = (sigma_T n0, sigma_w n1, sigma_w n2, sigma_w n3)
  for (thrust, body-rate x, y, z).
"""

import numpy as np

from .philox import philox4x32_10, split_seed


def words_to_uniform(words):
    """uint32 words -> float64 uniforms in (0, 1) on the 2**-24 grid."""
    w = np.asarray(words, dtype=np.uint64)
    return ((w >> np.uint64(8)).astype(np.float64) + 0.5) * 2.0 ** -24


def box_muller(ua, ub):
    """Box-Muller transform of two uniforms -> two standard normals."""
    r = np.sqrt(-2.0 * np.log(ua))
    theta = 2.0 * np.pi * ub
    return r * np.cos(theta), r * np.sin(theta)


def philox_words(K, H, seed, step, drone_id):
    """Raw Philox words for every (k, h): uint32 array [K, H, 4]."""
    k = np.arange(K, dtype=np.uint64)[:, None]
    h = np.arange(H, dtype=np.uint64)[None, :]
    ctr = np.empty((K, H, 4), dtype=np.uint64)
    ctr[..., 0] = k
    ctr[..., 1] = h
    ctr[..., 2] = np.uint64(int(step) & 0xFFFFFFFF)
    ctr[..., 3] = np.uint64(int(drone_id) & 0xFFFFFFFF)
    return philox4x32_10(ctr, split_seed(seed))


def standard_normals(words):
    """[..., 4] Philox words -> [..., 4] standard normals (n0, n1, n2, n3)."""
    u = words_to_uniform(words)
    n0, n1 = box_muller(u[..., 0], u[..., 1])
    n2, n3 = box_muller(u[..., 2], u[..., 3])
    return np.stack([n0, n1, n2, n3], axis=-1)


def control_noise(K, H, seed, step, drone_id, sigma_thrust, sigma_rate):
    """delta u for all rollouts and horizon steps: float64 [K, H, 4]."""
    n = standard_normals(philox_words(K, H, seed, step, drone_id))
    sigma = np.array([sigma_thrust, sigma_rate, sigma_rate, sigma_rate], dtype=np.float64)
    return n * sigma
