"""Pins for the gate geometry: Eq. 1-2 closed forms, the frame SDF by brute force."""
import math

import numpy as np
import pytest

from oracle import gate_sdf as S

AIN, AOUT, D = 0.5, 0.75, 0.1


@pytest.mark.parametrize("p,expect", [
    ((0.0, 0.0, 0.0), 0.5),                                  # centre: inner edge 0.5 away
    ((2.0, 0.0, 0.0), math.hypot(1.9, 0.5)),                 # on the axis
    ((-0.7, 0.0, 0.0), math.hypot(0.6, 0.5)),
    ((0.0, 0.2, 0.0), 0.3),                                  # in the opening plane
    ((0.0, -0.1, 0.45), 0.05),
    ((0.0, 2.0, 0.0), 1.25),                                 # beside the gate
    ((3.0, 0.0, 0.6), 2.9),                                  # in front of the top bar
    ((0.0, 0.6, 0.0), -0.1),                                 # inside a post, midway
    ((0.05, 0.6, 0.0), -0.05),                               # inside, nearer a face
    ((0.0, 0.7, 0.7), -0.05),                                # inside a corner, near the outer edge
    ((0.0, 1.75, 1.75), math.sqrt(2.0)),                     # off the outer corner
    ((1.1, 0.0, 1.75), math.hypot(1.0, 1.0)),                # off an outer edge
])
def test_frame_sdf_closed_forms(p, expect):
    assert abs(S.frame_sdf(np.array(p))[()] - expect) < 1e-12


def _frame_surface_samples(h):
    """Dense samples of the boundary of the frame solid, spacing about h."""
    pts = []
    g = np.arange(-AOUT, AOUT + 1e-12, h)
    Y, Z = np.meshgrid(g, g, indexing="ij")
    ring = np.maximum(np.abs(Y), np.abs(Z)) >= AIN
    for x in (-D, D):                                          # the two faces |x| = d
        pts.append(np.stack([np.full(ring.sum(), x), Y[ring], Z[ring]], 1))
    xs = np.arange(-D, D + 1e-12, h)
    for half in (AIN, AOUT):                                   # inner and outer square walls
        s = np.arange(-half, half + 1e-12, h)
        X, T = np.meshgrid(xs, s, indexing="ij")
        X, T = X.ravel(), T.ravel()
        for sgn in (-1.0, 1.0):
            pts.append(np.stack([X, np.full_like(X, sgn * half), T], 1))
            pts.append(np.stack([X, T, np.full_like(X, sgn * half)], 1))
    return np.concatenate(pts)


def _inside_by_boxes(p):
    # point-in-solid from the four bars' bounds, written out directly
    x, y, z = p
    if abs(x) > D:
        return False
    top = abs(y) <= AOUT and AIN <= abs(z) <= AOUT
    post = AIN <= abs(y) <= AOUT and abs(z) <= AIN
    return top or post


def test_frame_sdf_brute_force():
    h = 0.004
    surf = _frame_surface_samples(h)
    rng = np.random.default_rng(3)
    q = np.concatenate([
        rng.uniform(-1.2, 1.2, (120, 3)),
        rng.uniform([-D, -AOUT, -AOUT], [D, AOUT, AOUT], (120, 3)),   # many inside the frame
    ])
    s = S.frame_sdf(q)
    for i, p in enumerate(q):
        dmin = np.sqrt(np.min(np.sum((surf - p) ** 2, axis=1)))
        sign = -1.0 if _inside_by_boxes(p) else 1.0
        assert abs(s[i] - sign * dmin) <= h, (p, s[i], sign * dmin)


def test_frame_sdf_eikonal():
    rng = np.random.default_rng(4)
    q = rng.uniform(-1.5, 1.5, (4000, 3))
    e = 1e-6
    grad = np.stack([(S.frame_sdf(q + e * np.eye(3)[i]) - S.frame_sdf(q - e * np.eye(3)[i])) / (2 * e)
                     for i in range(3)], axis=1)
    gn = np.linalg.norm(grad, axis=1)
    # |grad s| = 1 except on the measure-zero medial set and at the kinks
    assert np.mean(np.abs(gn - 1.0) < 1e-4) > 0.99


def test_radial_metric_and_guide_sdf():
    p = np.array([[0.0, 0.3, -0.4], [2.0, 0.0, 0.0], [-1.0, 0.9, 0.2]])
    np.testing.assert_allclose(S.radial_linf(p), [0.4, 0.0, 0.9])
    np.testing.assert_allclose(S.guide_sdf(p, c=0.5, alpha=0.0), [0.1, 0.5, -0.4])
    np.testing.assert_allclose(S.guide_sdf(p, c=0.5, alpha=math.pi / 4), [0.1, 2.5, 0.6], atol=1e-12)


def test_gate_frame_transform():
    yaw = math.pi / 2   # gate x axis along world y
    pose = np.array([1.0, 2.0, 3.0, math.cos(yaw / 2), 0.0, 0.0, math.sin(yaw / 2)])
    np.testing.assert_allclose(S.gate_normal(pose), [0.0, 1.0, 0.0], atol=1e-15)
    pw = np.array([[1.0, 3.0, 3.0], [0.0, 2.0, 3.0], [1.0, 2.0, 4.5]])
    np.testing.assert_allclose(S.to_gate_frame(pw, pose), [[1, 0, 0], [0, 1, 0], [0, 0, 1.5]], atol=1e-12)
