"""Gate geometry: gate-frame transform, Eq. 1-2 and the exact frame SDF.

Test infrastructure only (see ``oracle/__init__.py``).

In the gate's own frame the gate plane is x = 0 and (y, z) are transverse
(Sec. III-A).  A gate pose is (t, q): its centre t in the world and the unit
quaternion q (w, x, y, z) rotating gate -> world, so a world point p has
gate-frame coordinates R(q)^T (p - t) and the gate normal is R(q) e_x.

Gates are square frames with a 1.0 m inner and 1.5 m outer side (Sec. V);
their depth along the normal (0.2 m) is a stated reading.  The frame solid is

    F = { |x| <= d, r(p) <= a_out } minus { r(p) < a_in },   r(p) = max(|y|, |z|)  (Eq. 1)

with a_in = 0.5, a_out = 0.75, d = 0.1.  ``frame_sdf`` is the exact signed
Euclidean distance to F, positive in free space:

* outside F it is the distance to F, the minimum of the distances to four
  disjoint boxes whose union is F (the distance to a union is the minimum of
  the distances);
* inside F it is minus the distance to the complement of F, the nearest of
  the two faces |x| = d, the outer square r = a_out and the inner opening
  (Euclidean distance from (y, z) to the square [-a_in, a_in]^2).

``guide_sdf`` is the paper's hourglass guidance field (Eq. 2).
"""

import numpy as np

from .dynamics import quat_conj, quat_rotate

GATE_INNER_HALF = 0.5
GATE_OUTER_HALF = 0.75
GATE_HALF_DEPTH = 0.1


def to_gate_frame(p, pose):
    """World points p [..., 3] -> gate-frame points for one pose [7] = (t, q)."""
    pose = np.asarray(pose, dtype=np.float64)
    t, q = pose[0:3], pose[3:7]
    qc = np.broadcast_to(quat_conj(q), p.shape[:-1] + (4,))
    return quat_rotate(qc, p - t)


def gate_normal(pose):
    """World-frame gate normal R(q) e_x."""
    pose = np.asarray(pose, dtype=np.float64)
    return quat_rotate(pose[3:7], np.array([1.0, 0.0, 0.0]))


def radial_linf(pg):
    """Eq. 1: r(p) = max(|y|, |z|) in the gate frame."""
    return np.maximum(np.abs(pg[..., 1]), np.abs(pg[..., 2]))


def guide_sdf(pg, c=GATE_INNER_HALF, alpha=0.0):
    """Eq. 2: s_guide(p) = c + |x| tan(alpha) - r(p)."""
    return c + np.abs(pg[..., 0]) * np.tan(alpha) - radial_linf(pg)


def box_distance(pg, lo, hi):
    """Euclidean distance from points to the closed axis-aligned box [lo, hi] (0 inside)."""
    lo = np.asarray(lo, dtype=np.float64)
    hi = np.asarray(hi, dtype=np.float64)
    gap = np.maximum(np.maximum(lo - pg, pg - hi), 0.0)
    return np.sqrt(np.sum(gap * gap, axis=-1))


def frame_boxes(a_in=GATE_INNER_HALF, a_out=GATE_OUTER_HALF, d=GATE_HALF_DEPTH):
    """Four disjoint-interior bars (lo, hi) whose union is the frame solid F."""
    return [
        ((-d, -a_out, a_in), (d, a_out, a_out)),      # top bar (full width)
        ((-d, -a_out, -a_out), (d, a_out, -a_in)),    # bottom bar (full width)
        ((-d, a_in, -a_in), (d, a_out, a_in)),        # right post
        ((-d, -a_out, -a_in), (d, -a_in, a_in)),      # left post
    ]


def in_frame(pg, a_in=GATE_INNER_HALF, a_out=GATE_OUTER_HALF, d=GATE_HALF_DEPTH):
    r = radial_linf(pg)
    return (np.abs(pg[..., 0]) <= d) & (r <= a_out) & (r >= a_in)


def frame_sdf(pg, a_in=GATE_INNER_HALF, a_out=GATE_OUTER_HALF, d=GATE_HALF_DEPTH):
    """Exact signed distance to the gate frame F for gate-frame points [..., 3]."""
    pg = np.asarray(pg, dtype=np.float64)
    outside = np.min(np.stack([box_distance(pg, lo, hi) for lo, hi in frame_boxes(a_in, a_out, d)]), axis=0)
    ay = np.abs(pg[..., 1])
    az = np.abs(pg[..., 2])
    to_face = d - np.abs(pg[..., 0])
    to_outer = a_out - np.maximum(ay, az)
    to_opening = np.sqrt(np.maximum(ay - a_in, 0.0) ** 2 + np.maximum(az - a_in, 0.0) ** 2)
    inside = -np.minimum(np.minimum(to_face, to_outer), to_opening)
    return np.where(in_frame(pg, a_in, a_out, d), inside, outside)
