"""Pins for the depth renderer of the oracle (Sec. III-B's depth observation): a closed form for
a camera facing a gate head-on, the axis conventions of the image, invariance under a common
rigid motion, brute-force ray marching against the point-in-solid test, monotonicity in the
frame's size, and the statistics of the sensor noise."""
import math

import numpy as np
import pytest

from oracle import gate_sdf as S
from oracle import render as R

AIN, AOUT, D = 0.5, 0.75, 0.1


def _quat_axis_angle(axis, angle):
    axis = np.asarray(axis, dtype=np.float64)
    axis = axis / np.linalg.norm(axis)
    return np.concatenate([[math.cos(angle / 2)], math.sin(angle / 2) * axis])


def _qmul(a, b):
    w1, x1, y1, z1 = a
    w2, x2, y2, z2 = b
    return np.array([w1 * w2 - x1 * x2 - y1 * y2 - z1 * z2, w1 * x2 + x1 * w2 + y1 * z2 - z1 * y2,
                     w1 * y2 - x1 * z2 + y1 * w2 + z1 * x2, w1 * z2 + x1 * y2 - y1 * x2 + z1 * w2])


def _rotmat(q):
    w, x, y, z = q / np.linalg.norm(q)
    return np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)],
                     [2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)],
                     [2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)]])


IDENT = np.array([1.0, 0.0, 0.0, 0.0])
CAM = dict(width=128, height=96, fx=118.3, fy=121.7, cx=61.7, cy=50.9)


def _head_on_closed_form(dist, width, height, fx, fy, cx, cy, max_range):
    """Camera at (-dist, 0, 0) looking along +x at the gate at the origin: per pixel, the ray
    (1, a, b) meets the front face x = -d at t = dist - d where max(|y|, |z|) = t max(|a|, |b|);
    inside the opening it meets the inner wall where max(|y|, |z|) = a_in, if that is before the
    back face."""
    u = np.arange(width) + 0.5
    v = np.arange(height) + 0.5
    a = -(u[None, :] - cx) / fx
    b = -(v[:, None] - cy) / fy
    m = np.maximum(np.abs(a), np.abs(b))
    t1 = dist - D
    r1 = t1 * m
    with np.errstate(divide="ignore"):
        t_in = np.where(m > 0, AIN / m, np.inf)
    out = np.full((height, width), max_range)
    front = (r1 >= AIN) & (r1 <= AOUT)
    out[front] = t1
    wall = (r1 < AIN) & (t_in <= dist + D)
    out[wall] = t_in[wall]
    return out


@pytest.mark.parametrize("dist", [2.0, 2.6, 4.0])
def test_head_on_closed_form(dist):
    cam = np.concatenate([[-dist, 0.0, 0.0], IDENT])
    gate = np.concatenate([[0.0, 0.0, 0.0], IDENT])
    got = R.depth_image(cam, gate, max_range=10.0, **CAM)
    want = _head_on_closed_form(dist, max_range=10.0, **CAM)
    assert np.count_nonzero(want < 10.0) > 200            # the frame fills a real part of the image
    assert np.count_nonzero((want > dist - D) & (want < 10.0)) > 0 or dist > 3.0   # inner-wall pixels
    np.testing.assert_allclose(got, want, rtol=0, atol=1e-12)


def test_depth_is_the_optical_axis_coordinate():
    """Every pixel that sees the front face reads dist - d, however oblique its ray."""
    cam = np.concatenate([[-3.0, 0.0, 0.0], IDENT])
    got = R.depth_image(cam, np.concatenate([[0.0, 0.0, 0.0], IDENT]), max_range=10.0, **CAM)
    vals = got[got < 10.0]
    assert np.count_nonzero(np.abs(vals - 2.9) < 1e-12) > 100


def test_image_axes():
    """y left / z up in the camera frame appear at u < cx / v < cy."""
    cam = np.concatenate([[0.0, 0.0, 0.0], IDENT])
    gate = np.concatenate([[6.0, 2.0, 1.0], IDENT])
    img = R.depth_image(cam, gate, max_range=20.0, **CAM)
    vv, uu = np.nonzero(img < 20.0)
    assert len(uu) > 50
    assert uu.mean() + 0.5 < CAM["cx"] - 20 and vv.mean() + 0.5 < CAM["cy"] - 10


def test_camera_yaw_turns_the_view():
    cam = np.concatenate([[0.0, 0.0, 0.0], _quat_axis_angle([0, 0, 1], math.pi / 2)])   # looks along +y
    facing = np.concatenate([[0.0, 6.0, 0.0], _quat_axis_angle([0, 0, 1], math.pi / 2)])
    behind = np.concatenate([[6.0, 0.0, 0.0], IDENT])
    img = R.depth_image(cam, facing, max_range=20.0, **CAM)
    vv, uu = np.nonzero(img < 20.0)
    assert abs(uu.mean() + 0.5 - CAM["cx"]) < 2.0 and abs(vv.mean() + 0.5 - CAM["cy"]) < 2.0
    assert np.all(img[img < 20.0] >= 5.9 - 1e-12)
    assert np.all(R.depth_image(cam, behind, max_range=20.0, **CAM) == 20.0)


def test_invariant_under_a_common_rigid_motion():
    cam = np.concatenate([[-2.6, 0.0, 0.0], IDENT])
    gate = np.concatenate([[0.0, 0.0, 0.0], IDENT])
    want = R.depth_image(cam, gate, max_range=10.0, **CAM)
    q = _quat_axis_angle([0.3, -0.5, 0.8], 1.1)
    t = np.array([3.0, -1.0, 2.0])
    Rm = _rotmat(q)
    cam2 = np.concatenate([Rm @ cam[0:3] + t, _qmul(q, cam[3:7])])
    gate2 = np.concatenate([Rm @ gate[0:3] + t, _qmul(q, gate[3:7])])
    got = R.depth_image(cam2, gate2, max_range=10.0, **CAM)
    diff = np.abs(got - want)
    # rounding can move a grazing ray across an edge; everything else agrees to rounding
    assert np.count_nonzero(diff > 1e-9) <= 3
    assert np.mean(want < 10.0) > 0.2


def _track():
    ga = np.concatenate([[4.0, 0.3, -0.2], _qmul(_quat_axis_angle([0, 0, 1], 0.44), _quat_axis_angle([0, 1, 0], -0.17))])
    gb = np.concatenate([[7.0, -1.5, 0.5], _qmul(_quat_axis_angle([0, 0, 1], -0.7), _quat_axis_angle([0, 1, 0], 0.26))])
    return np.stack([ga, gb])


def test_brute_force_ray_march():
    """March every ray in 2 mm steps with the point-in-solid test of the frame."""
    gates = _track()
    cam = np.concatenate([[0.0, 0.0, 0.0], _quat_axis_angle([0, 0, 1], 0.09)])
    kw = dict(width=40, height=30, fx=30.0, fy=30.0, cx=20.0, cy=15.0)
    max_range, step = 10.0, 2e-3
    t_or = R.first_hit(cam, gates, **kw)
    rays_c = R.pixel_rays(**kw).reshape(-1, 3)
    rays_w = rays_c @ _rotmat(cam[3:7]).T
    ts = np.arange(1, int(max_range / step) + 1) * step
    first = np.full(len(rays_w), np.inf)
    for g in gates:
        pts = cam[0:3] + ts[None, :, None] * rays_w[:, None, :]
        inside = S.in_frame(S.to_gate_frame(pts.reshape(-1, 3), g).reshape(pts.shape))
        idx = np.argmax(inside, axis=1)
        first = np.minimum(first, np.where(inside.any(axis=1), ts[idx], np.inf))
    t_or = t_or.reshape(-1)
    marched = np.isfinite(first)
    assert marched.sum() > 60
    # (b) a marched hit brackets the exact one within a step
    assert np.all(t_or[marched] <= first[marched] + 1e-12)
    assert np.all(t_or[marched] >= first[marched] - step - 1e-12)
    # (a) every exact hit lies on the surface of a frame and inside none
    hit = np.isfinite(t_or) & (t_or <= max_range)
    p = cam[0:3] + t_or[hit, None] * rays_w[hit]
    sd = np.stack([S.frame_sdf(S.to_gate_frame(p, g)) for g in gates])
    assert np.all(np.min(np.abs(sd), axis=0) < 1e-9)
    assert np.all(np.min(sd, axis=0) > -1e-9)
    # (c) hits the march stepped over are grazing chords, and rare
    assert np.count_nonzero(hit & ~marched) <= 0.02 * len(hit)


def test_growing_the_frame_never_deepens_a_pixel():
    gates = _track()
    cam = np.concatenate([[0.5, -0.4, 0.1], _quat_axis_angle([0, 0, 1], 0.05)])
    kw = dict(width=48, height=36, fx=36.0, fy=36.0, cx=24.3, cy=17.8, max_range=12.0)
    eps = 1e-3
    base = R.depth_image(cam, gates, **kw)
    grown = R.depth_image(cam, gates, a_in=AIN - eps, a_out=AOUT + eps, d=D + eps, **kw)
    shrunk = R.depth_image(cam, gates, a_in=AIN + eps, a_out=AOUT - eps, d=D - eps, **kw)
    assert np.all(grown <= base) and np.all(base <= shrunk)
    assert np.count_nonzero(grown < shrunk) > 0


def test_camera_inside_the_frame_reads_zero():
    cam = np.concatenate([[0.0, 0.6, 0.0], IDENT])            # inside the right post
    img = R.depth_image(cam, np.concatenate([[0.0, 0.0, 0.0], IDENT]), max_range=10.0, **CAM)
    assert np.all(img == 0.0)


# ---------------------------------------------------------------- sensor noise
def _flat(z, n_views=4, h=64, w=64):
    return np.full((n_views, h, w), z, dtype=np.float64)


def test_noise_off_is_identity():
    clean = R.depth_images(np.concatenate([[-2.6, 0.0, 0.0], IDENT])[None], np.concatenate([[0.0] * 3, IDENT]),
                           max_range=10.0, **CAM)
    np.testing.assert_array_equal(R.add_sensor_noise(clean, 10.0, 0.0, 0.0, seed=7, frame=3), clean)


def test_dropout_extremes_and_rate():
    clean = _flat(3.0)
    assert np.all(R.add_sensor_noise(clean, 10.0, 0.01, 1.0, seed=1, frame=0) == 0.0)
    noisy = R.add_sensor_noise(clean, 10.0, 0.0, 0.1, seed=1, frame=0)
    frac = np.mean(noisy == 0.0)
    assert abs(frac - 0.1) < 4 * math.sqrt(0.1 * 0.9 / noisy.size)
    assert np.all(noisy[noisy != 0.0] == 3.0)


@pytest.mark.parametrize("z", [2.0, 5.0])
def test_noise_sigma_grows_with_depth_squared(z):
    c = 0.01
    noisy = R.add_sensor_noise(_flat(z), 10.0, c, 0.0, seed=11, frame=2)
    n = ((noisy - z) / (c * z * z)).reshape(-1)
    assert abs(n.mean()) < 4.0 / math.sqrt(n.size)
    assert abs(n.var() - 1.0) < 4.0 * math.sqrt(2.0 / n.size)


def test_noise_clips_and_leaves_misses():
    clean = _flat(9.9)
    clean[:, :, :8] = 10.0                                      # pixels that saw nothing
    noisy = R.add_sensor_noise(clean, 10.0, 1.0, 0.0, seed=3, frame=0)
    assert np.all((noisy >= 0.0) & (noisy <= 10.0))
    assert np.all(noisy[:, :, :8] == 10.0)
    assert np.count_nonzero(noisy == 0.0) > 0 and np.count_nonzero(noisy[:, :, 8:] == 10.0) > 0


def test_noise_depends_on_view_and_frame():
    clean = _flat(4.0, n_views=2)
    a = R.add_sensor_noise(clean, 10.0, 0.01, 0.0, seed=5, frame=0)
    b = R.add_sensor_noise(clean, 10.0, 0.01, 0.0, seed=5, frame=1)
    assert not np.array_equal(a[0], a[1]) and not np.array_equal(a, b)
    np.testing.assert_array_equal(a, R.add_sensor_noise(clean, 10.0, 0.01, 0.0, seed=5, frame=0))


def test_noise_pairs_share_a_box_muller_radius():
    """The normals of pixels 2m and 2m + 1 are the cosine and sine branches of one Box-Muller
    draw: n_2m^2 + n_2m+1^2 = -2 ln u of that draw's first uniform, whatever the angle."""
    from oracle.noise import words_to_uniform
    from oracle.philox import philox4x32_10, split_seed
    pix = np.arange(0, 512, dtype=np.uint64)
    n, r = R.pixel_noise(pix, 3, seed=99, frame=4)
    ctr = np.stack([pix[0::2] >> np.uint64(1), np.full(256, 3, np.uint64), np.full(256, 4, np.uint64),
                    np.full(256, R.NORMAL_STREAM_TAG, np.uint64)], -1)
    u0 = words_to_uniform(philox4x32_10(ctr, split_seed(99))[:, 0])
    np.testing.assert_allclose(n[0::2] ** 2 + n[1::2] ** 2, -2.0 * np.log(u0), rtol=1e-12)
    # the angle differs between pairs and the dropout uniforms are all distinct
    assert len(np.unique(np.round(np.arctan2(n[1::2], n[0::2]), 12))) == 256
    assert len(np.unique(r)) > 500
