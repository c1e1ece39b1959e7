"""Depth images of the gate frames seen by a pinhole camera (the onboard depth observation
of Sec. III-B, which the paper renders with Genesis), by exact ray casting, and the
synthetic sensor noise that turns a clean image into the noisy input of the denoising
pre-training stage (Sec. III-B, I_noisy).

Test infrastructure only (see ``oracle/__init__.py``).

Readings (the paper gives neither a camera model nor its noise model):

* camera frame: x forward along the optical axis, y left, z up (the body axes of a drone
  with a forward-facing camera); a camera pose is (t, q) taking camera to world, and every
  quaternion (camera and gates) is normalised before use;
* pixel (u, v) of a W x H image, u to the right and v down, looks along
  d = (1, -(u + 1/2 - cx) / fx, -(v + 1/2 - cy) / fy) in the camera frame;
* the depth of a pixel is the optical-axis coordinate of the first point of any gate's
  frame on its ray (with d as above, the ray parameter t itself, t >= 0), or max_range
  when the ray meets no frame at or before max_range;
* a gate's frame is the union of four closed boxes in its gate frame
  (``gate_sdf.frame_boxes``); a ray enters a box where the slab intervals of the three
  axes first overlap;
* noise: with p = v W + u the pixel's linear index, its dropout uniform r is word (p mod 4)
  of the Philox block with counter (p div 4, view, frame, 0xDE9751), and its normal n is the
  cosine (p even) or sine (p odd) Box-Muller normal of words 0, 1 of the block with counter
  (p div 2, view, frame, 0xDE9750), both with key = the seed (one block serves four
  pixels' dropout and two pixels' normals); the noisy depth is 0 when r is below the dropout
  probability, else max_range for a pixel whose clean depth is max_range, else
  clip(z + c z^2 n, 0, max_range) (a stereo sensor's depth error grows with the square of
  the depth).
"""

import numpy as np

from . import gate_sdf
from .dynamics import quat_conj, quat_rotate
from .noise import box_muller, words_to_uniform
from .philox import philox4x32_10, split_seed

NORMAL_STREAM_TAG = 0xDE9750
DROPOUT_STREAM_TAG = 0xDE9751


def _unit_pose(pose):
    pose = np.array(pose, dtype=np.float64)
    pose[3:7] /= np.linalg.norm(pose[3:7])
    return pose


def pixel_rays(width, height, fx, fy, cx, cy):
    """Ray directions [H, W, 3] in the camera frame (x component 1)."""
    u = np.arange(width) + 0.5
    v = np.arange(height) + 0.5
    uu, vv = np.meshgrid(u, v)
    return np.stack([np.ones_like(uu), -(uu - cx) / fx, -(vv - cy) / fy], axis=-1)


def ray_box(o, d, lo, hi):
    """Entry parameter t >= 0 of rays o + t d [..., 3] into the closed box [lo, hi]; inf on a miss."""
    o = np.broadcast_to(o, d.shape)
    with np.errstate(divide="ignore", invalid="ignore"):
        t0 = (lo - o) / d
        t1 = (hi - o) / d
    tmin = np.minimum(t0, t1)
    tmax = np.maximum(t0, t1)
    # a ray parallel to a slab is inside it for every t, or for none
    par = d == 0.0
    inside = (o >= lo) & (o <= hi)
    tmin = np.where(par, np.where(inside, -np.inf, np.inf), tmin)
    tmax = np.where(par, np.where(inside, np.inf, -np.inf), tmax)
    enter = np.max(tmin, axis=-1)
    leave = np.min(tmax, axis=-1)
    hit = (enter <= leave) & (leave >= 0.0)
    return np.where(hit, np.maximum(enter, 0.0), np.inf)


def first_hit_rays(cam_pose, gate_poses, rays_c,
                   a_in=gate_sdf.GATE_INNER_HALF, a_out=gate_sdf.GATE_OUTER_HALF, d=gate_sdf.GATE_HALF_DEPTH):
    """Ray parameter [...] of the first frame point on camera-frame rays [..., 3] (inf: none)."""
    cam_pose = _unit_pose(cam_pose)
    rays_c = np.asarray(rays_c, dtype=np.float64)
    rays_w = quat_rotate(np.broadcast_to(cam_pose[3:7], rays_c.shape[:-1] + (4,)), rays_c)
    best = np.full(rays_c.shape[:-1], np.inf)
    for gp in np.asarray(gate_poses, dtype=np.float64).reshape(-1, 7):
        gp = _unit_pose(gp)
        o_g = gate_sdf.to_gate_frame(cam_pose[None, 0:3], gp)[0]
        q_inv = np.broadcast_to(quat_conj(gp[3:7]), rays_w.shape[:-1] + (4,))
        dirs_g = quat_rotate(q_inv, rays_w)
        for lo, hi in gate_sdf.frame_boxes(a_in, a_out, d):
            best = np.minimum(best, ray_box(o_g, dirs_g, np.asarray(lo), np.asarray(hi)))
    return best


def first_hit(cam_pose, gate_poses, width, height, fx, fy, cx, cy, **frame):
    """Ray parameter [H, W] of the first frame point on each pixel's ray (inf: none)."""
    return first_hit_rays(cam_pose, gate_poses, pixel_rays(width, height, fx, fy, cx, cy), **frame)


def pixel_depths(cam_pose, gate_poses, us, vs, fx, fy, cx, cy, max_range, **frame):
    """Clean depths of the pixels (us[i], vs[i]) of one view."""
    us = np.asarray(us, dtype=np.float64)
    vs = np.asarray(vs, dtype=np.float64)
    rays = np.stack([np.ones_like(us), -(us + 0.5 - cx) / fx, -(vs + 0.5 - cy) / fy], axis=-1)
    t = first_hit_rays(cam_pose, gate_poses, rays, **frame)
    return np.where(t <= max_range, t, max_range)


def depth_image(cam_pose, gate_poses, width, height, fx, fy, cx, cy, max_range, **frame):
    """Clean depth image [H, W] seen from camera pose (t, q) [7]."""
    t = first_hit(cam_pose, gate_poses, width, height, fx, fy, cx, cy, **frame)
    return np.where(t <= max_range, t, max_range)


def depth_images(cam_poses, gate_poses, width, height, fx, fy, cx, cy, max_range, **frame):
    """Clean depth images [N, H, W] for camera poses [N, 7]."""
    cams = np.asarray(cam_poses, dtype=np.float64).reshape(-1, 7)
    return np.stack([depth_image(c, gate_poses, width, height, fx, fy, cx, cy, max_range, **frame)
                     for c in cams]) if len(cams) else np.zeros((0, height, width))


def _blocks(index, view, seed, frame, tag):
    index, view = np.broadcast_arrays(np.asarray(index, dtype=np.uint64), np.asarray(view, dtype=np.uint64))
    ctr = np.empty(index.shape + (4,), dtype=np.uint64)
    ctr[..., 0] = index
    ctr[..., 1] = view
    ctr[..., 2] = np.uint64(int(frame) & 0xFFFFFFFF)
    ctr[..., 3] = np.uint64(tag)
    return philox4x32_10(ctr, split_seed(seed))


def pixel_noise(pix, view, seed, frame):
    """(normal n, dropout uniform r) of pixels with linear index pix = v W + u in views
    `view` (broadcast together)."""
    pix = np.asarray(pix, dtype=np.uint64)
    nw = _blocks(pix >> np.uint64(1), view, seed, frame, NORMAL_STREAM_TAG)
    un = words_to_uniform(nw)
    c, s_ = box_muller(un[..., 0], un[..., 1])
    n = np.where((pix & np.uint64(1)) == 0, c, s_)
    dw = _blocks(pix >> np.uint64(2), view, seed, frame, DROPOUT_STREAM_TAG)
    word = np.take_along_axis(dw, (pix & np.uint64(3)).astype(np.int64)[..., None], axis=-1)[..., 0]
    return n, words_to_uniform(word)


def image_noise(n_views, width, height, seed, frame):
    """(normals, dropout uniforms), each [N, H, W], of every pixel."""
    pix = np.arange(width * height, dtype=np.uint64)[None, :]
    view = np.arange(n_views, dtype=np.uint64)[:, None]
    n, r = pixel_noise(pix, view, seed, frame)
    return n.reshape(n_views, height, width), r.reshape(n_views, height, width)


def noisy_depths(clean, n, r, max_range, depth_coeff, dropout):
    """Noisy depths of pixels with clean depths `clean`, normals n and dropout uniforms r."""
    clean = np.asarray(clean, dtype=np.float64)
    hit = clean < max_range
    noisy = np.where(hit, np.clip(clean + depth_coeff * clean * clean * n, 0.0, max_range), max_range)
    # the dropout test compares the 24-bit uniform with the probability rounded to float32
    drop = r < float(np.float32(dropout))
    return np.where(drop, 0.0, noisy)


def add_sensor_noise(clean, max_range, depth_coeff, dropout, seed, frame):
    """Noisy images [N, H, W] from clean ones [N, H, W] (see the module readings)."""
    clean = np.asarray(clean, dtype=np.float64)
    n_views, height, width = clean.shape
    n, r = image_noise(n_views, width, height, seed, frame)
    return noisy_depths(clean, n, r, max_range, depth_coeff, dropout)
