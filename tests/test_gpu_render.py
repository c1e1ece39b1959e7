"""GPU parity of the depth renderer (the onboard depth observation of Sec. III-B) and of its
sensor noise against the FP64 oracle, through the C ABI.

Depth tolerance: on pixels whose depth is well conditioned -- where growing and shrinking the
frame by 0.1 mm moves the oracle's depth by at most 1 mm -- the FP32 kernel must match within
1e-4 m + 1e-5 z (its rounding of the 10-20 m coordinates is about 1e-6 m, times at most 10 for
that conditioning).  On the other pixels (rays that graze an edge or a face) any depth between
the grown and the shrunk frame's is correct, since rounding may move such a ray across the
edge; those must lie in that bracket (widened by 1e-4 m).  Dropout decisions are bit-exact
(24-bit uniforms compared in FP32 on both sides)."""
import numpy as np
import pytest

import workloads as W
from oracle import render as R
from paper_2603_07199_gb300 import binding as B

pytestmark = pytest.mark.gpu

EPS = 1e-4          # frame grown / shrunk by this much (m)
COND = 1e-3         # a pixel is well conditioned when the two differ by at most this (m)
ATOL, RTOL = 1e-4, 1e-5


def _torch():
    import torch
    return torch


def _camera(kw, noise=0.0, dropout=0.0, seed=0, frame=0):
    cam = B.mppi_depth_camera_default()
    for k, v in kw.items():
        setattr(cam, k, v)
    cam.noise_depth_coeff = noise
    cam.dropout = dropout
    cam.seed = seed
    cam.frame = frame
    return cam


def _render(cam, cams, gates, offset=0):
    torch = _torch()
    cams = np.ascontiguousarray(cams, dtype=np.float32).reshape(-1, 7)
    gates = np.ascontiguousarray(gates, dtype=np.float32).reshape(-1, 7)
    n = cams.shape[0]
    d_cams = torch.from_numpy(cams).cuda()
    d_gates = torch.from_numpy(gates).cuda() if len(gates) else None
    buf = torch.full((n * cam.height * cam.width + offset,), -1.0, dtype=torch.float32, device="cuda")
    B.mppi_render_depth(cam, n, d_cams, len(gates), d_gates, buf.data_ptr() + 4 * offset)
    torch.cuda.synchronize()
    return buf[offset:].cpu().numpy().reshape(n, cam.height, cam.width)


def _frames(kw):
    return dict(a_in=kw.get("gate_inner_half", 0.5), a_out=kw.get("gate_outer_half", 0.75),
                d=kw.get("gate_half_depth", 0.1))


def _oracle_triplet(cams, gates, kw):
    """Oracle depth images with the frame as given, grown by EPS and shrunk by EPS."""
    f = _frames(kw)
    geo = dict(width=kw["width"], height=kw["height"], fx=kw["fx"], fy=kw["fy"], cx=kw["cx"], cy=kw["cy"],
               max_range=kw["max_range"])
    base = R.depth_images(cams, gates, **geo, **f)
    grown = R.depth_images(cams, gates, **geo, a_in=f["a_in"] - EPS, a_out=f["a_out"] + EPS, d=f["d"] + EPS)
    shrunk = R.depth_images(cams, gates, **geo, a_in=f["a_in"] + EPS, a_out=f["a_out"] - EPS, d=f["d"] - EPS)
    return base, grown, shrunk


def _check_depth(got, base, grown, shrunk, name):
    good = (shrunk - grown) <= COND
    err = np.abs(got - base)
    tol = ATOL + RTOL * base
    bad = good & (err > tol)
    assert not bad.any(), f"{name}: {bad.sum()} well-conditioned pixels off, worst {err[good].max():.3e} m"
    inb = (got >= grown - ATOL) & (got <= shrunk + ATOL)
    assert inb.all(), f"{name}: {np.count_nonzero(~inb)} pixels outside the grown / shrunk bracket"
    assert np.isfinite(got).all()
    return dict(max_err=float(err[good].max(initial=0.0)), ill=int(np.count_nonzero(~good)), n=got.size)


SMALL = [dict(width=256, height=120, fx=150.0, fy=150.0, cx=128.0, cy=60.0, max_range=10.0),   # float4 stores
         dict(width=203, height=97, fx=118.3, fy=121.7, cx=97.2, cy=51.3, max_range=12.0),     # ragged, scalar
         dict(width=37, height=9, fx=20.0, fy=24.0, cx=18.1, cy=4.4, max_range=8.0)]


@pytest.mark.parametrize("kw", SMALL, ids=["256x120", "203x97", "37x9"])
def test_render_parity(kw):
    gates = W.gate_track(3, seed=13)
    cams = W.camera_views(6, gates, seed=21)
    got = _render(_camera(kw), cams, gates)
    base, grown, shrunk = _oracle_triplet(cams, gates, kw)
    rep = _check_depth(got, base, grown, shrunk, "clean")
    assert np.count_nonzero(base < kw["max_range"]) > 0
    print("render parity", kw["width"], kw["height"], rep)


def test_render_other_frame_geometry():
    kw = dict(SMALL[0], gate_inner_half=0.4, gate_outer_half=0.9, gate_half_depth=0.05)
    gates = W.gate_track(2, seed=4)
    cams = W.camera_views(4, gates, seed=5)
    got = _render(_camera(kw), cams, gates)
    _check_depth(got, *_oracle_triplet(cams, gates, kw), "geometry")


def test_render_unaligned_output_matches():
    kw = SMALL[0]
    gates = W.gate_track(2, seed=13)
    cams = W.camera_views(3, gates, seed=8)
    a = _render(_camera(kw), cams, gates)
    b = _render(_camera(kw), cams, gates, offset=1)     # 4-byte aligned only: the scalar-store kernel
    np.testing.assert_array_equal(a, b)


@pytest.mark.parametrize("noise,dropout", [(0.005, 0.0), (0.0, 0.05), (0.02, 0.1)])
def test_render_noise_parity(noise, dropout):
    kw = SMALL[1]
    gates = W.gate_track(3, seed=13)
    cams = W.camera_views(5, gates, seed=22)
    got = _render(_camera(kw, noise, dropout, seed=77, frame=5), cams, gates)
    base, grown, shrunk = _oracle_triplet(cams, gates, kw)
    want = R.add_sensor_noise(base, kw["max_range"], noise, dropout, seed=77, frame=5)
    _, u = R.image_noise(len(cams), kw["width"], kw["height"], 77, 5)
    drop = u < np.float32(dropout)
    np.testing.assert_array_equal(got[drop], 0.0)
    good = ((shrunk - grown) <= COND) & ~drop
    err = np.abs(got - want)
    assert np.all(err[good] <= 2 * ATOL + RTOL * want[good]), err[good].max()
    if dropout > 0:
        assert drop.sum() > 0
    # undropped pixels of either frame state: noisy depths stay in range
    assert np.all((got >= 0.0) & (got <= kw["max_range"]))


def test_render_full_size_sampled():
    """The 64-view 640 x 480 workload in the launch the bench times, clean and noisy: 4096
    sampled pixels against the oracle's per-pixel depths."""
    wl = W.depth_views()
    kw = wl["camera"]
    cams, gates = wl["cams"], wl["gates"]
    clean = _render(_camera(kw), cams, gates)
    noisy = _render(_camera(kw, wl["noise_depth_coeff"], wl["dropout"], wl["seed"], wl["frame"]), cams, gates)
    rng = np.random.default_rng(0)
    # half the samples on pixels the kernel saw a frame in, half anywhere
    hits = np.argwhere(clean < kw["max_range"])
    pick = np.concatenate([hits[rng.integers(len(hits), size=2048)],
                           np.stack([rng.integers(64, size=2048), rng.integers(kw["height"], size=2048),
                                     rng.integers(kw["width"], size=2048)], 1)])
    geo = dict(fx=kw["fx"], fy=kw["fy"], cx=kw["cx"], cy=kw["cy"], max_range=kw["max_range"])
    n_checked = 0
    for view in np.unique(pick[:, 0]):
        sel = pick[pick[:, 0] == view]
        vs, us = sel[:, 1], sel[:, 2]
        base = R.pixel_depths(cams[view], gates, us, vs, **geo)
        grown = R.pixel_depths(cams[view], gates, us, vs, **geo, a_in=0.5 - EPS, a_out=0.75 + EPS, d=0.1 + EPS)
        shrunk = R.pixel_depths(cams[view], gates, us, vs, **geo, a_in=0.5 + EPS, a_out=0.75 - EPS, d=0.1 - EPS)
        _check_depth(clean[view, vs, us], base, grown, shrunk, f"view {view}")
        n_checked += len(sel)
    assert n_checked == 4096
    # noise at the sampled pixels: dropout decisions exact, noisy depths within tolerance
    view, vs, us = pick[:, 0], pick[:, 1], pick[:, 2]
    n, r = R.pixel_noise(vs * kw["width"] + us, view, wl["seed"], wl["frame"])
    base = np.concatenate([R.pixel_depths(cams[v], gates, us[view == v], vs[view == v], **geo) for v in range(64)])
    order = np.concatenate([np.nonzero(view == v)[0] for v in range(64)])
    want = np.empty(len(pick))
    want[order] = R.noisy_depths(base, n[order], r[order], kw["max_range"], wl["noise_depth_coeff"], wl["dropout"])
    drop = r < np.float32(wl["dropout"])
    got = noisy[view, vs, us]
    np.testing.assert_array_equal(got[drop], 0.0)
    err = np.abs(got - want)
    close = err <= 2 * ATOL + RTOL * want
    assert np.count_nonzero(~close) <= 8, err[~close]          # only ill-conditioned edge pixels may differ
    assert abs(np.mean(noisy == 0.0) - wl["dropout"]) < 2e-3


def test_render_edge_cases():
    torch = _torch()
    kw = SMALL[2]
    cam = _camera(kw)
    gate = W.origin_gate()
    # no gates: every pixel reads max_range
    got = _render(cam, W.camera_views(2, gate, seed=1), np.zeros((0, 7)))
    assert np.all(got == kw["max_range"])
    # a camera inside a post reads 0 everywhere
    inside = np.array([[0.0, 0.6, 0.0, 1.0, 0.0, 0.0, 0.0]], dtype=np.float32)
    assert np.all(_render(cam, inside, gate) == 0.0)
    # one pixel
    one = _camera(dict(width=1, height=1, fx=10.0, fy=10.0, cx=0.5, cy=0.5, max_range=10.0))
    front = np.array([[-3.0, 0.0, 0.625, 1.0, 0.0, 0.0, 0.0]], dtype=np.float32)    # axis hits the top bar
    assert abs(_render(one, front, gate)[0, 0, 0] - 2.9) < 1e-5
    # zero views enqueue nothing
    buf = torch.full((4,), 7.0, device="cuda")
    B.mppi_render_depth(cam, 0, None, 1, None, buf)
    torch.cuda.synchronize()
    assert torch.all(buf == 7.0)
    # invalid arguments are rejected with MPPI_E_INVALID before any launch
    d_cam = torch.zeros(7, device="cuda")
    for field, value in [("width", 0), ("height", B.MPPI_MAX_IMAGE_SIDE + 1), ("fx", 0.0), ("max_range", -1.0),
                         ("dropout", 1.5), ("noise_depth_coeff", -0.1), ("gate_inner_half", 0.8), ("reserved", 1)]:
        bad = _camera(kw)
        setattr(bad, field, value)
        with pytest.raises(B.MppiError) as e:
            B.mppi_render_depth(bad, 1, d_cam, 0, None, buf)
        assert e.value.code == B.MPPI_E_INVALID
    with pytest.raises(B.MppiError):
        B.mppi_render_depth(cam, 1, d_cam, B.MPPI_MAX_RENDER_GATES + 1, d_cam, buf)
    with pytest.raises(B.MppiError):
        B.mppi_render_depth(cam, 1, None, 0, None, buf)


def test_render_many_gates_and_extreme_shapes():
    """40 gates (the per-warp gate masks span two 32-lane ballots), an axis-aligned camera whose
    rays run exactly parallel to slab planes, and images of 8192 x 2 and 3 x 8192 pixels."""
    rng = np.random.default_rng(5)
    gates = np.zeros((40, 7), np.float32)
    gates[:, 0] = rng.uniform(3.0, 25.0, 40)
    gates[:, 1] = rng.uniform(-6.0, 6.0, 40)
    gates[:, 2] = rng.uniform(-3.0, 3.0, 40)
    yaw = rng.uniform(-0.8, 0.8, 40)
    gates[:, 3] = np.cos(yaw / 2)
    gates[:, 6] = np.sin(yaw / 2)
    kw = dict(width=160, height=96, fx=80.0, fy=80.0, cx=80.0, cy=48.0, max_range=30.0)
    cams = np.array([[0.0, 0.0, 0.0, 1.0, 0.0, 0.0, 0.0], [1.0, -0.5, 0.3, 0.995, 0.0, 0.0, 0.0998]], np.float32)
    got = _render(_camera(kw), cams, gates)
    rep = _check_depth(got, *_oracle_triplet(cams, gates, kw), "40 gates")
    assert np.mean(got < kw["max_range"]) > 0.05
    # axis-aligned: a gate straight ahead, camera on its axis; pixel centres on the principal
    # point's row and column give ray components exactly 0 in the gate frame
    kw2 = dict(width=65, height=33, fx=20.0, fy=20.0, cx=32.5, cy=16.5, max_range=10.0)
    ahead = np.array([[4.0, 0.0, 0.0, 1.0, 0.0, 0.0, 0.0]], np.float32)
    cam0 = np.array([[0.0, 0.0, 0.0, 1.0, 0.0, 0.0, 0.0]], np.float32)
    got2 = _render(_camera(kw2), cam0, ahead)
    _check_depth(got2, *_oracle_triplet(cam0, ahead, kw2), "axis-aligned")
    for shape in [(8192, 2), (3, 8192)]:
        kw3 = dict(width=shape[0], height=shape[1], fx=1200.0, fy=1200.0, cx=shape[0] / 2, cy=shape[1] / 2,
                   max_range=12.0)
        got3 = _render(_camera(kw3), cams[:1], gates)
        _check_depth(got3, *_oracle_triplet(cams[:1], gates, kw3), f"{shape}")
    print("many gates", rep)
