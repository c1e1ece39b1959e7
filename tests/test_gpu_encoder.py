"""GPU parity of the depth encoder (the convolutional reading of E_theta, Sec. III-B) against the
FP64 oracle, through the C ABI, on depth images the oracle renders.

Tolerance: each latent is a 64-term dot product of means of FP32 convolution chains whose
sums have at most 9 x 64 terms of O(1); FP32 rounding gives about 1e-6 relative, so
|z_gpu - z_oracle| <= 1e-4 (1 + |z|) leaves a wide margin while catching any wrong tap, channel
or scale.  A ReLU decided differently by rounding changes z by at most the rounding itself.
Both convolution paths are held to that bar: the FP32 CUDA-core GEMMs and the tensor-core
kernels, whose BF16 hi/lo split keeps every product within ~3 x 2^-16 of its FP32 value
(the dropped lo x lo term and the split's own rounding), errors that average out over the
sums instead of adding up."""
import numpy as np
import pytest

import workloads as W
from oracle import encoder as E
from oracle import render as R
from paper_2603_07199_gb300 import binding as B

pytestmark = pytest.mark.gpu

SMALL_CAM = dict(width=160, height=120, fx=96.25, fy=96.25, cx=80.0, cy=60.0, max_range=10.0)


def _torch():
    import torch
    return torch


def _flat(layers):
    out = []
    for Wm, b in layers:
        out += [np.ascontiguousarray(Wm, np.float32), np.ascontiguousarray(b, np.float32)]
    return out


PATHS = {"tc": B.MPPI_ENC_CONV_TC, "fp32": B.MPPI_ENC_CONV_FP32}


def _encode(layers, imgs, max_range, max_images=None, path="tc"):
    torch = _torch()
    imgs = np.ascontiguousarray(imgs, np.float32)
    n, h, w = imgs.shape
    enc = B.mppi_encoder_create(h, w, max_images or max(n, 1), _flat(layers))
    try:
        B.mppi_encoder_set_conv_path(enc, PATHS[path])
        d = torch.from_numpy(imgs).cuda()
        z = torch.full((max(n, 1), 64), 7.0, device="cuda")
        B.mppi_encode_depth(enc, n, d, max_range, z)
        B.mppi_encoder_check(enc)
        torch.cuda.synchronize()
        return z.cpu().numpy()[:n]
    finally:
        B.mppi_encoder_destroy(enc)


def _check(got, want):
    err = np.abs(got - want)
    tol = 1e-4 * (1.0 + np.abs(want))
    assert np.all(err <= tol), f"max err {err.max():.3e}"
    return float(err.max())


def _views(n, kw, seed):
    gates = W.gate_track(2)
    cams = W.camera_views(n, gates, seed=seed)
    return R.depth_images(cams, gates, **kw)


@pytest.mark.parametrize("path", ["tc", "fp32"])
def test_encoder_parity_rendered_views(path):
    layers = W.encoder_weights(7)
    imgs = _views(6, SMALL_CAM, seed=31)
    assert np.mean(imgs < 10.0) > 0.01
    got = _encode(layers, imgs, 10.0, path=path)
    print("encoder", path, "max err", _check(got, E.encode(imgs, 10.0, layers)))


@pytest.mark.parametrize("path", ["tc", "fp32"])
@pytest.mark.parametrize("h,w", [(37, 53), (1, 1), (2, 3), (97, 203)])
def test_encoder_parity_ragged_sizes(h, w, path):
    layers = W.encoder_weights(8)
    rng = np.random.default_rng(h * 1000 + w)
    imgs = rng.uniform(0.0, 12.0, (3, h, w))
    imgs[:, ::3, ::2] = 12.0
    _check(_encode(layers, imgs, 12.0, path=path), E.encode(imgs, 12.0, layers))


@pytest.mark.parametrize("path", ["tc", "fp32"])
def test_encoder_noisy_views_and_full_batch(path):
    """The 64-view batch of the bench at 160 x 120, with sensor noise (depth dropouts read 0)."""
    layers = W.encoder_weights(7)
    clean = _views(64, SMALL_CAM, seed=6)
    noisy = R.add_sensor_noise(clean, 10.0, 0.005, 0.02, seed=9, frame=0)
    got = _encode(layers, noisy, 10.0, path=path)
    print("encoder", path, "64-view max err", _check(got, E.encode(noisy, 10.0, layers)))


def test_encoder_paths_agree_and_tc_batch_is_exact():
    """The tensor-core path computes every output pixel in one CTA over the whole reduction, in
    the same order whatever the batch, so an image's code alone equals its code in a batch bit
    for bit; the two paths agree within the rounding of their different summation orders."""
    layers = W.encoder_weights(9)
    imgs = _views(5, SMALL_CAM, seed=40)
    batch = _encode(layers, imgs, 10.0, max_images=8, path="tc")
    for i in range(5):
        np.testing.assert_array_equal(_encode(layers, imgs[i:i + 1], 10.0, path="tc"), batch[i:i + 1])
    np.testing.assert_allclose(_encode(layers, imgs, 10.0, path="fp32"), batch, rtol=1e-4, atol=1e-4)


def test_encoder_batch_independence_and_errors():
    torch = _torch()
    layers = W.encoder_weights(9)
    imgs = _views(5, SMALL_CAM, seed=40)
    batch = _encode(layers, imgs, 10.0, max_images=8, path="fp32")
    # a batch may split the reductions differently (fewer output tiles -> more split-K
    # slices), so an image's code matches its code alone up to summation order
    for i in range(5):
        np.testing.assert_allclose(_encode(layers, imgs[i:i + 1], 10.0, path="fp32"), batch[i:i + 1], rtol=1e-5,
                                   atol=1e-5)
    np.testing.assert_array_equal(_encode(layers, imgs, 10.0, max_images=8, path="fp32"), batch)  # same bits
    enc = B.mppi_encoder_create(120, 160, 2, _flat(layers))
    try:
        for bad in (-1, 2, 7):
            with pytest.raises(B.MppiError) as e:
                B.mppi_encoder_set_conv_path(enc, bad)
            assert e.value.code == B.MPPI_E_INVALID
        assert B.mppi_encoder_check(enc) == B.MPPI_OK
        d = torch.zeros(3, 120, 160, device="cuda")
        z = torch.zeros(3, 64, device="cuda")
        for args in [(3, d, 10.0, z), (1, d, 0.0, z), (1, None, 10.0, z), (-1, d, 10.0, z)]:
            with pytest.raises(B.MppiError) as e:
                B.mppi_encode_depth(enc, *args)
            assert e.value.code == B.MPPI_E_INVALID
        B.mppi_encode_depth(enc, 0, None, 10.0, None)          # nothing to do
    finally:
        B.mppi_encoder_destroy(enc)
    with pytest.raises(B.MppiError):
        B.mppi_encoder_create(0, 160, 1, _flat(layers))
    with pytest.raises(B.MppiError):
        B.mppi_encoder_create(120, 160, 1, _flat(layers)[:8])


def test_render_then_encode_pipeline():
    """GPU render -> GPU encode against oracle render -> oracle encode.  Rays that graze an edge may
    flip between a hit and a miss under FP32 rounding (a depth jump of metres for that pixel), so
    the bar here is looser (1e-2) than the encoder's own; the report shows the actual error."""
    torch = _torch()
    layers = W.encoder_weights(7)
    gates = W.gate_track(2)
    cams = W.camera_views(8, gates, seed=33)
    cam = B.mppi_depth_camera_default()
    for k, v in SMALL_CAM.items():
        setattr(cam, k, v)
    d_cams = torch.from_numpy(np.ascontiguousarray(cams, np.float32)).cuda()
    d_gates = torch.from_numpy(np.ascontiguousarray(gates, np.float32)).cuda()
    depth = torch.empty(8, 120, 160, device="cuda")
    B.mppi_render_depth(cam, 8, d_cams, 2, d_gates, depth)
    enc = B.mppi_encoder_create(120, 160, 8, _flat(layers))
    try:
        z = torch.empty(8, 64, device="cuda")
        B.mppi_encode_depth(enc, 8, depth, 10.0, z)
        torch.cuda.synchronize()
        got = z.cpu().numpy()
    finally:
        B.mppi_encoder_destroy(enc)
    want = E.encode(R.depth_images(cams, gates, **SMALL_CAM), 10.0, layers)
    err = np.abs(got - want)
    print("render+encode max err", float(err.max()))
    assert np.all(err <= 1e-2 * (1.0 + np.abs(want)))


@pytest.mark.parametrize("path", ["tc", "fp32"])
def test_encoder_parity_full_resolution(path):
    """The renderer's full 640 x 480 views (2,400 output tiles of the first layer per image pair,
    320 x 240 .. 40 x 30 activations): every convolution path against the FP64 encoder."""
    layers = W.encoder_weights(7)
    kw = dict(width=640, height=480, fx=385.0, fy=385.0, cx=320.0, cy=240.0, max_range=10.0)
    imgs = _views(2, kw, seed=12)
    got = _encode(layers, imgs, 10.0, path=path)
    print("encoder", path, "640 x 480 max err", _check(got, E.encode(imgs, 10.0, layers)))
