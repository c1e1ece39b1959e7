"""Failure detection on the GPU without a fault: the update kernel's grid barrier is a bounded
wait (2 s of %globaltimer).  mppi_debug_inject_timeout makes the next step's blocks wait for
arrivals that never come; each gives up, sets the device error word and returns, the step
reports MPPI_E_TIMEOUT, and the context then steps exactly like a fresh one."""
import time

import numpy as np
import pytest

import workloads as W
from paper_2603_07199_gb300 import binding as B

from .gpu_helpers import GpuController

pytestmark = pytest.mark.gpu


def _controller():
    wl = W.two_gate_mlp()
    return wl, GpuController(wl, "bf16", W.params(1024, 20))


def test_barrier_timeout_is_reported_and_the_context_recovers():
    wl, ctl = _controller()
    ref_wl, ref = _controller()
    try:
        ctl.step(wl["state"], W.hover_nominal(20))
        B.mppi_debug_inject_timeout(ctl.ctx)
        t0 = time.perf_counter()
        with pytest.raises(B.MppiError) as e:
            ctl.step(wl["state"], W.hover_nominal(20))
        waited = time.perf_counter() - t0
        assert e.value.code == B.MPPI_E_TIMEOUT, e.value
        assert 1.5 < waited < 30.0, waited
        # recovered: the same step as a fresh context (same counter, state, warm start), bit for bit
        for c in (ctl, ref):
            B.mppi_set_step_counter(c.ctx, 7)
        out = ctl.step(wl["state"], W.hover_nominal(20))
        want = ref.step(wl["state"], W.hover_nominal(20))
        np.testing.assert_array_equal(out["U_new"], want["U_new"])
        np.testing.assert_array_equal(out["weights"], want["weights"])
        np.testing.assert_array_equal(ctl.state(), ref.state())
    finally:
        ctl.close()
        ref.close()


def test_barrier_timeout_through_the_async_path():
    import torch
    wl, ctl = _controller()
    try:
        U = torch.zeros(20, 4, device="cuda")
        ctl.step(wl["state"], W.hover_nominal(20))
        B.mppi_debug_inject_timeout(ctl.ctx)
        B.mppi_step_async(ctl.ctx, None, None, None, None, U, None, None)
        with pytest.raises(B.MppiError) as e:
            B.mppi_sync(ctl.ctx)
        assert e.value.code == B.MPPI_E_TIMEOUT
        B.mppi_step_async(ctl.ctx, None, None, None, None, U, None, None)
        B.mppi_sync(ctl.ctx)
        assert torch.isfinite(U).all()
    finally:
        ctl.close()


def test_encoder_tensor_core_wait_timeout_is_reported_and_recovers():
    """The tensor-core convolutions' waits are bounded too: with the test hook, every CTA of the
    next encoding's first convolution waits for a barrier phase that never completes, gives up
    after 2 s, sets the encoder's error word and returns; mppi_encoder_check reports
    MPPI_E_TIMEOUT once, and the next encoding equals one from before, bit for bit."""
    import torch
    layers = []
    for Wm, b in W.encoder_weights(7):
        layers += [np.ascontiguousarray(Wm, np.float32), np.ascontiguousarray(b, np.float32)]
    rng = np.random.default_rng(3)
    d = torch.from_numpy(rng.uniform(0.5, 9.5, (1, 120, 160)).astype(np.float32)).cuda()
    z = torch.zeros(1, 64, device="cuda")
    enc = B.mppi_encoder_create(120, 160, 1, layers)     # one image: the first layer is one wave of CTAs
    try:
        B.mppi_encode_depth(enc, 1, d, 10.0, z)
        assert B.mppi_encoder_check(enc) == B.MPPI_OK
        want = z.cpu().numpy().copy()
        B.mppi_encoder_debug_inject_timeout(enc)
        t0 = time.perf_counter()
        B.mppi_encode_depth(enc, 1, d, 10.0, z)
        with pytest.raises(B.MppiError) as e:
            B.mppi_encoder_check(enc)
        waited = time.perf_counter() - t0
        assert e.value.code == B.MPPI_E_TIMEOUT, e.value
        assert 1.5 < waited < 30.0, waited
        assert B.mppi_encoder_check(enc) == B.MPPI_OK       # reported once
        B.mppi_encode_depth(enc, 1, d, 10.0, z)
        assert B.mppi_encoder_check(enc) == B.MPPI_OK
        np.testing.assert_array_equal(z.cpu().numpy(), want)
        B.mppi_encoder_set_conv_path(enc, B.MPPI_ENC_CONV_FP32)
        with pytest.raises(B.MppiError) as e:
            B.mppi_encoder_debug_inject_timeout(enc)
        assert e.value.code == B.MPPI_E_INVALID
    finally:
        B.mppi_encoder_destroy(enc)


def test_encoder_trainer_reports_a_tensor_core_timeout():
    """The trainer's forward pass is the encoder's: after the hook, a training step that reads its
    loss reports MPPI_E_TIMEOUT (and applies no Adam step); the next step runs normally."""
    import torch
    layers = []
    for Wm, b in W.encoder_weights(7):
        layers += [np.ascontiguousarray(Wm, np.float32), np.ascontiguousarray(b, np.float32)]
    rng = np.random.default_rng(4)
    noisy = torch.from_numpy(rng.uniform(0.5, 9.5, (1, 48, 64)).astype(np.float32)).cuda()
    clean = torch.from_numpy(rng.uniform(0.5, 9.5, (1, 48, 64)).astype(np.float32)).cuda()
    enc = B.mppi_encoder_create(48, 64, 1, layers)
    T = 6 * 8
    tr = B.mppi_encoder_train_create(enc, 1, 1e-3, rng.normal(0, 0.1, (T, 64)).astype(np.float32),
                                     np.zeros(T, np.float32))
    try:
        l0 = B.mppi_encoder_train_loss_grads(tr, 1, noisy, clean, 10.0)
        B.mppi_encoder_debug_inject_timeout(enc)
        with pytest.raises(B.MppiError) as e:
            B.mppi_encoder_train_step(tr, 1, noisy, clean, 10.0)
        assert e.value.code == B.MPPI_E_TIMEOUT, e.value
        assert B.mppi_encoder_train_loss_grads(tr, 1, noisy, clean, 10.0) == l0   # no update was applied
        assert np.isfinite(B.mppi_encoder_train_step(tr, 1, noisy, clean, 10.0))
    finally:
        B.mppi_encoder_train_destroy(tr)
        B.mppi_encoder_destroy(enc)
