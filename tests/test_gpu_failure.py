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
