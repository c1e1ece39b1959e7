"""The allocation-free update entry point against the regular control step.

mppi_softmax_update_noalloc serves callers that cannot allocate device memory
(code inside a CUDA stream capture, real-time loops that forbid allocation
after start-up, hosts whose device memory belongs to another allocator): it
takes the costs, the noise and the nominal sequence from the caller and keeps
its only scratch in a static device array.  This file is collected last so a
run that stops at the first failure has run every other test first.
"""
import numpy as np
import pytest

import workloads as W
from paper_2603_07199_gb300 import binding as B

from .gpu_helpers import GpuController

pytestmark = pytest.mark.gpu

CTRL_ATOL = 1e-4     # the control tolerance of the parity tests (N, rad/s)
W_ATOL = 1e-5        # the weight tolerance of the parity tests


def test_noalloc_update_matches_mppi_step_on_two_calls(lib):
    import torch
    wl = W.two_gate_mlp()
    K, H = 1000, 12
    prm = dict(wl["params"], K=K, H=H)
    g = GpuController(wl, "fp32", prm)
    dev = torch.device("cuda")
    stream = torch.cuda.current_stream().cuda_stream
    try:
        for call in range(2):
            # first call from the given start, second from the device-resident warm start
            nominal = W.hover_nominal(H) if call == 0 else g.nominal()
            out = g.step(state=wl["state"] if call == 0 else None, nominal=nominal if call == 0 else None)
            J = g.read(B.MPPI_BUF_COSTS)
            # the step's noise ([k][h][4]) in the [h][k][4] layout the entry point takes
            noise = np.ascontiguousarray(g.read(B.MPPI_BUF_NOISE).transpose(1, 0, 2))
            dJ = torch.from_numpy(J).to(dev)
            dnoise = torch.from_numpy(noise).to(dev)
            dnom = torch.from_numpy(np.ascontiguousarray(nominal, dtype=np.float32)).to(dev)
            dU = torch.full((H, 4), float("nan"), device=dev)
            dw = torch.full((K,), float("nan"), device=dev)
            B.mppi_softmax_update_noalloc(dJ, dnoise, dnom, K, H, prm["lam"], prm["thrust_min"], prm["thrust_max"],
                                          prm["rate_max"], dU, dw, stream)
            torch.cuda.synchronize()
            np.testing.assert_allclose(dU.cpu().numpy(), out["U_new"], atol=CTRL_ATOL, rtol=0)
            np.testing.assert_allclose(dw.cpu().numpy(), out["weights"], atol=W_ATOL, rtol=0)
    finally:
        g.close()


def test_noalloc_rejects_k_beyond_its_maximum(lib):
    # rejected on the host before anything is enqueued, so the placeholder pointers are never used
    with pytest.raises(B.MppiError) as e:
        B.mppi_softmax_update_noalloc(16, 16, 16, B.MPPI_NOALLOC_MAX_K + 1, 4, 0.1, 0.0, 30.0, 8.0, 16, None, None)
    assert e.value.code == B.MPPI_E_INVALID
    assert "MPPI_NOALLOC_MAX_K" in B.mppi_last_error(None)
