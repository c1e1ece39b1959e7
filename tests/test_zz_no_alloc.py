"""The allocation-free update entry point, against the FP64 oracle and the regular control step.

mppi_softmax_update_noalloc serves callers that cannot allocate device memory
(code inside a CUDA stream capture, real-time loops that forbid allocation
after start-up, hosts whose device memory belongs to another allocator): it
takes the costs, the noise and the nominal sequence from the caller and keeps
its only scratch in a static device array.  Its outputs are checked against
the oracle's Eq. 5 weights and update computed in FP64 from the same costs,
noise and nominal sequence, and against mppi_step's own update.  This file is
collected last so a run that stops at the first failure has run every other
test first.
"""
import numpy as np
import pytest

import workloads as W
from oracle import mppi as O
from paper_2603_07199_gb300 import binding as B

from .gpu_helpers import GpuController

pytestmark = pytest.mark.gpu

CTRL_ATOL = 1e-4     # the control tolerance of the parity tests (N, rad/s)
W_ATOL = 1e-5        # the weight tolerance of the parity tests


def _oracle_update(J, noise_hk, nominal, prm):
    """Eq. 5 in FP64 from the caller's inputs: weights from J, U*_new from the clipped samples."""
    w = O.softmax_weights(np.asarray(J, np.float64), prm.lam)
    delta = np.asarray(noise_hk, np.float64).transpose(1, 0, 2)            # [K][H][4]
    U = O.clip_controls(np.asarray(nominal, np.float64)[None, :, :] + delta, prm)
    return w, O.weighted_update(w, U)


def _call(torch, J, noise_hk, nominal, prm, with_weights, stream):
    dev = torch.device("cuda")
    K, H = J.shape[0], nominal.shape[0]
    dJ = torch.from_numpy(np.ascontiguousarray(J, np.float32)).to(dev)
    dnoise = torch.from_numpy(np.ascontiguousarray(noise_hk, np.float32)).to(dev)
    dnom = torch.from_numpy(np.ascontiguousarray(nominal, np.float32)).to(dev)
    dU = torch.full((H, 4), float("nan"), device=dev)
    dw = torch.full((K,), float("nan"), device=dev) if with_weights else None
    B.mppi_softmax_update_noalloc(dJ, dnoise, dnom, K, H, prm.lam, prm.thrust_min, prm.thrust_max, prm.rate_max,
                                  dU, dw, stream)
    torch.cuda.synchronize()
    return dU.cpu().numpy(), None if dw is None else dw.cpu().numpy()


def test_noalloc_update_matches_mppi_step_on_two_calls(lib):
    import torch
    wl = W.two_gate_mlp()
    K, H = 1000, 12
    prm = dict(wl["params"], K=K, H=H)
    oprm = O.Params(**prm)
    g = GpuController(wl, "fp32", prm)
    stream = torch.cuda.current_stream().cuda_stream
    try:
        for call in range(2):
            # first call from the given start, second from the device-resident warm start
            nominal = W.hover_nominal(H) if call == 0 else g.nominal()
            out = g.step(state=wl["state"] if call == 0 else None, nominal=nominal if call == 0 else None)
            J = g.read(B.MPPI_BUF_COSTS)
            # the step's noise ([k][h][4]) in the [h][k][4] layout the entry point takes
            noise = np.ascontiguousarray(g.read(B.MPPI_BUF_NOISE).transpose(1, 0, 2))
            U, w = _call(torch, J, noise, nominal, oprm, True, stream)
            w_ref, U_ref = _oracle_update(J, noise, nominal, oprm)
            np.testing.assert_allclose(U, U_ref, atol=CTRL_ATOL, rtol=0)
            np.testing.assert_allclose(w, w_ref, atol=W_ATOL, rtol=0)
            np.testing.assert_allclose(U, out["U_new"], atol=CTRL_ATOL, rtol=0)
            np.testing.assert_allclose(w, out["weights"], atol=W_ATOL, rtol=0)
    finally:
        g.close()


@pytest.mark.parametrize("K,H,with_weights", [(4096, 50, True), (B.MPPI_NOALLOC_MAX_K, 8, True), (1000, 12, False)])
def test_noalloc_update_matches_oracle(lib, K, H, with_weights):
    """Seeded synthetic costs and noise at the bench size, at the largest K the scratch allows
    (1024 partials: the strided loops over the partials), and without the weights output."""
    import torch
    prm = O.Params(**dict(W.two_gate_mlp()["params"], K=K, H=H))
    rng = np.random.default_rng(1234 + K + H)
    J = rng.uniform(0.0, 4.0, K).astype(np.float32)
    noise = (rng.standard_normal((H, K, 4)) * np.array([2.0, 1.5, 1.5, 1.5])).astype(np.float32)
    nominal = W.hover_nominal(H)
    U, w = _call(torch, J, noise, nominal, prm, with_weights, torch.cuda.current_stream().cuda_stream)
    w_ref, U_ref = _oracle_update(J, noise, nominal, prm)
    np.testing.assert_allclose(U, U_ref, atol=CTRL_ATOL, rtol=0)
    if with_weights:
        np.testing.assert_allclose(w, w_ref, atol=W_ATOL, rtol=0)


def test_noalloc_rejects_misaligned_buffers(lib):
    """A float4 buffer 4 bytes off a 16-byte boundary is refused on the host: nothing is enqueued,
    so the outputs keep their contents."""
    import torch
    K, H = 256, 4
    dev = torch.device("cuda")
    dJ = torch.zeros(K, device=dev)
    noise = torch.zeros(H * K * 4 + 4, device=dev)
    nom = torch.zeros(H * 4 + 4, device=dev)
    dU = torch.full((H * 4 + 4,), float("nan"), device=dev)
    good = (noise.data_ptr(), nom.data_ptr(), dU.data_ptr())
    for which in range(3):
        ptrs = list(good)
        ptrs[which] += 4
        with pytest.raises(B.MppiError) as e:
            B.mppi_softmax_update_noalloc(dJ, ptrs[0], ptrs[1], K, H, 0.1, 0.0, 30.0, 8.0, ptrs[2], None, None)
        assert e.value.code == B.MPPI_E_INVALID
        assert "16-byte aligned" in B.mppi_last_error(None)
    torch.cuda.synchronize()
    assert torch.isnan(dU).all()


def test_noalloc_rejects_k_beyond_its_maximum(lib):
    # rejected on the host before anything is enqueued, so the placeholder pointers are never used
    with pytest.raises(B.MppiError) as e:
        B.mppi_softmax_update_noalloc(16, 16, 16, B.MPPI_NOALLOC_MAX_K + 1, 4, 0.1, 0.0, 30.0, 8.0, 16, None, None)
    assert e.value.code == B.MPPI_E_INVALID
    assert "MPPI_NOALLOC_MAX_K" in B.mppi_last_error(None)
