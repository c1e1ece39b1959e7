"""GPU parity of the decoder with positional encoding, g_phi(z, PE(p)) (Sec. III-B), queried
in the cached frame of each gate's latent (the frame the gate pose gives), against the FP64
oracle: the FP32 path at the FP32 bars (SDF 2e-5 m, costs 1e-4 relative, controls 1e-4), the
tensor-core paths' SDF errors reported and bounded."""
import numpy as np
import pytest

import workloads as W
from oracle import mppi as O
from paper_2603_07199_gb300 import binding as B

from .gpu_helpers import GpuController, cost_scale
from .test_gpu_parity import COST_RTOL, CTRL_ATOL, _bf16_errors, _report

pytestmark = pytest.mark.gpu


def _workload(levels):
    wl = dict(W.two_gate_mlp())
    wl["layers"] = W.xavier_mlp(1, in_dim=3 + 6 * levels + 64)
    return wl


@pytest.mark.parametrize("levels,K,H", [(1, 300, 6), (4, 300, 6), (6, 129, 2), (4, 4096, 50)])
def test_pe_fp32_parity(levels, K, H):
    """With several encoding levels the untrained network reports every state inside the
    frame (s < 0), so every state pays the hinge and the query's FP32 rounding, amplified by
    the encoding's frequencies (up to 2^5 pi per metre), reaches J and, through exp(-J /
    lambda), the controls.  The SDF and the costs are held to the FP32 bars; the controls to
    the first-order effect of the measured cost differences on Eq. 5 (plus 1e-4).  w_col = 10
    keeps |J| near the configured workload's size."""
    wl = _workload(levels)
    prm = dict(wl["params"], K=K, H=H, pe_levels=levels, w_col=10.0)
    g = GpuController(wl, "fp32", prm)
    try:
        out = g.step(state=wl["state"], nominal=W.hover_nominal(H))
        ref = O.mppi_step(wl["state"], W.hover_nominal(H), wl["poses"], O.Params(**prm), 0, wl["latents"], wl["layers"])
        np.testing.assert_allclose(g.read(B.MPPI_BUF_SDF).astype(np.float64), ref["sdf"], atol=2e-5, rtol=0)
        dJ = out["J"].astype(np.float64) - ref["J"]
        assert np.all(np.abs(dJ) <= COST_RTOL * cost_scale(ref) + 1e-7), np.abs(dJ).max()
        # Eq. 5 to first order: dU*_h = -sum_k w_k (dJ_k - sum_m w_m dJ_m) / lambda (U_kh - U*_h);
        # the controls must agree up to what the measured cost differences explain, plus 1e-4
        w = ref["weights"]
        dw = -w * (dJ - np.sum(w * dJ)) / prm["lam"]
        explained = np.abs(np.einsum("k,khc->hc", dw, ref["U"] - ref["U_new"][None]))
        np.testing.assert_array_less(np.abs(out["U_new"] - ref["U_new"]), 2.0 * explained + CTRL_ATOL)
    finally:
        g.close()


@pytest.mark.parametrize("mode,bound", [("fp16", 2.0), ("bf16", 15.0), ("fp8", 80.0)])
@pytest.mark.parametrize("levels", [2, 4])
def test_pe_tensor_core_errors(mode, bound, levels):
    wl = _workload(levels)
    prm = dict(wl["params"], K=1024, H=20, pe_levels=levels)
    g = GpuController(wl, mode, prm)
    try:
        out = g.step(state=wl["state"], nominal=W.hover_nominal(20))
        ref = O.mppi_step(wl["state"], W.hover_nominal(20), wl["poses"], O.Params(**prm), 0, wl["latents"], wl["layers"])
        err = _bf16_errors(g, ref, out)
        _report(f"pe{levels}_{mode}_K1024_H20", err)
        assert err["sdf_mae_mm"] < bound, err
    finally:
        g.close()


def test_pe_levels_out_of_range_are_rejected():
    cfg = B.mppi_config_default()
    cfg.pe_levels = B.MPPI_MAX_PE_LEVELS + 1
    with pytest.raises(B.MppiError) as e:
        B.mppi_create(cfg)
    assert e.value.code == B.MPPI_E_INVALID
