"""GPU parity of the rotor-thrust-rate model (Sec. IV-A, oracle.rotor) against the FP64 oracle.

FP32 bars as in the parity tests: positions 5e-5 m, per-rollout cost 1e-4 relative to the
magnitude of its terms, controls 1e-4 absolute (N/s).
"""
import numpy as np
import pytest

import workloads as W
from oracle import mppi as O
from paper_2603_07199_gb300 import binding as B

from .gpu_helpers import GpuController, cost_scale
from .test_gpu_parity import COST_RTOL, CTRL_ATOL, POS_ATOL, _bf16_errors, _report

pytestmark = pytest.mark.gpu


def _check(out, ref, g=None):
    err = np.abs(out["J"].astype(np.float64) - ref["J"])
    bound = COST_RTOL * cost_scale(ref) + 1e-6
    assert np.all(err <= bound), f"max cost err {err.max():.3e}, worst ratio {np.max(err / bound):.2f}"
    np.testing.assert_allclose(out["U_new"], ref["U_new"], atol=CTRL_ATOL, rtol=0)
    if g is not None:
        pos = g.read(B.MPPI_BUF_POSITIONS)[..., :3].astype(np.float64)
        np.testing.assert_allclose(pos, ref["positions"], atol=POS_ATOL, rtol=0)


def _start():
    return W.rotor_state([-4.0, 0.2, -0.1], yaw=0.3, rates=(0.4, -0.3, 0.2), thrust_offsets=(0.3, -0.2, 0.1, -0.1))


@pytest.mark.parametrize("cost", ["configured", "paper"])
def test_rotor_analytic_step(cost):
    wl = W.hover_gate()
    prm = W.rotor_params(256, 20, **(dict(cost_mode="paper", d_safe=1.0) if cost == "paper" else {}))
    g = GpuController(wl, "analytic", prm)
    try:
        s = _start()
        out = g.step(state=s, nominal=np.zeros((20, 4), np.float32))
        ref = O.mppi_step(s, np.zeros((20, 4)), wl["poses"], O.Params(**prm), 0)
        _check(out, ref, g)
        noise = g.read(B.MPPI_BUF_NOISE).astype(np.float64)
        np.testing.assert_allclose(noise, ref["delta"], atol=4e-6 * prm["sigma_tdot"] * 6, rtol=0)
    finally:
        g.close()


def test_rotor_closed_loop_teacher_forced():
    wl = W.hover_gate()
    prm = W.rotor_params(512, 16)
    g = GpuController(wl, "analytic", prm)
    try:
        state, nominal = _start(), np.zeros((16, 4), np.float32)
        for step in range(5):
            s_gpu = g.state() if step > 0 else state
            n_gpu = g.nominal() if step > 0 else nominal
            out = g.step(state=None if step > 0 else state, nominal=None if step > 0 else nominal)
            ref = O.mppi_step(s_gpu, n_gpu, wl["poses"], O.Params(**prm), step)
            _check(out, ref)
            nxt, _ = O.receding_horizon(s_gpu.astype(np.float64), ref["U_new"], O.Params(**prm))
            assert s_gpu.shape == (17,)
        # the plant update of the last step, against the oracle's rotor step from the same inputs
        s_after = g.state().astype(np.float64)
        nxt, _ = O.receding_horizon(s_gpu.astype(np.float64), out["U_new"].astype(np.float64), O.Params(**prm))
        np.testing.assert_allclose(s_after, nxt, atol=2e-5, rtol=0)
    finally:
        g.close()


@pytest.mark.parametrize("K,H", [(300, 6), (4096, 50)])
def test_rotor_mlp_fp32(K, H):
    wl = W.two_gate_mlp()
    prm = W.rotor_params(K, H)
    s = W.rotor_state([0.3, -0.2, 0.1], yaw=-0.2, rates=(0.1, 0.2, -0.1))
    g = GpuController(wl, "fp32", prm)
    try:
        out = g.step(state=s, nominal=np.zeros((H, 4), np.float32))
        ref = O.mppi_step(s, np.zeros((H, 4)), wl["poses"], O.Params(**prm), 0, wl["latents"], wl["layers"])
        np.testing.assert_allclose(g.read(B.MPPI_BUF_SDF).astype(np.float64), ref["sdf"], atol=2e-5, rtol=0)
        _check(out, ref, g)
    finally:
        g.close()


def test_rotor_bf16_errors():
    wl = W.two_gate_mlp()
    prm = W.rotor_params(4096, 50)
    s = W.rotor_state([0.0, 0.0, 0.0])
    g = GpuController(wl, "bf16", prm)
    try:
        out = g.step(state=s, nominal=np.zeros((50, 4), np.float32))
        ref = O.mppi_step(s, np.zeros((50, 4)), wl["poses"], O.Params(**prm), 0, wl["latents"], wl["layers"])
        err = _bf16_errors(g, ref, out)
        _report("rotor_bf16_K4096_H50", err)
        assert err["sdf_mae_mm"] < 10.0, err
    finally:
        g.close()
