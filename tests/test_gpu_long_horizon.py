"""Horizons longer than one chunk of the rollout kernel's scans (64 steps: 32 lanes x 2 steps
with a warp per rollout, 16 lanes x 4 steps with a half warp), so that the state carried from
chunk to chunk (position, velocity, attitude at the chunk's end) is on the tested path, in both
lane layouts and with a ragged last chunk; analytic SDF, against the FP64 oracle.

Tolerances: a position is a sum of up to H per-step increments in FP32, so its error grows
with the horizon: the 5e-5 m of the H = 50 parity tests scaled by H / 50, plus 1e-6 of |p|.
The cost parts keep the 1e-4 relative bound.  The controls are checked against a first-order
bound derived from the measured cost errors: with dJ = max_k |J_k(GPU) - J_k(oracle)|, every
log-weight moves by at most 2 dJ / lambda, so |dU_h| <= (2 dJ / lambda) max_k |U_k,h| (+ 1e-4)."""
import numpy as np
import pytest

import workloads as W
from oracle import mppi as O
from paper_2603_07199_gb300 import binding as B

from .gpu_helpers import GpuController, cost_scale

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("K,H", [(1000, 150), (8193, 70)])
def test_long_horizon_rollouts_against_the_oracle(K, H):
    wl = W.hover_gate()
    prm = dict(wl["params"], K=K, H=H)
    g = GpuController(wl, "analytic", prm)
    try:
        nominal = W.hover_nominal(H)
        out = g.step(state=wl["state"], nominal=nominal)
        ref = O.mppi_step(wl["state"], nominal, wl["poses"], O.Params(**prm), 0)
        pos = g.read(B.MPPI_BUF_POSITIONS)[..., :3].astype(np.float64)
        tol = 5e-5 * H / 50.0 + 1e-6 * np.abs(ref["positions"])
        err = np.abs(pos - ref["positions"])
        print(f"K={K} H={H}: max position error {err.max():.2e} m, |p| up to {np.abs(ref['positions']).max():.1f} m")
        assert np.all(err <= tol), float(np.max(err / tol))
        parts = g.read(B.MPPI_BUF_COST_PARTS).astype(np.float64)
        scale = cost_scale(ref) + 1e-7
        for i, key in enumerate(("J_col", "J_prog", "J_ctl")):
            assert np.all(np.abs(parts[i] - ref[key]) <= 1e-4 * scale), key
        dJ = float(np.max(np.abs(out["J"].astype(np.float64) - ref["J"])))
        bound = (2.0 * dJ / prm["lam"]) * np.max(np.abs(ref["U"]), axis=0) + 1e-4
        assert 2.0 * dJ / prm["lam"] < 0.1, dJ                      # the first-order bound applies
        assert np.all(np.abs(out["U_new"] - ref["U_new"]) <= bound)
        assert abs(float(out["weights"].astype(np.float64).sum()) - 1.0) < 1e-5
    finally:
        g.close()
