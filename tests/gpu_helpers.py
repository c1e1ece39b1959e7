"""Test-side helpers: drive the CUDA library through its C-ABI binding and
lay its buffers out like the oracle's arrays."""
import numpy as np

from paper_2603_07199_gb300 import binding as B

MODES = {"analytic": B.MPPI_SDF_ANALYTIC, "fp32": B.MPPI_SDF_MLP_FP32, "bf16": B.MPPI_SDF_MLP_BF16,
         "fp16": B.MPPI_SDF_MLP_FP16, "fp8": B.MPPI_SDF_MLP_FP8}
_KEYS = ("K", "H", "dt", "mass", "gravity", "thrust_min", "thrust_max", "rate_max", "sigma_thrust",
         "sigma_rate", "w_col", "d_safe", "w_u", "seed", "drone_id")


def make_config(prm, mode, max_gates):
    cfg = B.mppi_config_default()
    for key in _KEYS:
        setattr(cfg, key, prm[key])
    cfg.lam = prm["lam"]
    cfg.max_gates = max(1, int(max_gates))
    cfg.sdf_mode = MODES[mode]
    cfg.cost_mode = {"configured": B.MPPI_COST_CONFIGURED, "paper": B.MPPI_COST_PAPER}[prm.get("cost_mode", "configured")]
    for key in ("q_gate", "q_vis", "q_sdf", "guide_tan_alpha"):
        if key in prm:
            setattr(cfg, key, prm[key])
    cfg.dynamics_mode = {"ctbr": B.MPPI_DYN_CTBR, "rotor": B.MPPI_DYN_ROTOR}[prm.get("dynamics", "ctbr")]
    for key in ("tdot_max", "rotor_thrust_max", "sigma_tdot", "arm_length"):
        if key in prm:
            setattr(cfg, key, prm[key])
    if "kappa" in prm:
        cfg.torque_coeff = prm["kappa"]
    if "inertia" in prm:
        cfg.inertia_x, cfg.inertia_y, cfg.inertia_z = prm["inertia"]
    cfg.pe_levels = int(prm.get("pe_levels", 0))
    return cfg


def flat_layers(layers):
    out = []
    for W, b in layers:
        out += [np.ascontiguousarray(W, dtype=np.float32), np.ascontiguousarray(b, dtype=np.float32)]
    return out


class GpuController:
    """One library context set up from a workload dict (see ``workloads``)."""

    def __init__(self, wl, mode, prm=None, stream=None, max_gates=None, fp8_scales=None, store_sdf=True,
                 single_cta=False):
        self.prm = dict(prm if prm is not None else wl["params"])
        poses = np.ascontiguousarray(wl["poses"], dtype=np.float32).reshape(-1, 7)
        self.G = poses.shape[0]
        self.cfg = make_config(self.prm, mode, max_gates or max(1, self.G))
        self.ctx = B.mppi_create(self.cfg, stream)
        self._keep = []
        lat = np.ascontiguousarray(wl["latents"], dtype=np.float32).reshape(-1, 64)[: self.G]
        if mode != "analytic":
            self._keep = flat_layers(wl["layers"])
            self._scales = None if fp8_scales is None else np.ascontiguousarray(fp8_scales, dtype=np.float32)
            B.mppi_set_sdf_weights(self.ctx, self._keep, self._scales)
        B.mppi_set_gates(self.ctx, self.G, poses if self.G else None, lat if self.G else None)
        # tests read s(p) of every rollout state: the SDF kernel stores it beside its cost fold;
        # single_cta selects the 16-bit SDF kernel's single-CTA form instead of the CTA pairs
        flags = (B.MPPI_DIAG_STORE_SDF if store_sdf and mode != "analytic" else 0) | \
            (B.MPPI_DIAG_SDF_SINGLE_CTA if single_cta else 0)
        if flags:
            B.mppi_set_diagnostics(self.ctx, flags)
        self.K, self.H = self.prm["K"], self.prm["H"]

    def close(self):
        if self.ctx is not None:
            B.mppi_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        self.close()

    def step(self, state=None, nominal=None):
        U = np.zeros((self.H, 4), dtype=np.float32)
        w = np.zeros(self.K, dtype=np.float32)
        J = np.zeros(self.K, dtype=np.float32)
        st = None if state is None else np.ascontiguousarray(state, dtype=np.float32)
        nom = None if nominal is None else np.ascontiguousarray(nominal, dtype=np.float32)
        B.mppi_step(self.ctx, st, None, None, nom, U, w, J)
        return dict(U_new=U, weights=w, J=J)

    def read(self, which):
        K, H = self.K, self.H
        if which in (B.MPPI_BUF_NOISE, B.MPPI_BUF_POSITIONS):
            out = np.zeros(H * K * 4, dtype=np.float32)
            B.mppi_read_buffer(self.ctx, which, out)
            return out.reshape(K, H, 4)                              # [K, H, 4] like the oracle
        if which == B.MPPI_BUF_COST_PARTS:
            out = np.zeros(3 * K, dtype=np.float32)
            B.mppi_read_buffer(self.ctx, which, out)
            return out.reshape(3, K)
        if which == B.MPPI_BUF_SDF:
            out = np.zeros(H * K, dtype=np.float32)
            B.mppi_read_buffer(self.ctx, which, out)
            return out.reshape(K, H)
        out = np.zeros(K, dtype=np.float32)
        B.mppi_read_buffer(self.ctx, which, out)
        return out

    def state(self):
        s = np.zeros(B.mppi_state_dim(self.cfg), dtype=np.float32)
        B.mppi_get_state(self.ctx, s)
        return s

    def nominal(self):
        n = np.zeros((self.H, 4), dtype=np.float32)
        B.mppi_get_nominal(self.ctx, n)
        return n

    def noise_words(self):
        out = np.zeros(self.H * self.K * 4, dtype=np.uint32)
        B.mppi_read_noise_words(self.ctx, out)
        return out.reshape(self.K, self.H, 4)


def cost_scale(ref):
    """Per-rollout magnitude of the summed cost terms: the scale of the relative cost tolerance."""
    return np.abs(ref["J_col"]) + np.abs(ref["J_prog"]) + np.abs(ref["J_ctl"])
