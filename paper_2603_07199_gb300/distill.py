"""Distil the exact gate-frame SDF into the Gate-SDF MLP on the GPU (Sec. III-B) and
write the learned weights.

    python -m paper_2603_07199_gb300.distill --steps 20000 --gemm bf16 --out gate_sdf.npz

Training points, loss (L1 + Eikonal), Adam and the held-out check all run in the
library (mppi_train_*); this module only chooses the initial weights, the latent
and the learning-rate schedule (a linear warm-up to the peak, then a half-cosine
decay, set once per chunk of steps at the chunk's midpoint), and reports
training steps/s and the held-out error against the exact SDF.  The output
holds the ten arrays of mppi_set_sdf_weights (W1, b1, ..., w5, b5) and the
latent z0.
"""
import argparse
import time

import numpy as np

from . import binding as B


def initial_layers(seed, in_dim=3 + B.MPPI_LATENT_DIM, hidden=B.MPPI_HIDDEN):
    """Glorot-uniform weights and zero biases for the 67-128-128-128-128-1 network."""
    rng = np.random.default_rng(seed)
    dims = [in_dim, hidden, hidden, hidden, hidden, 1]
    out = []
    for i in range(5):
        lim = np.sqrt(6.0 / (dims[i] + dims[i + 1]))
        W = rng.uniform(-lim, lim, (dims[i + 1], dims[i])).astype(np.float32)
        b = np.zeros(dims[i + 1], np.float32)
        out += [np.ascontiguousarray(W if i < 4 else W.reshape(-1)), b]
    return out


def lr_at(step_mid, steps, peak, warmup):
    if step_mid < warmup:
        return peak * step_mid / warmup
    return peak * 0.5 * (1.0 + np.cos(np.pi * (step_mid - warmup) / max(1, steps - warmup)))


def distil(steps, gemm="bf16", peak_lr=2e-3, warmup=1000, chunk=250, seed=1, latent_seed=2, verbose=True):
    """Train from Glorot-uniform weights; returns (layers, z0, report)."""
    cfg = B.mppi_train_config_default()
    layers = initial_layers(seed)
    z0 = np.random.default_rng(latent_seed).standard_normal((1, B.MPPI_LATENT_DIM)).astype(np.float32)[0]
    tr = B.mppi_train_create(cfg, layers, z0)
    try:
        B.mppi_train_set_gemm_precision(tr, B.MPPI_TRAIN_GEMM_BF16 if gemm == "bf16" else B.MPPI_TRAIN_GEMM_FP32)
        t0, done, loss = time.perf_counter(), 0, float("nan")
        while done < steps:
            n = min(chunk, steps - done)
            B.mppi_train_set_lr(tr, lr_at(done + 0.5 * n, steps, peak_lr, warmup))
            loss = B.mppi_train_step(tr, n)
            done += n
            if verbose:
                print(f"step {done:6d}  loss {loss:.5f}", flush=True)
        seconds = time.perf_counter() - t0
        ev = B.mppi_train_evaluate(tr)
        out = [np.zeros_like(a) for a in layers]
        B.mppi_train_get_weights(tr, out)
    finally:
        B.mppi_train_destroy(tr)
    report = {"steps": steps, "gemm": gemm, "seconds": seconds, "steps_per_s": steps / seconds if seconds > 0 else None,
              "final_loss": loss, "holdout_mm": {k: v * 1e3 for k, v in ev.items()}}
    return out, z0, report


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--steps", type=int, default=20000)
    ap.add_argument("--gemm", choices=["bf16", "fp32"], default="bf16",
                    help="hidden-layer GEMMs: BF16 on the tensor cores or FP32 on the CUDA cores")
    ap.add_argument("--peak-lr", type=float, default=2e-3)
    ap.add_argument("--warmup", type=int, default=1000)
    ap.add_argument("--seed", type=int, default=1)
    ap.add_argument("--latent-seed", type=int, default=2)
    ap.add_argument("--out", default=None, help="write the learned weights and z0 to this .npz file")
    ap.add_argument("--quiet", action="store_true")
    a = ap.parse_args(argv)
    layers, z0, report = distil(a.steps, a.gemm, a.peak_lr, a.warmup, seed=a.seed, latent_seed=a.latent_seed,
                                verbose=not a.quiet)
    print(report)
    if a.out:
        names = ["W1", "b1", "W2", "b2", "W3", "b3", "W4", "b4", "w5", "b5"]
        np.savez(a.out, z0=z0, **dict(zip(names, layers)))


if __name__ == "__main__":
    main()
