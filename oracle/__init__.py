"""FP64 CPU oracle for the MPPI + Gate-SDF control step.

TEST INFRASTRUCTURE ONLY.  Nothing on the product path may import, call or
execute anything in this package: only ``tests/``, ``__graft_entry__.smoke()``
and the ``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` use it.
It shares no code with the CUDA path (no kernels, headers, helpers, tables
or constant generators) and imports nothing from it.

The oracle restates the paper's method step by step in float64 with numpy:

* ``philox``    -- Philox4x32-10 counter-based generator (published definition,
                   Salmon et al., SC'11), the noise source of the sampling step.
* ``noise``     -- uniform mapping, Box-Muller normals and the sampled
                   perturbations delta u ~ N(0, Sigma) of Sec. IV-A (Eq. 5).
* ``dynamics``  -- quadrotor model x_dot = f(x, u) with state [p, v, q, w]
                   (Sec. IV-A) in collective-thrust + body-rate form, RK4.
* ``rotor``     -- the paper's rotor-thrust-rate model (state + four rotor thrusts,
                   command = thrust rates) and its RK4 step, with stated airframe readings.
* ``gate_sdf``  -- gate-frame transform, the l-infinity radial metric (Eq. 1),
                   the hourglass guide SDF (Eq. 2) and the exact signed
                   distance to the rectangular gate frame.
* ``mlp``       -- the Gate-SDF decoder g_phi(z, p) (Sec. III-B), softplus MLP,
                   and its input gradient (for the Eikonal term).
* ``render``    -- depth images of the gate frames through a pinhole camera (exact ray
                   casting) and the synthetic sensor noise (Sec. III-B).
* ``encoder``   -- the depth encoder E_theta (depth image -> latent z) in the stated
                   convolutional reading (Sec. III-B).
* ``encoder_train`` -- denoising training of the encoder (L1 reconstruction of the pooled
                   clean image through a linear depth decoder), its gradients and Adam.
* ``distill``   -- the distillation loss (L1 + Eikonal), its gradients and Adam.
* ``mppi``      -- per-rollout costs (Eq. 8-10 in the configured form),
                   softmax weights and the weighted update (Eq. 5), the
                   receding-horizon shift, one whole control step and a
                   closed-loop driver.

Every random number the method draws comes from ``philox`` keyed exactly as
the CUDA path keys it; all other inputs (gate poses, latents, weights, start
states) are passed in by the caller from the seeded generators in
``workloads``.
"""

from . import philox, noise, dynamics, rotor, gate_sdf, mlp, mppi, distill, render, encoder, encoder_train  # noqa: F401
