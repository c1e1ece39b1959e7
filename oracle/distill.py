"""Distilling the analytic gate SDF into the Gate-SDF MLP: loss, gradients, Adam.

Test infrastructure only (see ``oracle/__init__.py``).

The paper trains its decoder g_phi with an L1 loss on the SDF (Sec. III-B,
Eq. 3-4).  The distillation workload here fits the MLP of ``oracle.mlp`` at a
fixed latent z0 to the exact frame SDF (``oracle.gate_sdf``), adding an
Eikonal term on the input gradient:

    L = mean_b |s_b - s*_b| + lambda_e mean_b (|grad_p s_b| - 1)^2 ,

with grad_p s the derivative of the network output with respect to the 3
point coordinates.  ``loss_and_grads`` evaluates it in forward mode (the three
tangent directions e_x, e_y, e_z carried through every layer next to the
values) and differentiates the whole computation in reverse mode:

    tangents:  a1^j = W1[:, j],  h_l^j = sp'(a_l) * a_l^j,  a_{l+1}^j = W_{l+1} h_l^j,
               g_j = w5 . h4^j;
    adjoints:  for h = sp(a), h^j = sp'(a) a^j:
               da  += dh * sp'(a) + sum_j dh^j * a^j * sp''(a),  da^j = dh^j * sp'(a);
               for a = W x + b, a^j = W x^j:
               dW += da x^T + sum_j da^j (x^j)^T,  db += da,  dx = W^T da,  dx^j = W^T da^j,
               and for the first layer dW1[:, j] += sum_b da1^j (its tangent seed is W1 e_j),
    with sp'(a) = logistic(beta a), sp''(a) = beta sp'(a) (1 - sp'(a)).

Adam (Kingma and Ba, "Adam: A Method for Stochastic Optimization", ICLR 2015,
Algorithm 1): m = b1 m + (1 - b1) g, v = b2 v + (1 - b2) g^2,
theta -= lr * (m / (1 - b1^t)) / (sqrt(v / (1 - b2^t)) + eps).

Training points (stated reading of the hybrid sampling of Sec. III-B, Fig. 3b,
in the configured form): 70 % near the frame surface -- a point drawn
uniformly over the surface area, plus N(0, 0.05^2 I) -- and 30 % uniform in an
8 m cube [-4, 4]^3 around the gate, all in the gate frame.
"""

import numpy as np

from . import gate_sdf, mlp


def forward_tangents(layers, P, z, beta=mlp.BETA):
    """Values and input gradients of the MLP at gate-frame points P [B, 3] with latent z.

    Returns (s [B], g [B, 3], cache) where cache holds the pre-activations and
    tangents needed by ``backward``.
    """
    layers = mlp.as_f64_layers(layers)
    P = np.asarray(P, dtype=np.float64)
    z = np.asarray(z, dtype=np.float64)
    W1, b1 = layers[0]
    x0 = np.concatenate([P, np.broadcast_to(z, (P.shape[0], z.shape[0]))], axis=1)
    a = x0 @ W1.T + b1
    at = np.stack([np.broadcast_to(W1[:, j], a.shape) for j in range(3)])      # [3, B, H]
    cache = [(x0, None, a, at)]
    h = mlp.softplus(a, beta)
    ht = mlp.softplus_grad(a, beta)[None] * at
    for W, b in layers[1:-1]:
        a = h @ W.T + b
        at = ht @ W.T
        cache.append((h, ht, a, at))
        h = mlp.softplus(a, beta)
        ht = mlp.softplus_grad(a, beta)[None] * at
    w5, b5 = layers[-1]
    s = (h @ w5.T + b5)[:, 0]
    g = (ht @ w5.T)[..., 0].T                                                  # [B, 3]
    cache.append((h, ht, None, None))
    return s, g, cache


def loss_value(s, g, target, lam_e):
    gn = np.linalg.norm(g, axis=1)
    return np.mean(np.abs(s - target)) + lam_e * np.mean((gn - 1.0) ** 2)


def loss_and_grads(layers, P, z, target, lam_e=0.1, beta=mlp.BETA):
    """Loss and its gradients with respect to every weight and bias (same shapes as layers)."""
    layers64 = mlp.as_f64_layers(layers)
    target = np.asarray(target, dtype=np.float64)
    s, g, cache = forward_tangents(layers64, P, z, beta)
    B = s.shape[0]
    gn = np.linalg.norm(g, axis=1)
    loss = loss_value(s, g, target, lam_e)
    ds = np.sign(s - target) / B                                              # dL/ds
    dg = (lam_e * 2.0 * (gn - 1.0) / np.maximum(gn, 1e-30))[:, None] * g / B   # dL/dg  [B, 3]
    grads = [None] * len(layers64)
    # output layer: s = h4 . w5 + b5, g_j = h4^j . w5
    h4, h4t, _, _ = cache[-1]
    w5, b5 = layers64[-1]
    grads[-1] = (ds @ h4 + np.einsum("jb,jbh->h", dg.T, h4t))[None, :], np.array([ds.sum()])
    dh = ds[:, None] * w5[0][None, :]
    dht = dg.T[:, :, None] * w5[0][None, None, :]
    for li in range(len(layers64) - 2, -1, -1):
        x, xt, a, at = cache[li]
        W, _ = layers64[li]
        sig = mlp.softplus_grad(a, beta)
        sig2 = beta * sig * (1.0 - sig)
        da = dh * sig + np.sum(dht * at * sig2[None], axis=0)
        dat = dht * sig[None]
        if li == 0:
            dW = da.T @ x
            dW[:, 0:3] += dat.sum(axis=1).T                                    # tangent seeds W1 e_j
        else:
            dW = da.T @ x + np.einsum("jbo,jbi->oi", dat, xt)
            dh = da @ W
            dht = dat @ W
        grads[li] = (dW, da.sum(axis=0))
    return loss, grads


def adam_update(param, grad, m, v, t, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam step (t counts from 1); returns the new (param, m, v)."""
    m = b1 * m + (1.0 - b1) * grad
    v = b2 * v + (1.0 - b2) * grad * grad
    mhat = m / (1.0 - b1 ** t)
    vhat = v / (1.0 - b2 ** t)
    return param - lr * mhat / (np.sqrt(vhat) + eps), m, v


def surface_areas(a_in=gate_sdf.GATE_INNER_HALF, a_out=gate_sdf.GATE_OUTER_HALF, d=gate_sdf.GATE_HALF_DEPTH):
    """Areas of the frame's boundary parts: the two faces |x| = d, the outer and the inner walls."""
    face = (2 * a_out) ** 2 - (2 * a_in) ** 2
    return dict(faces=2 * face, outer=4 * (2 * a_out) * (2 * d), inner=4 * (2 * a_in) * (2 * d))


def targets(P):
    """Training targets: the exact frame SDF at gate-frame points."""
    return gate_sdf.frame_sdf(np.asarray(P, dtype=np.float64))
