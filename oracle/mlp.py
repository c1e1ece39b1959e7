"""Gate-SDF decoder g_phi(z, p): a softplus MLP (Sec. III-B, Fig. 2).

Test infrastructure only (see ``oracle/__init__.py``).

The decoder maps the concatenation [p, z] of a gate-frame query point
(3 numbers) and the gate's latent code z to a scalar signed distance.  The
paper applies a positional encoding to p before concatenation and queries in
the camera frame; this build queries in the gate frame with no encoding, with
the explicit gate pose doing the job of the encoder's pose information.
Shape (stated reading of "four hidden layers of width 128"): 67 -> 128 ->
128 -> 128 -> 128 -> 1, i.e. four hidden activations, five affine maps, no
activation on the output.  Activation: softplus with beta = 100,

    sp(x) = log(1 + exp(beta x)) / beta.

Layers are (W, b) with W of shape [out, in], row-major.
"""

import numpy as np

BETA = 100.0


def softplus(x, beta=BETA):
    """sp(x) = log(1 + exp(beta x)) / beta, evaluated without overflow."""
    return np.logaddexp(0.0, beta * x) / beta


def softplus_grad(x, beta=BETA):
    """d sp / dx = logistic(beta x)."""
    return 0.5 * (1.0 + np.tanh(0.5 * beta * x))


def as_f64_layers(layers):
    return [(np.asarray(W, dtype=np.float64), np.asarray(b, dtype=np.float64)) for W, b in layers]


def forward(layers, x, beta=BETA):
    """MLP output for inputs x [N, in]: returns s [N]."""
    layers = as_f64_layers(layers)
    h = np.asarray(x, dtype=np.float64)
    for W, b in layers[:-1]:
        h = softplus(h @ W.T + b, beta)
    W, b = layers[-1]
    return (h @ W.T + b)[:, 0]


def positional_encoding(p, levels):
    """PE(p) of Sec. III-B (applied to the query coordinates before concatenation with z):
    [p, then for l = 0 .. levels-1: sin(2^l pi p), cos(2^l pi p)] -> [N, 3 + 6 levels];
    levels = 0 is the point itself."""
    p = np.asarray(p, dtype=np.float64)
    feats = [p]
    for l in range(levels):
        a = (2.0 ** l) * np.pi * p
        feats += [np.sin(a), np.cos(a)]
    return np.concatenate(feats, axis=-1)


def sdf(layers, pg, z, beta=BETA, pe_levels=0):
    """g_phi(z, PE(p)) for query points pg [N, 3] in the latent's frame and one latent z [Z]."""
    pg = np.asarray(pg, dtype=np.float64)
    z = np.asarray(z, dtype=np.float64)
    x = np.concatenate([positional_encoding(pg, pe_levels), np.broadcast_to(z, (pg.shape[0], z.shape[0]))], axis=1)
    return forward(layers, x, beta)


def input_gradient(layers, x, beta=BETA):
    """Gradient of the output with respect to the inputs x [N, in] (reverse mode)."""
    layers = as_f64_layers(layers)
    h = np.asarray(x, dtype=np.float64)
    pre = []
    for W, b in layers[:-1]:
        a = h @ W.T + b
        pre.append(a)
        h = softplus(a, beta)
    g = np.broadcast_to(layers[-1][0][0], (h.shape[0], h.shape[1])).copy()
    for (W, _), a in zip(reversed(layers[:-1]), reversed(pre)):
        g = (g * softplus_grad(a, beta)) @ W
    return g
