"""Denoising training of the depth encoder (the reconstruction term of Sec. III-B's first stage):
the encoder E_theta reads a noisy depth image, a depth decoder D_psi maps the latent back to a
coarse clean depth image, and the L1 distance between the two is minimised with Adam.

Test infrastructure only (see ``oracle/__init__.py``).

Readings (the paper gives neither D_psi nor the target resolution):

* target: the clean image scaled by 1 / max_range and averaged over 8 x 8 pixel blocks (blocks
  at the right and bottom edges average the pixels they contain), T = ceil(H / 8) x ceil(W / 8)
  values per image;
* D_psi: one affine map 64 -> T (W_D [T, 64], b_D [T]);
* loss: mean over the batch and the T values of |D(E(I_noisy)) - target|, with d|r|/dr = sign(r)
  (0 at r = 0);
* Adam (beta1 0.9, beta2 0.999, eps 1e-8, bias-corrected) on the encoder's four convolutions,
  its head and D_psi.

The gradients are the chain rule through the encoder of ``encoder.py`` written out layer by
layer (stride-2 3x3 convolutions: weight gradient = correlation of the output gradient with
the layer input's taps; input gradient = the transposed scatter of each output gradient back
to its nine taps).
"""

import numpy as np

from .encoder import conv3x3_s2

POOL = 8


def pooled_target(clean, max_range):
    """Clean images [N, H, W] -> targets [N, ceil(H / 8), ceil(W / 8)] (block means of depth / max_range)."""
    clean = np.asarray(clean, dtype=np.float64) / max_range
    n, h, w = clean.shape
    th, tw = -(-h // POOL), -(-w // POOL)
    out = np.zeros((n, th, tw))
    for a in range(th):
        for b in range(tw):
            out[:, a, b] = clean[:, a * POOL:(a + 1) * POOL, b * POOL:(b + 1) * POOL].mean(axis=(1, 2))
    return out


def forward(noisy, max_range, enc_layers):
    """Encoder forward keeping every activation: returns (inputs x0..x4, z [N, 64])."""
    xs = [np.asarray(noisy, dtype=np.float64)[:, None] / max_range]
    for W, b in enc_layers[:4]:
        xs.append(np.stack([np.maximum(conv3x3_s2(x, W, b), 0.0) for x in xs[-1]]))
    W5, b5 = (np.asarray(a, dtype=np.float64) for a in enc_layers[4])
    m = xs[-1].mean(axis=(2, 3))
    return xs, m @ W5.T + b5


def loss(noisy, clean, max_range, enc_layers, dec):
    """L1 reconstruction loss of one batch."""
    _, z = forward(noisy, max_range, enc_layers)
    Wd, bd = (np.asarray(a, dtype=np.float64) for a in dec)
    t = pooled_target(clean, max_range).reshape(len(z), -1)
    return float(np.mean(np.abs(z @ Wd.T + bd - t)))


def conv_weight_grad(x, delta):
    """d loss / d W of a stride-2 3x3 convolution: x [N, Ci, H, W] its input, delta [N, Co, Ho, Wo]
    the gradient at its output (before the ReLU's mask is applied by the caller)."""
    n, ci, h, w = x.shape
    ho, wo = delta.shape[2:]
    xp = np.zeros((n, ci, 2 * ho + 1, 2 * wo + 1))
    xp[:, :, 1:h + 1, 1:w + 1] = x
    gw = np.zeros((delta.shape[1], ci, 3, 3))
    for ky in range(3):
        for kx in range(3):
            tap = xp[:, :, ky:ky + 2 * ho:2, kx:kx + 2 * wo:2]          # x[n, ci, 2i + ky - 1, 2j + kx - 1]
            gw[:, :, ky, kx] = np.einsum("nohw,nchw->oc", delta, tap)
    return gw


def conv_input_grad(delta, W, h, w):
    """d loss / d x of a stride-2 3x3 convolution with input size h x w: each output gradient
    scattered back to its nine taps (zero padding drops the taps outside the image)."""
    n, co, ho, wo = delta.shape
    ci = W.shape[1]
    gp = np.zeros((n, ci, 2 * ho + 1, 2 * wo + 1))
    for ky in range(3):
        for kx in range(3):
            gp[:, :, ky:ky + 2 * ho:2, kx:kx + 2 * wo:2] += np.einsum("nohw,oc->nchw", delta, W[:, :, ky, kx])
    return gp[:, :, 1:h + 1, 1:w + 1]


def gradients(noisy, clean, max_range, enc_layers, dec):
    """Loss and the gradients of every tensor: (loss, [(gW1, gb1) .. (gW5, gb5)], (gWd, gbd))."""
    enc = [(np.asarray(W, dtype=np.float64), np.asarray(b, dtype=np.float64)) for W, b in enc_layers]
    Wd, bd = (np.asarray(a, dtype=np.float64) for a in dec)
    xs, z = forward(noisy, max_range, enc)
    n = len(z)
    t = pooled_target(clean, max_range).reshape(n, -1)
    r = z @ Wd.T + bd - t
    L = float(np.mean(np.abs(r)))
    g = np.sign(r) / r.size                      # d L / d (D(z))
    gWd, gbd = g.T @ z, g.sum(axis=0)
    dz = g @ Wd
    W5 = enc[4][0]
    x4 = xs[4]
    m = x4.mean(axis=(2, 3))
    gW5, gb5 = dz.T @ m, dz.sum(axis=0)
    dm = dz @ W5
    hw = x4.shape[2] * x4.shape[3]
    delta = (dm / hw)[:, :, None, None] * (x4 > 0.0)     # gradient at conv 4's pre-activation
    grads = [None] * 4
    for l in range(3, -1, -1):
        x_in = xs[l]
        grads[l] = (conv_weight_grad(x_in, delta), delta.sum(axis=(0, 2, 3)))
        if l > 0:
            dx = conv_input_grad(delta, enc[l][0], x_in.shape[2], x_in.shape[3])
            delta = dx * (x_in > 0.0)
    grads.append((gW5, gb5))
    return L, grads, (gWd, gbd)


def adam_step(params, grads, m, v, step, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update of lists of arrays (step counts from 1); returns new (params, m, v)."""
    out_p, out_m, out_v = [], [], []
    for p, g, mi, vi in zip(params, grads, m, v):
        mi = b1 * mi + (1 - b1) * g
        vi = b2 * vi + (1 - b2) * g * g
        mh = mi / (1 - b1 ** step)
        vh = vi / (1 - b2 ** step)
        out_p.append(p - lr * mh / (np.sqrt(vh) + eps))
        out_m.append(mi)
        out_v.append(vi)
    return out_p, out_m, out_v
