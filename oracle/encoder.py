"""Depth encoder E_theta: depth image -> latent code z (Sec. III-B, Fig. 2).

Test infrastructure only (see ``oracle/__init__.py``).

The paper encodes each depth image once per control cycle into z in R^64 (Sec. IV-B, V)
but gives neither the encoder's architecture nor its weights.  Reading used on both sides
of the parity check: a small convolutional encoder of a depth image of H x W pixels,

    x_0 = I / max_range                                   (1 channel, depths scaled to [0, 1])
    x_l = relu(conv3x3_stride2_pad1(x_{l-1}; W_l, b_l))   l = 1..4, channels 16, 32, 64, 64
    z   = W_5 mean_{i,j} x_4[:, i, j] + b_5               (64 -> 64)

with the convolution out[co, i, j] = b[co] + sum_{ci, ky, kx} W[co, ci, ky, kx]
x[ci, 2 i + ky - 1, 2 j + kx - 1] (zero outside the image), so each layer halves the
size, rounding up: H_l = ceil(H_{l-1} / 2).  Weights are inputs (W_l [co, ci, 3, 3],
W_5 [64, 64], row-major).
"""

import numpy as np

CHANNELS = (16, 32, 64, 64)
LATENT = 64


def out_size(n):
    """Output length of a 3-tap, stride-2, pad-1 convolution of length n."""
    return (n + 1) // 2


def conv3x3_s2(x, W, b):
    """x [Ci, H, W_] -> [Co, ceil(H / 2), ceil(W_ / 2)] (definition in the module docstring)."""
    x = np.asarray(x, dtype=np.float64)
    W = np.asarray(W, dtype=np.float64)
    ci, h, w = x.shape
    ho, wo = out_size(h), out_size(w)
    # zero padding: one row / column before, enough after for the last window
    xp = np.zeros((ci, 2 * ho + 1, 2 * wo + 1))
    xp[:, 1:h + 1, 1:w + 1] = x
    out = np.broadcast_to(np.asarray(b, dtype=np.float64)[:, None, None], (W.shape[0], ho, wo)).copy()
    for ky in range(3):
        for kx in range(3):
            tap = xp[:, ky:ky + 2 * ho:2, kx:kx + 2 * wo:2]         # x[ci, 2i + ky - 1, 2j + kx - 1]
            out += np.einsum("oc,chw->ohw", W[:, :, ky, kx], tap)
    return out


def encode(depth, max_range, layers):
    """Latent codes [N, 64] of depth images [N, H, W]; layers = [(W1, b1) .. (W4, b4), (W5, b5)]."""
    depth = np.asarray(depth, dtype=np.float64)
    if depth.ndim == 2:
        depth = depth[None]
    out = []
    for img in depth:
        x = img[None] / max_range
        for W, b in layers[:4]:
            x = np.maximum(conv3x3_s2(x, W, b), 0.0)
        W5, b5 = (np.asarray(a, dtype=np.float64) for a in layers[4])
        out.append(W5 @ x.mean(axis=(1, 2)) + b5)
    return np.stack(out)
