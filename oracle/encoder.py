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


def bf16_round(a):
    """Values rounded to the nearest bfloat16 (8 significant bits, ties to even), from their
    float32 rounding: the 16 high bits of the float32 pattern after adding half of the dropped
    low 16 bits' unit (0x7FFF, plus one when the kept part is odd).  Returned as float64."""
    u = np.ascontiguousarray(np.asarray(a, dtype=np.float32)).view(np.uint32).astype(np.uint64)
    kept = (u + 0x7FFF + ((u >> 16) & 1)) >> 16
    return (kept << 16).astype(np.uint32).view(np.float32).astype(np.float64)


def bf16_split(a):
    """a (rounded to float32) = hi + lo + e with hi = bf16(a), lo = bf16(a - hi), |e| <= 2^-16 |a|."""
    a32 = np.asarray(a, dtype=np.float32).astype(np.float64)
    hi = bf16_round(a32)
    return hi, bf16_round(a32 - hi)


def conv3x3_s2_split(x, W, b):
    """The convolution of ``conv3x3_s2`` with every product x w replaced by x_hi w_hi + x_hi w_lo
    + x_lo w_hi of the operands' BF16 splits (``bf16_split``), summed exactly: the precision
    model of a tensor-core convolution on BF16 operand pairs.  Each product is within
    ~3 x 2^-16 of x w.  Used to take the ReLU decisions of a gradient check in the precision
    that kernel computes in."""
    xh, xl = bf16_split(x)
    wh, wl = bf16_split(W)
    zero = np.zeros_like(np.asarray(b, dtype=np.float64))
    return conv3x3_s2(xh, wh, b) + conv3x3_s2(xh, wl, zero) + conv3x3_s2(xl, wh, zero)


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
