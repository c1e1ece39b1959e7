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

from .encoder import conv3x3_s2, conv3x3_s2_split

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


def forward(noisy, max_range, enc_layers, split=False):
    """Encoder forward keeping every activation: returns (inputs x0..x4, z [N, 64]).  With
    split=True the convolutions use the BF16 operand-split products of ``conv3x3_s2_split`` (each
    layer's input and output rounded to float32, as a kernel stores them), so that the ReLU
    decisions are taken in the precision of a tensor-core forward pass."""
    xs = [np.asarray(noisy, dtype=np.float64)[:, None] / max_range]
    for W, b in enc_layers[:4]:
        if split:
            xs.append(np.stack([np.maximum(conv3x3_s2_split(x, W, b), 0.0) for x in xs[-1]])
                      .astype(np.float32).astype(np.float64))
        else:
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


def gradients(noisy, clean, max_range, enc_layers, dec, split=False):
    """Loss and the gradients of every tensor: (loss, [(gW1, gb1) .. (gW5, gb5)], (gWd, gbd)).
    split: the forward pass of ``forward(..., split=True)`` (the gradients of the network as a
    BF16-operand-split tensor-core forward pass computes it; ReLU kinks decided there)."""
    enc = [(np.asarray(W, dtype=np.float64), np.asarray(b, dtype=np.float64)) for W, b in enc_layers]
    Wd, bd = (np.asarray(a, dtype=np.float64) for a in dec)
    xs, z = forward(noisy, max_range, enc, split=split)
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


# ---------------------------------------------------------------- the SDF term (frozen decoder)
# Sec. III-B supervises the latent through the SDF decoder: |g_phi(E(I_noisy), PE(p)) - s(p)| at
# query points p of the camera frame whose exact SDF s is known from the rendered scene.  Here
# the decoder is frozen (as in the paper's second stage) and only the encoder and D_psi learn.
# Query points (a reading: the paper samples near-surface, interior, collision-prone and
# frustum points, Sec. III-A): with Philox blocks A = (j, i, frame, 0x5DF0A) and
# B = (j, i, frame, 0x5DF0B) of key = seed for point j of image i,
#   * near a gate when the uniform of A's word 3 is below near_frac: gate g = ((A0 >> 8) G) >> 24,
#     the gate-frame point ((2 uB0 - 1)(d + 0.3), (2 uB1 - 1)(a_out + 0.3), (2 uB2 - 1)(a_out + 0.3));
#   * else in the view frustum: depth x = 0.2 + uA1 (max_range - 0.2) along the ray of the image
#     position (W uA2, H uB3): y = -(W uA2 - cx) x / fx, z = -(H uB3 - cy) x / fy;
# label = the exact frame SDF of the nearest gate (min over gates).

QUERY_TAG_A = 0x5DF0A
QUERY_TAG_B = 0x5DF0B


def sample_queries(cam_poses, gate_poses, n_points, width, height, fx, fy, cx, cy, max_range, near_frac, seed, frame,
                   a_in=0.5, a_out=0.75, d=0.1):
    """Camera-frame query points [N, n_points, 3] and their exact SDF labels [N, n_points]."""
    from . import gate_sdf
    from .dynamics import quat_rotate, quat_conj
    from .noise import words_to_uniform
    from .philox import philox4x32_10, split_seed
    cams = np.asarray(cam_poses, dtype=np.float64).reshape(-1, 7)
    gates = np.asarray(gate_poses, dtype=np.float64).reshape(-1, 7)
    n, G = len(cams), len(gates)
    j = np.arange(n_points, dtype=np.uint64)[None, :]
    i = np.arange(n, dtype=np.uint64)[:, None]

    def block(tag):
        j_b, i_b = np.broadcast_arrays(j, i)
        ctr = np.stack([j_b, i_b, np.full(j_b.shape, int(frame) & 0xFFFFFFFF, np.uint64),
                        np.full(j_b.shape, tag, np.uint64)], axis=-1)
        return philox4x32_10(ctr, split_seed(seed))

    A, Bw = block(QUERY_TAG_A), block(QUERY_TAG_B)
    uA, uB = words_to_uniform(A), words_to_uniform(Bw)
    near = uA[..., 3] < float(np.float32(near_frac))
    gi = ((A[..., 0].astype(np.uint64) >> np.uint64(8)) * np.uint64(max(G, 1))) >> np.uint64(24)
    cam_q = cams[:, 3:7] / np.linalg.norm(cams[:, 3:7], axis=1, keepdims=True)
    pts = np.zeros((n, n_points, 3))
    # frustum points
    x = 0.2 + uA[..., 1] * (max_range - 0.2)
    pts_f = np.stack([x, -(width * uA[..., 2] - cx) * x / fx, -(height * uB[..., 3] - cy) * x / fy], axis=-1)
    pts[~near] = pts_f[~near]
    if G > 0 and near.any():
        half = np.array([d + 0.3, a_out + 0.3, a_out + 0.3])
        pg = (2.0 * uB[..., 0:3] - 1.0) * half
        gq = gates[gi.astype(np.int64), 3:7]
        gq = gq / np.linalg.norm(gq, axis=-1, keepdims=True)
        world = quat_rotate(gq, pg) + gates[gi.astype(np.int64), 0:3]
        cq = np.broadcast_to(cam_q[:, None, :], world.shape[:-1] + (4,))
        pc = quat_rotate(quat_conj(cq), world - cams[:, None, 0:3])
        pts[near] = pc[near]
    # labels: exact SDF of the nearest frame
    cq = np.broadcast_to(cam_q[:, None, :], pts.shape[:-1] + (4,))
    world = quat_rotate(cq, pts) + cams[:, None, 0:3]
    lab = np.full((n, n_points), np.inf)
    for gp in gates:
        gp = np.array(gp, dtype=np.float64)
        gp[3:7] /= np.linalg.norm(gp[3:7])
        lab = np.minimum(lab, gate_sdf.frame_sdf(gate_sdf.to_gate_frame(world.reshape(-1, 3), gp).reshape(world.shape),
                                                 a_in, a_out, d))
    return pts, lab


def sdf_term(z, points, labels, dec_layers, pe_levels):
    """(mean |g(z_i, PE(p_ij)) - s_ij|, d/dz [N, 64]) with the decoder frozen."""
    from .mlp import input_gradient, positional_encoding, sdf
    z = np.asarray(z, dtype=np.float64)
    n, m, _ = np.asarray(points).shape
    L = 0.0
    dz = np.zeros_like(z)
    nf = 3 + 6 * pe_levels
    for i in range(n):
        s = sdf(dec_layers, points[i], z[i], pe_levels=pe_levels)
        r = s - labels[i]
        L += float(np.sum(np.abs(r)))
        x = np.concatenate([positional_encoding(points[i], pe_levels), np.broadcast_to(z[i], (m, z.shape[1]))], axis=1)
        gx = input_gradient(dec_layers, x)
        dz[i] = (np.sign(r)[:, None] * gx[:, nf:]).sum(axis=0) / (n * m)
    return L / (n * m), dz


def gradients_joint(noisy, clean, max_range, enc_layers, dec, points, labels, sdf_layers, pe_levels, lam_recon,
                    lam_sdf, split=False):
    """Loss lam_recon L_recon + lam_sdf L_sdf and the gradients of the encoder's tensors and D_psi
    (the SDF decoder frozen): (loss, L_recon, L_sdf, enc grads, dec grads).  split as in
    ``gradients``."""
    enc = [(np.asarray(W, dtype=np.float64), np.asarray(b, dtype=np.float64)) for W, b in enc_layers]
    Wd, bd = (np.asarray(a, dtype=np.float64) for a in dec)
    xs, z = forward(noisy, max_range, enc, split=split)
    n = len(z)
    t = pooled_target(clean, max_range).reshape(n, -1)
    r = z @ Wd.T + bd - t
    L_rec = float(np.mean(np.abs(r)))
    g = lam_recon * np.sign(r) / r.size
    gWd, gbd = g.T @ z, g.sum(axis=0)
    L_sdf, dz_sdf = sdf_term(z, points, labels, sdf_layers, pe_levels)
    dz = g @ Wd + lam_sdf * dz_sdf
    W5 = enc[4][0]
    x4 = xs[4]
    m = x4.mean(axis=(2, 3))
    gW5, gb5 = dz.T @ m, dz.sum(axis=0)
    dm = dz @ W5
    hw = x4.shape[2] * x4.shape[3]
    delta = (dm / hw)[:, :, None, None] * (x4 > 0.0)
    grads = [None] * 4
    for l in range(3, -1, -1):
        x_in = xs[l]
        grads[l] = (conv_weight_grad(x_in, delta), delta.sum(axis=(0, 2, 3)))
        if l > 0:
            dx = conv_input_grad(delta, enc[l][0], x_in.shape[2], x_in.shape[3])
            delta = dx * (x_in > 0.0)
    grads.append((gW5, gb5))
    return lam_recon * L_rec + lam_sdf * L_sdf, L_rec, L_sdf, grads, (gWd, gbd)


# ---------------------------------------------------------------- stage 1 in full: the decoder trains too
def decoder_grads(z, points, labels, dec_layers, pe_levels, beta=100.0):
    """SDF term with the decoder trainable: (mean |r|, d/dz [N, 64], [(dW, db) of the 5 layers])."""
    from .mlp import positional_encoding, softplus, softplus_grad
    layers = [(np.asarray(W, dtype=np.float64), np.asarray(b, dtype=np.float64)) for W, b in dec_layers]
    z = np.asarray(z, dtype=np.float64)
    n, m, _ = np.asarray(points).shape
    nf = 3 + 6 * pe_levels
    gW = [np.zeros_like(W) for W, _ in layers]
    gb = [np.zeros_like(b) for _, b in layers]
    dz = np.zeros_like(z)
    L = 0.0
    for i in range(n):
        x = np.concatenate([positional_encoding(points[i], pe_levels), np.broadcast_to(z[i], (m, z.shape[1]))], axis=1)
        hs, pre = [x], []
        for W, b in layers[:-1]:
            a = hs[-1] @ W.T + b
            pre.append(a)
            hs.append(softplus(a, beta))
        s = (hs[-1] @ layers[-1][0].T + layers[-1][1])[:, 0]
        r = s - labels[i]
        L += float(np.sum(np.abs(r)))
        g = (np.sign(r) / (n * m))[:, None]                     # d L / d s, [m, 1]
        gW[-1] += g.T @ hs[-1]
        gb[-1] += g.sum(axis=0)
        g = g @ layers[-1][0]                                    # d L / d h4
        for l in range(len(layers) - 2, -1, -1):
            g = g * softplus_grad(pre[l], beta)                  # d L / d a_{l+1}
            gW[l] += g.T @ hs[l]
            gb[l] += g.sum(axis=0)
            g = g @ layers[l][0]                                 # d L / d (layer input)
        dz[i] = g[:, nf:].sum(axis=0)
    return L / (n * m), dz, list(zip(gW, gb))
