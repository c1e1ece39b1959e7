"""Pins for the denoising training of the depth encoder in the oracle: the pooled target by hand,
every gradient against central differences of the loss, and Adam's first step in closed form."""
import numpy as np
import pytest

import workloads as W
from oracle import encoder_train as T


def test_pooled_target_blocks():
    img = np.arange(2 * 10 * 17, dtype=np.float64).reshape(2, 10, 17)
    t = T.pooled_target(img, 2.0)
    assert t.shape == (2, 2, 3)
    assert abs(t[0, 0, 0] - img[0, :8, :8].mean() / 2) < 1e-12
    assert abs(t[1, 1, 2] - img[1, 8:, 16:].mean() / 2) < 1e-12      # 2 x 1 edge block


def _setup(seed=0):
    rng = np.random.default_rng(seed)
    enc = [(W.astype(np.float64), b.astype(np.float64)) for W, b in W.encoder_weights(11)]
    dec = (rng.normal(0, 0.2, (6, 64)), rng.normal(0, 0.1, 6))
    clean = rng.uniform(0.5, 10.0, (2, 13, 17))
    noisy = clean + rng.normal(0, 0.3, clean.shape)
    return noisy, clean, enc, dec


def test_gradients_match_central_differences():
    noisy, clean, enc, dec = _setup()
    L, g_enc, g_dec = T.gradients(noisy, clean, 10.0, enc, dec)
    assert abs(L - T.loss(noisy, clean, 10.0, enc, dec)) < 1e-14
    rng = np.random.default_rng(1)
    h = 1e-6

    def fd(get, setter, idx):
        base = get()
        old = base[idx]
        base[idx] = old + h
        setter(base)
        lp = T.loss(noisy, clean, 10.0, enc, dec)
        base[idx] = old - h
        setter(base)
        lm = T.loss(noisy, clean, 10.0, enc, dec)
        base[idx] = old
        setter(base)
        return (lp - lm) / (2 * h)

    for li in range(5):
        for which in (0, 1):
            arr = enc[li][which]
            grad = g_enc[li][which]
            scale = np.max(np.abs(grad)) + 1e-12
            for _ in range(6):
                idx = tuple(rng.integers(s) for s in arr.shape)
                num = fd(lambda: enc[li][which], lambda a: None, idx)
                assert abs(num - grad[idx]) <= 1e-5 * scale + 1e-9, (li, which, idx, num, grad[idx])
    for which in (0, 1):
        arr = dec[which]
        for _ in range(6):
            idx = tuple(rng.integers(s) for s in arr.shape)
            num = fd(lambda: dec[which], lambda a: None, idx)
            assert abs(num - g_dec[which][idx]) <= 1e-5 * (np.max(np.abs(g_dec[which])) + 1e-12) + 1e-9


def test_split_precision_gradients_reduce_to_the_exact_ones():
    """The split-operand forward (tensor-core precision model) changes only the forward values:
    with bfloat16-representable weights and inputs its products are exact, so its gradients
    equal the exact ones up to the float32 storage of the activations; on general weights they
    stay within the split's rounding of the exact gradients when no ReLU or residual sign sits
    that close to its kink."""
    from oracle import encoder as E
    noisy, clean, enc, dec = _setup()
    enc_b = [(E.bf16_round(Wm), E.bf16_round(b)) for Wm, b in enc]
    noisy_b = E.bf16_round(noisy / 10.0) * 10.0          # depth / 10 is then a bfloat16 number
    L0, g0, d0 = T.gradients(noisy_b, clean, 10.0, enc_b, dec)
    L1, g1, d1 = T.gradients(noisy_b, clean, 10.0, enc_b, dec, split=True)
    assert abs(L1 - L0) <= 1e-6 * L0
    for (a, b), (c, d) in zip(g0, g1):
        assert np.max(np.abs(a - c)) <= 1e-5 * np.max(np.abs(a))
        assert np.max(np.abs(b - d)) <= 1e-5 * np.max(np.abs(b))
    L2, g2, _ = T.gradients(noisy, clean, 10.0, enc, dec, split=True)
    Lx, gx, _ = T.gradients(noisy, clean, 10.0, enc, dec)
    xs, _ = T.forward(noisy, 10.0, enc)
    margin = min(np.min(np.abs(x[np.abs(x) > 0])) for x in xs[1:])
    assert abs(L2 - Lx) <= 1e-4 * Lx
    if margin > 1e-4:                                   # no kink within reach of the split's rounding
        for (a, _), (c, _) in zip(gx, g2):
            assert np.max(np.abs(a - c)) <= 1e-3 * np.max(np.abs(a))


def test_adam_first_step_is_lr_sign():
    p = [np.array([1.0, -2.0, 3.0])]
    g = [np.array([0.5, -1e-3, 0.0])]
    out, m, v = T.adam_step(p, g, [np.zeros(3)], [np.zeros(3)], 1, 0.01)
    np.testing.assert_allclose(out[0], [0.99, -1.99, 3.0], rtol=0, atol=1e-7)


def _scene():
    gates = W.gate_track(2)
    cams = W.camera_views(3, gates, seed=5)
    kw = dict(width=64, height=48, fx=38.5, fy=38.5, cx=32.0, cy=24.0, max_range=10.0)
    return gates, cams, kw


def test_query_sampler_geometry():
    from oracle import gate_sdf as S
    from oracle.dynamics import quat_rotate
    gates, cams, kw = _scene()
    p, lab = T.sample_queries(cams, gates, 512, near_frac=0.5, seed=7, frame=0, **kw)
    assert p.shape == (3, 512, 3) and lab.shape == (3, 512)
    world = quat_rotate(np.broadcast_to(cams[:, None, 3:7] / np.linalg.norm(cams[:, None, 3:7], axis=-1, keepdims=True),
                                        p.shape[:-1] + (4,)), p) + cams[:, None, 0:3]
    per_gate = np.stack([S.frame_sdf(S.to_gate_frame(world.reshape(-1, 3), g).reshape(world.shape)) for g in gates])
    np.testing.assert_allclose(lab, per_gate.min(axis=0), rtol=0, atol=1e-5)      # float32 quaternions
    # points near a gate lie in its box grown by 0.3 m; frustum points are in front of the camera,
    # project into the image and have depth in [0.2, max_range]
    pg = np.stack([S.to_gate_frame(world.reshape(-1, 3), g).reshape(world.shape) for g in gates])
    in_box = np.any(np.all(np.abs(pg) <= np.array([0.4, 1.05, 1.05]) + 1e-9, axis=-1), axis=0)
    u = kw["cx"] - p[..., 1] / p[..., 0] * kw["fx"]
    v = kw["cy"] - p[..., 2] / p[..., 0] * kw["fy"]
    in_view = (p[..., 0] >= 0.2 - 1e-9) & (p[..., 0] <= 10.0 + 1e-9) & (u >= -1e-9) & (u <= 64 + 1e-9) & \
        (v >= -1e-9) & (v <= 48 + 1e-9)
    assert np.all(in_box | in_view)
    assert 0.35 < np.mean(in_box & ~in_view) + 0.5 * np.mean(in_box & in_view) < 0.65
    assert np.mean(lab < 0.3) > 0.2                     # many points near the frames


def test_sdf_term_gradient_matches_central_differences():
    rng = np.random.default_rng(2)
    gates, cams, kw = _scene()
    p, lab = T.sample_queries(cams, gates, 64, near_frac=0.5, seed=3, frame=1, **kw)
    dec = W.xavier_mlp(1, in_dim=3 + 6 * 2 + 64)
    z = rng.normal(0, 1, (3, 64))
    L, dz = T.sdf_term(z, p, lab, dec, 2)
    h = 1e-6
    for _ in range(12):
        i, c = rng.integers(3), rng.integers(64)
        zp, zm = z.copy(), z.copy()
        zp[i, c] += h
        zm[i, c] -= h
        num = (T.sdf_term(zp, p, lab, dec, 2)[0] - T.sdf_term(zm, p, lab, dec, 2)[0]) / (2 * h)
        assert abs(num - dz[i, c]) <= 1e-6 * (np.max(np.abs(dz)) + 1e-12) + 1e-9


def test_joint_gradients_reduce_to_reconstruction_and_match_differences():
    noisy, clean, enc, dec = _setup()
    gates, cams, kw = _scene()
    p, lab = T.sample_queries(cams[:2], gates, 32, near_frac=0.5, seed=3, frame=1, **kw)
    sdf_dec = W.xavier_mlp(1)
    L0, g0, gd0 = T.gradients(noisy, clean, 10.0, enc, dec)
    L, Lr, Ls, g, gd = T.gradients_joint(noisy, clean, 10.0, enc, dec, p, lab, sdf_dec, 0, 1.0, 0.0)
    assert abs(L - L0) < 1e-14
    for (a, b), (c, d) in zip(g, g0):
        np.testing.assert_array_equal(a, c)
    # the SDF term alone: encoder weight gradients against central differences
    L, Lr, Ls, g, gd = T.gradients_joint(noisy, clean, 10.0, enc, dec, p, lab, sdf_dec, 0, 0.0, 1.0)
    assert np.all(gd[0] == 0.0)

    def sdf_loss():
        _, z = T.forward(noisy, 10.0, enc)
        return T.sdf_term(z, p, lab, sdf_dec, 0)[0]

    rng = np.random.default_rng(4)
    h = 1e-6
    for li in (0, 2, 4):
        Wt = enc[li][0]
        scale = np.max(np.abs(g[li][0]))
        for _ in range(4):
            idx = tuple(rng.integers(s) for s in Wt.shape)
            old = Wt[idx]
            Wt[idx] = old + h
            lp = sdf_loss()
            Wt[idx] = old - h
            lm = sdf_loss()
            Wt[idx] = old
            assert abs((lp - lm) / (2 * h) - g[li][0][idx]) <= 1e-5 * scale + 1e-9


def test_decoder_grads_match_frozen_dz_and_central_differences():
    rng = np.random.default_rng(8)
    gates, cams, kw = _scene()
    p, lab = T.sample_queries(cams, gates, 48, near_frac=0.5, seed=3, frame=4, **kw)
    dec = [(W.astype(np.float64), b.astype(np.float64) + 0.01 * rng.normal(size=b.shape))
           for W, b in W.xavier_mlp(2, in_dim=3 + 6 + 64)]
    z = rng.normal(0, 1, (3, 64))
    L, dz, gl = T.decoder_grads(z, p, lab, dec, 1)
    L2, dz2 = T.sdf_term(z, p, lab, dec, 1)
    assert abs(L - L2) < 1e-12
    np.testing.assert_allclose(dz, dz2, rtol=1e-10, atol=1e-14)
    h = 1e-6
    for li in range(5):
        for which in (0, 1):
            arr = dec[li][which]
            ref = gl[li][which]
            scale = np.max(np.abs(ref)) + 1e-12
            for _ in range(4):
                idx = tuple(rng.integers(s) for s in arr.shape)
                old = arr[idx]
                arr[idx] = old + h
                lp = T.sdf_term(z, p, lab, dec, 1)[0]
                arr[idx] = old - h
                lm = T.sdf_term(z, p, lab, dec, 1)[0]
                arr[idx] = old
                assert abs((lp - lm) / (2 * h) - ref[idx]) <= 1e-5 * scale + 1e-10, (li, which, idx)
