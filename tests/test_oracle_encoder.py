"""Pins for the depth encoder of the oracle (the convolutional reading of E_theta, Sec. III-B):
the stride-2 convolution against brute-force loops and against PyTorch's CPU convolution, closed
forms for delta and box kernels, and closed forms and invariances of the whole encoder."""
import numpy as np
import pytest

import workloads as W
from oracle import encoder as E


def _brute_conv(x, w, b):
    ci, h, wd = x.shape
    co = w.shape[0]
    ho, wo = (h + 1) // 2, (wd + 1) // 2
    out = np.zeros((co, ho, wo))
    for o in range(co):
        for i in range(ho):
            for j in range(wo):
                acc = b[o]
                for c in range(ci):
                    for ky in range(3):
                        for kx in range(3):
                            yy, xx = 2 * i + ky - 1, 2 * j + kx - 1
                            if 0 <= yy < h and 0 <= xx < wd:
                                acc += w[o, c, ky, kx] * x[c, yy, xx]
                out[o, i, j] = acc
    return out


@pytest.mark.parametrize("h,w", [(5, 7), (6, 4), (1, 1), (2, 3)])
def test_conv_brute_force(h, w):
    rng = np.random.default_rng(h * 10 + w)
    x = rng.standard_normal((2, h, w))
    wt = rng.standard_normal((3, 2, 3, 3))
    b = rng.standard_normal(3)
    np.testing.assert_allclose(E.conv3x3_s2(x, wt, b), _brute_conv(x, wt, b), rtol=0, atol=1e-12)


@pytest.mark.parametrize("h,w", [(17, 24), (30, 40), (9, 9)])
def test_conv_matches_torch_cpu(h, w):
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(h + w)
    x = rng.standard_normal((4, h, w))
    wt = rng.standard_normal((8, 4, 3, 3))
    b = rng.standard_normal(8)
    ref = torch.nn.functional.conv2d(torch.from_numpy(x)[None], torch.from_numpy(wt), torch.from_numpy(b),
                                     stride=2, padding=1)[0].numpy()
    np.testing.assert_allclose(E.conv3x3_s2(x, wt, b), ref, rtol=1e-12, atol=1e-12)


def test_delta_kernel_subsamples():
    x = np.arange(2 * 7 * 9, dtype=np.float64).reshape(2, 7, 9)
    wt = np.zeros((2, 2, 3, 3))
    wt[0, 0, 1, 1] = 1.0                      # centre tap of channel 0 -> output 0
    wt[1, 1, 1, 1] = -2.0                     # centre tap of channel 1 -> output 1
    out = E.conv3x3_s2(x, wt, np.array([0.5, 0.0]))
    np.testing.assert_array_equal(out[0], x[0, ::2, ::2] + 0.5)
    np.testing.assert_array_equal(out[1], -2.0 * x[1, ::2, ::2])


def test_box_kernel_counts_taps_inside():
    """All-ones 3x3 kernel on a constant image: 9 c inside, 4 c at the top-left corner (rows and
    columns -1 are padding), 6 c along the top edge."""
    c = 0.7
    out = E.conv3x3_s2(np.full((1, 8, 8), c), np.ones((1, 1, 3, 3)), np.zeros(1))[0]
    assert abs(out[0, 0] - 4 * c) < 1e-12 and abs(out[0, 2] - 6 * c) < 1e-12 and abs(out[2, 2] - 9 * c) < 1e-12


def test_output_sizes():
    x = np.zeros((1, 480, 640))
    sizes = []
    for co in (16, 32, 64, 64):
        x = E.conv3x3_s2(x, np.zeros((co, x.shape[0], 3, 3)), np.zeros(co))
        sizes.append(x.shape)
    assert sizes == [(16, 240, 320), (32, 120, 160), (64, 60, 80), (64, 30, 40)]


def test_encode_constant_chain_closed_form():
    """With zero convolution weights every x_l is relu(b_l) everywhere, so z = W5 relu(b4) + b5."""
    layers = [(np.zeros_like(w), b) for w, b in W.encoder_weights(3)[:4]] + [W.encoder_weights(3)[4]]
    b5 = np.linspace(-1, 1, 64)
    layers[4] = (layers[4][0], b5)
    z = E.encode(np.random.default_rng(0).uniform(0, 10, (2, 24, 32)), 10.0, layers)
    want = layers[4][0].astype(np.float64) @ np.maximum(layers[3][1].astype(np.float64), 0.0) + b5
    np.testing.assert_allclose(z, np.stack([want, want]), rtol=0, atol=1e-12)


def test_encode_scale_invariance_and_batch():
    layers = W.encoder_weights(5)
    rng = np.random.default_rng(1)
    imgs = rng.uniform(0.0, 10.0, (3, 30, 40))
    z = E.encode(imgs, 10.0, layers)
    np.testing.assert_allclose(E.encode(imgs * 2.5, 25.0, layers), z, rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(E.encode(imgs[1], 10.0, layers)[0], z[1], rtol=0, atol=0)
    assert np.std(z[0] - z[1]) > 1e-3            # different images give different codes


def test_bf16_round_known_values_and_torch():
    """bfloat16 rounding: exact values stay, ties go to the even pattern, the rest to nearest;
    against PyTorch's CPU float32 -> bfloat16 conversion on random and extreme values."""
    one = 1.0
    assert E.bf16_round(np.array([one]))[0] == 1.0
    assert E.bf16_round(np.array([1.0 + 2.0 ** -8]))[0] == 1.0                    # tie -> even (1.0)
    assert E.bf16_round(np.array([1.0 + 3 * 2.0 ** -8]))[0] == 1.0 + 2.0 ** -6    # tie -> even (up)
    assert E.bf16_round(np.array([1.0 + 2.0 ** -8 + 2.0 ** -12]))[0] == 1.0 + 2.0 ** -7
    assert E.bf16_round(np.array([-3.0]))[0] == -3.0
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(5)
    v = np.concatenate([rng.standard_normal(10000) * 10.0 ** rng.integers(-30, 30, 10000),
                        [0.0, -0.0, 1e-40, 3.0e38]]).astype(np.float32)
    ref = torch.from_numpy(v).to(torch.bfloat16).to(torch.float64).numpy()
    np.testing.assert_array_equal(E.bf16_round(v), ref)


def test_bf16_split_bound_and_exact_cases():
    rng = np.random.default_rng(6)
    a = (rng.standard_normal(20000) * 10.0 ** rng.integers(-8, 8, 20000)).astype(np.float32).astype(np.float64)
    hi, lo = E.bf16_split(a)
    assert np.all(np.abs(a - hi - lo) <= 2.0 ** -16 * np.abs(a))
    exact = E.bf16_round(a)                     # already bfloat16: the remainder is zero
    h2, l2 = E.bf16_split(exact)
    np.testing.assert_array_equal(h2, exact)
    assert not np.any(l2)


def test_split_conv_exact_on_bf16_operands_and_close_otherwise():
    """On operands that are bfloat16 numbers the split convolution is the exact one (the lo parts
    vanish); on general FP32 operands it stays within 3 x 2^-16 of the sum of |products|."""
    rng = np.random.default_rng(7)
    x = E.bf16_round(rng.standard_normal((3, 9, 11)))
    wt = E.bf16_round(rng.standard_normal((4, 3, 3, 3)))
    b = rng.standard_normal(4)
    np.testing.assert_allclose(E.conv3x3_s2_split(x, wt, b), E.conv3x3_s2(x, wt, b), rtol=0, atol=1e-12)
    x = rng.standard_normal((3, 9, 11)).astype(np.float32).astype(np.float64)
    wt = rng.standard_normal((4, 3, 3, 3)).astype(np.float32).astype(np.float64)
    bound = 3 * 2.0 ** -16 * E.conv3x3_s2(np.abs(x), np.abs(wt), np.zeros(4))
    err = np.abs(E.conv3x3_s2_split(x, wt, b) - E.conv3x3_s2(x, wt, b))
    assert np.all(err <= bound + 1e-12)
    assert err.max() > 0.0
