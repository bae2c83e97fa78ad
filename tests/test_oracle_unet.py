"""Pins of the warm-start network oracle (CPU): bfloat16 rounding against
torch's conversion, the convolution against scipy's correlation, adjoint
identities of every layer, and the network's gradients against central finite
differences."""
import numpy as np
import pytest
from scipy.signal import correlate2d

from oracle import unet


def test_bf16_rounding_matches_torch():
    import torch
    rng = np.random.default_rng(0)
    x = np.concatenate([rng.standard_normal(10000) * 10 ** rng.uniform(-6, 6, 10000),
                        [0.0, -0.0, 1.0, 1.00390625, 1.005859375, 65504.0, 3.0e38]])
    want = torch.from_numpy(x.astype(np.float32)).to(torch.bfloat16).to(torch.float64).numpy()
    np.testing.assert_array_equal(unet.bf16(x), want)
    # ties go to even: 1 + 2^-8 lies halfway between 1 and 1 + 2^-7
    assert unet.bf16(np.array([1.0 + 2.0 ** -8]))[0] == 1.0
    assert unet.bf16(np.array([1.0 + 3 * 2.0 ** -8]))[0] == 1.0 + 2.0 ** -6


def test_conv3x3_matches_scipy_correlation():
    rng = np.random.default_rng(1)
    x = rng.standard_normal((9, 7, 3))
    w = rng.standard_normal((4, 3, 3, 3))
    b = rng.standard_normal(4)
    y = unet.conv3x3(x, w, b)
    for co in range(4):
        ref = b[co] + sum(correlate2d(x[:, :, ci], w[co, :, :, ci], mode="same")
                          for ci in range(3))
        np.testing.assert_allclose(y[:, :, co], ref, rtol=1e-12, atol=1e-12)


def test_layer_adjoint_identities():
    rng = np.random.default_rng(2)
    x = rng.standard_normal((8, 6, 3))
    w = rng.standard_normal((5, 3, 3, 3))
    g = rng.standard_normal((8, 6, 5))
    zero = np.zeros(5)
    lhs = np.sum(unet.conv3x3(x, w, zero) * g)
    assert abs(lhs - np.sum(x * unet.conv3x3_grad_input(g, w))) <= 1e-10 * abs(lhs)
    assert abs(lhs - np.sum(w * unet.conv3x3_grad_weight(x, g))) <= 1e-10 * abs(lhs)
    a = rng.standard_normal((8, 6, 2))
    p = rng.standard_normal((4, 3, 2))
    assert np.isclose(np.sum(unet.avgpool2(a) * p), np.sum(a * unet.avgpool2_grad(p)))
    assert np.isclose(np.sum(unet.upsample2(p) * a), np.sum(p * unet.upsample2_grad(a)))
    # pooling averages, upsampling copies
    np.testing.assert_allclose(unet.avgpool2(np.ones((4, 4, 1))), np.ones((2, 2, 1)))
    np.testing.assert_array_equal(unet.upsample2(p)[1::2, ::2], p)


def test_conv_shapes_follow_the_architecture():
    spec = unet.UNetSpec(levels=3, width=16, in_channels=2)
    assert spec.conv_shapes() == [(16, 2), (16, 16), (32, 16), (32, 32), (64, 32), (64, 64),
                                  (32, 96), (32, 32), (16, 48), (16, 16), (1, 16)]


@pytest.mark.parametrize("levels", [2, 3])
def test_network_gradient_matches_finite_differences(levels):
    spec = unet.UNetSpec(levels=levels, width=4, in_channels=2)
    rng = np.random.default_rng(3)
    params = unet.init_params(spec, rng)
    for p in params:
        p["b"] = rng.standard_normal(p["b"].shape) * 0.1
    x = rng.standard_normal((8, 8, 2))
    t = rng.standard_normal((8, 8))
    y, cache = unet.forward(spec, params, x)
    grads = unet.backward(spec, params, cache, y, t)
    h = 1e-6
    for k in rng.choice(len(params), size=min(6, len(params)), replace=False):
        for name in ("w", "b"):
            arr = params[k][name]
            for _ in range(3):
                idx = tuple(rng.integers(0, s) for s in arr.shape)
                old = arr[idx]
                arr[idx] = old + h
                lp = unet.loss(unet.forward(spec, params, x)[0], t)
                arr[idx] = old - h
                lm = unet.loss(unet.forward(spec, params, x)[0], t)
                arr[idx] = old
                fd = (lp - lm) / (2 * h)
                assert abs(fd - grads[k][name][idx]) <= 1e-6 + 1e-5 * abs(fd), (k, name, idx)


def test_quantized_forward_is_close_to_exact():
    spec = unet.UNetSpec(levels=3, width=8)
    rng = np.random.default_rng(4)
    params = unet.init_params(spec, rng)
    x = rng.standard_normal((16, 16, 2))
    y, _ = unet.forward(spec, params, x)
    yq, _ = unet.forward(spec, params, x, quantize=True)
    rel = np.linalg.norm(yq - y) / np.linalg.norm(y)
    assert 1e-5 < rel < 3e-2   # bfloat16 has an 8-bit significand


def test_adam_step_closed_form():
    params = [{"w": np.array([1.0]), "b": np.array([0.0])}]
    grads = [{"w": np.array([0.5]), "b": np.array([0.0])}]
    state = {}
    unet.adam_step(params, grads, state, lr=0.1)
    # first step: m^ = g, v^ = g^2, so the update is lr * g / (|g| + eps)
    assert abs(params[0]["w"][0] - (1.0 - 0.1 * 0.5 / (0.5 + 1e-8))) < 1e-15
