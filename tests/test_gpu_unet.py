"""The learned warm start's network on the GPU (bfloat16 tensor-core
products, FP32 accumulation) against the FP64 oracle with the same rounding
points: forward output, loss, every parameter gradient, and the Adam step."""
import numpy as np
import pytest

from oracle import unet as ou

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ms():
    import torch
    import paper_2406_18356_gb300 as pkg
    from paper_2406_18356_gb300 import _build
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    _build.build()
    pkg.load_library()
    return pkg


def unpack(spec, flat):
    params, off = [], 0
    for co, ci in spec.conv_shapes():
        nw = co * 9 * ci
        params.append({"w": flat[off:off + nw].astype(np.float64).reshape(co, 3, 3, ci),
                       "b": flat[off + nw:off + nw + co].astype(np.float64)})
        off += nw + co
    assert off == flat.size
    return params


def pack(params):
    return np.concatenate([np.concatenate([p["w"].ravel(), p["b"].ravel()]) for p in params])


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


def _case(ms, levels, width, side, seed):
    import torch
    net = ms.WarmStartNet(levels=levels, width=width, max_side=side, seed=seed)
    spec = ou.UNetSpec(levels=levels, width=width)
    rng = np.random.default_rng(seed)
    flat = net.get_params()
    params = unpack(spec, flat)
    # non-zero biases exercise the bias paths; the head (created at zero so
    # that the untrained network returns the step-one image) gets weights
    for p in params:
        p["b"] = rng.standard_normal(p["b"].shape) * 0.05
    params[-1]["w"] = rng.standard_normal(params[-1]["w"].shape) * 0.1
    net.set_params(pack(params).astype(np.float32))
    params = unpack(spec, net.get_params())
    x = rng.standard_normal((side, side, 2))
    t = rng.standard_normal((side, side))
    return net, spec, params, x, t, torch.from_numpy(x.astype(np.float32)).cuda(), \
        torch.from_numpy(t.astype(np.float32)).cuda()


@pytest.mark.parametrize("levels,width,side", [(3, 16, 32), (2, 8, 16), (3, 16, 48)])
def test_forward_matches_oracle(ms, levels, width, side):
    net, spec, params, x, t, xd, td = _case(ms, levels, width, side, 1)
    y = net.forward(xd).cpu().numpy()
    ref, _ = ou.forward(spec, params, x.astype(np.float32).astype(np.float64), quantize=True)
    assert rel(y, ref) <= 2e-3
    net.close()


# Tolerances: both sides round the same values to bfloat16 (unit roundoff
# 2^-9), but FP32 and FP64 sums can land on opposite sides of a rounding
# boundary; such a flip changes a value by 2^-8 relative, and through 11
# layers of rounded activations and rounded pre-activation gradients a few
# flips reach about 1e-2 of a gradient (most in the first layer, the end of
# the backward chain).  The small case sums few terms and shows no flip: there
# the two sides agree to FP32 accuracy.
@pytest.mark.parametrize("levels,width,side,tol,tol_layer",
                         [(3, 16, 32, 1e-2, 5e-2), (2, 8, 16, 1e-4, 1e-3)])
def test_gradients_match_oracle(ms, levels, width, side, tol, tol_layer):
    net, spec, params, x, t, xd, td = _case(ms, levels, width, side, 2)
    y, loss, g = net.gradients(xd, td)
    x64 = x.astype(np.float32).astype(np.float64)
    t64 = t.astype(np.float32).astype(np.float64)
    ref_y, cache = ou.forward(spec, params, x64, quantize=True)
    ref_g = pack(ou.backward(spec, params, cache, ref_y, t64, quantize=True))
    assert abs(loss - ou.loss(ref_y, t64)) <= 2e-3 * ou.loss(ref_y, t64)
    assert rel(g, ref_g) <= tol
    # layer by layer (weights and biases of every convolution)
    got, want = unpack(spec, g), unpack(spec, ref_g)
    for k, (a, b) in enumerate(zip(got, want)):
        assert rel(a["w"], b["w"]) <= tol_layer, k
        assert rel(a["b"], b["b"]) <= tol_layer, k
    net.close()


def test_adam_step_matches_oracle_update(ms):
    net, spec, params, x, t, xd, td = _case(ms, 2, 8, 16, 3)
    before = net.get_params().astype(np.float64)
    _, _, g = net.gradients(xd, td)
    net.train_step(xd, td, lr=1e-3)
    after = net.get_params().astype(np.float64)
    p = unpack(spec, before)
    ou.adam_step(p, unpack(spec, g.astype(np.float64)), {}, lr=1e-3)
    want = pack(p)
    # the first Adam step moves every weight by about lr * sign(g)
    assert np.max(np.abs(after - want)) <= 1e-6
    net.close()


def test_untrained_network_returns_the_step_one_image(ms):
    import torch
    net = ms.WarmStartNet(levels=3, width=8, max_side=32, seed=5)
    x = torch.randn((32, 32, 2), device="cuda")
    assert torch.equal(net.forward(x), x[:, :, 0])
    net.close()


def test_training_lowers_the_loss(ms):
    import torch
    net = ms.WarmStartNet(levels=3, width=8, max_side=32, seed=4)
    rng = np.random.default_rng(4)
    x = torch.from_numpy(rng.standard_normal((32, 32, 2)).astype(np.float32)).cuda()
    # target: a smooth function of the inputs the network can fit
    t = (0.5 * x[:, :, 0] - 0.3 * x[:, :, 1]).contiguous()
    first = net.train_step(x, t, lr=3e-3)
    for _ in range(200):
        last = net.train_step(x, t, lr=3e-3)
    assert last < 0.2 * first
    net.close()


def test_rejects_bad_sizes(ms):
    import torch
    net = ms.WarmStartNet(levels=3, width=8, max_side=32, seed=0)
    with pytest.raises(ms.MsError):
        net.forward(torch.zeros((24, 24, 2), device="cuda"))   # not a multiple of 16
    with pytest.raises(ms.MsError):
        net.forward(torch.zeros((64, 64, 2), device="cuda"))   # above max_side
    net.close()
