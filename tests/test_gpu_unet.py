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


# (6, 6, 128): the configured warm-start network's shape (6 levels, base width
# 6: 1,106,455 parameters) on the smallest image its 5 poolings take
@pytest.mark.parametrize("levels,width,side", [(3, 16, 32), (2, 8, 16), (3, 16, 48), (6, 6, 128)])
def test_forward_matches_oracle(ms, levels, width, side):
    net, spec, params, x, t, xd, td = _case(ms, levels, width, side, 1)
    y = net.forward(xd).cpu().numpy()
    ref, _ = ou.forward(spec, params, x.astype(np.float32).astype(np.float64), quantize=True)
    assert rel(y, ref) <= 2e-3
    net.close()


def _flips(got, want):
    """Elements where two bfloat16 arrays differ, and the largest difference
    in units of the bfloat16 spacing at the larger magnitude.  Values within
    2^-16 of the array's largest magnitude count as one step: there an FP32
    sum that cancels can round differently by more than one spacing of its
    small result, which a rounding flip of a large value never does."""
    d = np.abs(got - want)
    n = int(np.count_nonzero(d))
    if n == 0:
        return 0, 0.0
    scale = np.maximum(np.abs(got), np.abs(want))
    floor = 2.0 ** -16 * max(float(np.max(np.abs(want))), 1e-30)
    ulp = np.exp2(np.floor(np.log2(np.maximum(scale, floor))) - 7)
    return n, float(np.max(d / np.maximum(ulp, floor)))


@pytest.mark.parametrize("levels,width,side", [(3, 16, 32), (2, 8, 16), (3, 16, 48), (6, 6, 128)])
def test_gradients_match_oracle_layer_by_layer(ms, levels, width, side):
    """Every layer's weight and bias gradient against the oracle's products
    of the device's own stored bfloat16 input activation and pre-activation
    gradient (teacher forcing), so a rounding flip earlier in the network
    cannot propagate: the two sides then differ only by FP32 against FP64
    accumulation, held at 5e-3 relative.  Rounding flips between the device's
    stored values and the oracle's recomputation of them from the device's
    inputs are counted and printed: each is one bfloat16 step."""
    net, spec, params, x, t, xd, td = _case(ms, levels, width, side, 2)
    net.keep_intermediates(True)
    y, loss, g = net.gradients(xd, td)
    got = unpack(spec, g)
    shapes = spec.conv_shapes()
    level = _layer_levels(levels)
    flips_fwd = flips_bwd = total = 0
    for k, (co, ci) in enumerate(shapes):
        hl = side >> level[k]
        a_in = net.layer_tensor(k, "in", (hl, hl, ci)).astype(np.float64)
        dz = net.layer_tensor(k, "grad", (hl, hl, co)).astype(np.float64)
        want_w = ou.conv3x3_grad_weight(a_in, dz)
        want_b = dz.sum(axis=(0, 1))
        ew, eb = rel(got[k]["w"], want_w), rel(got[k]["b"], want_b)
        assert ew <= 5e-3 and eb <= 5e-3, (k, ew, eb)
        if k < len(shapes) - 1:   # forward: out = bf16(relu(conv(a_in)))
            out = net.layer_tensor(k, "out", (hl, hl, co)).astype(np.float64)
            ref = ou.bf16(np.maximum(ou.conv3x3(a_in, ou.bf16(params[k]["w"]), params[k]["b"]),
                                     0.0))
            n, worst = _flips(out, ref)
            assert worst <= 1.0 + 1e-9, (k, worst)
            flips_fwd += n
            total += out.size
        if k + 1 < len(shapes) - 1 and level[k + 1] == level[k] and shapes[k + 1][1] == co:
            # backward within a level: dz_k = bf16(dx_{k+1} * relu'(out_k))
            out = net.layer_tensor(k, "out", (hl, hl, co)).astype(np.float64)
            dz_next = net.layer_tensor(k + 1, "grad", (hl, hl, shapes[k + 1][0]))
            dx = ou.conv3x3_grad_input(dz_next.astype(np.float64), ou.bf16(params[k + 1]["w"]))
            n, worst = _flips(dz, ou.bf16(dx * (out > 0)))
            assert worst <= 1.0 + 1e-9, (k, worst)
            flips_bwd += n
    print(f"unet {levels}x{width} @ {side}: {flips_fwd} forward flips of {total} stored "
          f"values, {flips_bwd} backward flips")
    net.close()


def _layer_levels(levels):
    """Resolution level of every conv in execution order."""
    out = []
    for lv in range(levels):
        out += [lv, lv]
    for lv in range(levels - 2, -1, -1):
        out += [lv, lv]
    return out + [0]


def test_gradients_match_oracle_end_to_end(ms):
    """The small case, where no rounding flip occurs: the whole backward
    chain against the oracle run from the same inputs."""
    net, spec, params, x, t, xd, td = _case(ms, 2, 8, 16, 2)
    y, loss, g = net.gradients(xd, td)
    x64 = x.astype(np.float32).astype(np.float64)
    t64 = t.astype(np.float32).astype(np.float64)
    ref_y, cache = ou.forward(spec, params, x64, quantize=True)
    ref_g = pack(ou.backward(spec, params, cache, ref_y, t64, quantize=True))
    assert abs(loss - ou.loss(ref_y, t64)) <= 2e-3 * ou.loss(ref_y, t64)
    assert rel(g, ref_g) <= 1e-4
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
