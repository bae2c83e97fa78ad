"""The FLOP count behind the warm-start network's reported rates (CPU): the
sum over the oracle's convolution shapes of 2 x 9 x c_in x c_out per pixel
of each layer's resolution level."""
import pytest

from oracle import unet as ou
from paper_2406_18356_gb300.warm_start import conv_flops


def _levels(levels):
    out = []
    for lv in range(levels):
        out += [lv, lv]
    for lv in range(levels - 2, -1, -1):
        out += [lv, lv]
    return out + [0]


@pytest.mark.parametrize("levels,width,side", [(6, 6, 512), (3, 16, 512), (2, 8, 16)])
def test_conv_flops_follow_the_oracle_layers(levels, width, side):
    shapes = ou.UNetSpec(levels=levels, width=width).conv_shapes()
    want = sum(2 * 9 * ci * co * (side >> lv) ** 2 for (co, ci), lv in zip(shapes, _levels(levels)))
    assert conv_flops(levels, width, side) == want


def test_configured_network_forward_flops():
    # 6 levels, width 6 at 512 px: the count the reported 512 px rates divide
    assert conv_flops(6, 6, 512) == 4_926_210_048
