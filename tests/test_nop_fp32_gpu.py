"""Gradient check of the neural-operator kernels in FP32 operand mode
(nop_set_fp32): forward output, input gradient and every layer's weight and
bias gradient against the FP64 oracle without operand rounding.

Tolerance 1e-5 relative L2 per quantity.  In this mode every product and sum
is an FP32 operation on unrounded operands, so each layer contributes about
the FP32 rounding of its sums (2^-24 times the square root of the 9 c_in
terms of a convolution, or of the pixel count of a weight-gradient chunk),
and the reverse pass can amplify that by the cancellation of the random
network (the BF16-operand tests measure it at up to about 100 at full
width): 6e-8 x 30 x 3 leaves 1e-5 with room at 16 channels and at the
default widths.  The oracle's own backward is checked against central
finite differences on the CPU (tests/test_oracle_nop.py)."""
import numpy as np
import pytest

from oracle import nop as onop

pytestmark = pytest.mark.gpu

H, W, B = 24, 40, 2          # levels 24x40, 12x20, 6x10, 3x5
CIN, COUT = 3, 4


def _rel(a, b):
    return float(np.linalg.norm(np.ravel(a) - np.ravel(b)) / np.linalg.norm(np.ravel(b)))


@pytest.mark.parametrize("ch", [(16, 16, 16, 16), (32, 64, 96, 128)])
def test_fp32_gradients_match_fp64_oracle(ch):
    import torch
    from paper_2607_07432_b300.nop import NeuralOperator
    rng = np.random.Generator(np.random.PCG64(21))
    x = rng.standard_normal((B, H, W, CIN)).astype(np.float32)
    dy = rng.standard_normal((B, H, W, COUT)).astype(np.float32)
    n = NeuralOperator(height=H, width=W, max_batch=B, channels=ch)
    n.init_params(5)
    n.set_fp32(True)
    theta = n.params().astype(np.float64)
    xd = torch.from_numpy(x).cuda()
    y = torch.empty((B, H, W, COUT), device="cuda")
    n.forward(xd, y)
    dp = torch.empty(n.n_params, device="cuda")
    dx = torch.empty((B, H, W, CIN), device="cuda")
    n.backward(xd, torch.from_numpy(dy).cuda(), dp, dx)
    # back on the BF16 tensor-core path the same network is farther away
    n.set_fp32(False)
    y_bf = torch.empty((B, H, W, COUT), device="cuda")
    n.forward(xd, y_bf)
    n.close()
    yo, cache = onop.forward(theta, x.astype(np.float64), CIN, COUT, ch)
    go, gxo = onop.backward(theta, cache, dy.astype(np.float64), CIN, COUT, ch)
    assert _rel(y.cpu().numpy(), yo) < 1e-5
    assert _rel(y_bf.cpu().numpy(), yo) > 1e-4
    assert _rel(dx.cpu().numpy(), gxo) < 1e-5
    dp = dp.cpu().numpy().astype(np.float64)
    off = 0
    for (ci, co), name in zip(onop.layer_shapes(CIN, COUT, ch), onop.LAYER_NAMES):
        nw = co * 9 * ci
        assert _rel(dp[off:off + nw], go[off:off + nw]) < 1e-5, (name, "W")
        assert _rel(dp[off + nw:off + nw + co], go[off + nw:off + nw + co]) < 1e-5, (name, "b")
        off += nw + co
    assert off == len(go)
