"""The tensor-core (tcgen05) convolution path of the warm-start network:
image rows that are multiples of 128 pixels run their 3x3 convolutions
(forward and input gradient) on tcgen05 MMAs with tensor-memory
accumulators.  Checked against the FP64 oracle with the same BF16 operand
rounding: centre-tap identity weights give the oracle's output bit for bit
(every pixel / channel placement of the operands and accumulators is
exercised), and a 16-channel network matches the forward pass to 1e-4 and
every gradient to 1e-2 (the bars of the mma.sync path's tests)."""
import numpy as np
import pytest

from oracle import nop as onop

pytestmark = pytest.mark.gpu

H, W, B = 8, 256, 2   # forward and input gradient: levels 8x256 and 4x128 on tcgen05, 2x64 and 1x32 on
#                        mma.sync; weight gradient: levels 0-2 on tcgen05, 1x32 on mma.sync
CIN, COUT = 3, 4


def _rng(seed):
    return np.random.Generator(np.random.PCG64(seed))


def _rel(a, b):
    return float(np.linalg.norm(np.ravel(a) - np.ravel(b)) / np.linalg.norm(np.ravel(b)))


@pytest.mark.parametrize("C", [16, 32, 128])
def test_identity_network_is_exact_on_tensor_cores(C):
    import torch
    from paper_2607_07432_b300.nop import NeuralOperator
    n = NeuralOperator(height=H, width=W, max_batch=B, in_channels=min(C, 16), out_channels=min(C, 16),
                       channels=(C, C, C, C))
    cio = min(C, 16)
    parts = []
    for ci, co in onop.layer_shapes(cio, cio, (C, C, C, C)):
        Wt = np.zeros((co, 3, 3, ci))
        Wt[:, 1, 1, :] = np.eye(co, ci)
        parts += [Wt.ravel(), np.zeros(co)]
    theta = np.concatenate(parts)
    n.set_params(theta.astype(np.float32))
    x = (1.0 + _rng(12).random((B, H, W, cio))).astype(np.float32)
    y = torch.empty((B, H, W, cio), device="cuda")
    n.forward(torch.from_numpy(x).cuda(), y)
    n.close()
    yo, _ = onop.forward(theta, x.astype(np.float64), cio, cio, (C, C, C, C), bf16=True)
    assert np.array_equal(y.cpu().numpy().astype(np.float64), yo)


def test_small_network_matches_oracle_on_tensor_cores():
    import torch
    from paper_2607_07432_b300.nop import NeuralOperator
    rng = _rng(21)
    x = rng.standard_normal((B, H, W, CIN)).astype(np.float32)
    dy = rng.standard_normal((B, H, W, COUT)).astype(np.float32)
    ch = (16, 16, 16, 16)
    n = NeuralOperator(height=H, width=W, max_batch=B, channels=ch)
    n.init_params(3)
    theta = n.params().astype(np.float64)
    y = torch.empty((B, H, W, COUT), device="cuda")
    xd = torch.from_numpy(x).cuda()
    n.forward(xd, y)
    dp = torch.empty(n.n_params, device="cuda")
    dx = torch.empty((B, H, W, CIN), device="cuda")
    n.backward(xd, torch.from_numpy(dy).cuda(), dp, dx)
    n.close()
    yo, cache = onop.forward(theta, x.astype(np.float64), CIN, COUT, ch, bf16=True)
    assert _rel(y.cpu().numpy(), yo) < 1e-4
    g, gx = onop.backward(theta, cache, dy.astype(np.float64), CIN, COUT, ch, bf16=True)
    assert _rel(dx.cpu().numpy(), gx) < 1e-2
    off = 0
    dp = dp.cpu().numpy()
    for (ci, co), name in zip(onop.layer_shapes(CIN, COUT, ch), onop.LAYER_NAMES):
        k = co * 9 * ci + co
        assert _rel(dp[off:off + k], g[off:off + k]) < 1e-2, name
        off += k


def test_wide_network_forward_matches_oracle():
    """Channels 32-128 (the study's network) at 8x256: forward within the
    BF16 cascade bar of the mma.sync tests (1e-2)."""
    import torch
    from paper_2607_07432_b300.nop import NeuralOperator
    ch = (32, 64, 96, 128)
    x = _rng(22).standard_normal((B, H, W, CIN)).astype(np.float32)
    n = NeuralOperator(height=H, width=W, max_batch=B, channels=ch)
    n.init_params(5)
    theta = n.params().astype(np.float64)
    y = torch.empty((B, H, W, COUT), device="cuda")
    n.forward(torch.from_numpy(x).cuda(), y)
    n.close()
    yo, _ = onop.forward(theta, x.astype(np.float64), CIN, COUT, ch, bf16=True)
    assert _rel(y.cpu().numpy(), yo) < 1e-2


def test_wide_network_backward_matches_oracle_on_tensor_cores():
    """Channels 32-128 at 8x256: the weight gradients of the levels whose
    rows are multiples of 64 pixels come from the tcgen05 weight-gradient
    kernel (M = c_out up to 128, several 32-channel input tiles).  As in the
    full-width mma.sync test, each layer's gradient must be as close to the
    FP64 gradient as the BF16-operand oracle is (within 1.5x) and no farther
    from that oracle than twice the oracle's own distance from FP64."""
    import torch
    from paper_2607_07432_b300.nop import NeuralOperator
    ch = (32, 64, 96, 128)
    rng = _rng(23)
    x = rng.standard_normal((B, H, W, CIN)).astype(np.float32)
    dy = rng.standard_normal((B, H, W, COUT)).astype(np.float32)
    n = NeuralOperator(height=H, width=W, max_batch=B, channels=ch)
    n.init_params(5)
    theta = n.params().astype(np.float64)
    dp = torch.empty(n.n_params, device="cuda")
    dx = torch.empty((B, H, W, CIN), device="cuda")
    n.backward(torch.from_numpy(x).cuda(), torch.from_numpy(dy).cuda(), dp, dx)
    n.close()
    dp = dp.cpu().numpy().astype(np.float64)
    _, cache = onop.forward(theta, x.astype(np.float64), CIN, COUT, ch, bf16=True)
    g, _ = onop.backward(theta, cache, dy.astype(np.float64), CIN, COUT, ch, bf16=True)
    _, c64 = onop.forward(theta, x.astype(np.float64), CIN, COUT, ch)
    g64, _ = onop.backward(theta, c64, dy.astype(np.float64), CIN, COUT, ch)
    off = 0
    for (ci, co), name in zip(onop.layer_shapes(CIN, COUT, ch), onop.LAYER_NAMES):
        k = co * 9 * ci + co
        a, b, c = dp[off:off + k], g[off:off + k], g64[off:off + k]
        assert _rel(a, c) <= 1.5 * _rel(b, c) + 1e-3, (name, _rel(a, c), _rel(b, c))
        assert _rel(a, b) <= 2.0 * _rel(b, c) + 1e-2, (name, _rel(a, b), _rel(b, c))
        off += k
