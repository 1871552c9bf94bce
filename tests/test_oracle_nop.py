"""Pins of the neural-operator oracle against definitions that do not reuse
its code: a scalar loop over the convolution's defining sum, adjoint
identities of pooling and up-sampling, central finite differences of the
whole network, the closed form of the first Adam step and exact BF16
rounding cases."""
import numpy as np
import pytest

from oracle import nop as onop

IN, OUT, CH = 3, 4, (4, 6, 8, 10)


def _rng(seed):
    return np.random.Generator(np.random.PCG64(seed))


def test_conv_matches_scalar_definition():
    rng = _rng(1)
    x = rng.standard_normal((2, 4, 6, 3))
    W = rng.standard_normal((5, 3, 3, 3))
    b = rng.standard_normal(5)
    y = onop.conv(x, W, b)
    B, H, Wd, C = x.shape
    ref = np.zeros((B, H, Wd, 5))
    for n in range(B):
        for yy in range(H):
            for xx in range(Wd):
                for o in range(5):
                    s = b[o]
                    for ky in range(3):
                        for kx in range(3):
                            sy, sx = yy + ky - 1, xx + kx - 1
                            if 0 <= sy < H and 0 <= sx < Wd:
                                for i in range(C):
                                    s += W[o, ky, kx, i] * x[n, sy, sx, i]
                    ref[n, yy, xx, o] = s
    assert np.allclose(y, ref, rtol=0, atol=1e-12)


def test_conv_backward_matches_finite_differences():
    rng = _rng(2)
    x = rng.standard_normal((1, 4, 4, 2))
    W = rng.standard_normal((3, 3, 3, 2))
    b = rng.standard_normal(3)
    gy = rng.standard_normal((1, 4, 4, 3))
    gx, gW, gb = onop.conv_backward(x, W, gy)
    f = lambda xx, WW, bb: float(np.sum(onop.conv(xx, WW, bb) * gy))
    h = 1e-6
    for idx in [(0, 0, 0, 0), (0, 1, 2, 1), (0, 3, 3, 0), (0, 2, 0, 1)]:
        e = np.zeros_like(x); e[idx] = h
        fd = (f(x + e, W, b) - f(x - e, W, b)) / (2 * h)
        assert abs(fd - gx[idx]) < 1e-7 * max(1.0, abs(fd))
    for idx in [(0, 0, 0, 0), (2, 1, 2, 1), (1, 2, 0, 0)]:
        e = np.zeros_like(W); e[idx] = h
        fd = (f(x, W + e, b) - f(x, W - e, b)) / (2 * h)
        assert abs(fd - gW[idx]) < 1e-7 * max(1.0, abs(fd))
    assert np.allclose(gb, gy.sum(axis=(0, 1, 2)))


def test_pool_and_up_adjoints():
    rng = _rng(3)
    x = rng.standard_normal((2, 8, 6, 3))
    g = rng.standard_normal((2, 4, 3, 3))
    assert abs(np.sum(onop.pool(x) * g) - np.sum(x * onop.pool_backward(g))) < 1e-12
    xl = rng.standard_normal((2, 4, 3, 3))
    gh = rng.standard_normal((2, 8, 6, 3))
    assert abs(np.sum(onop.up(xl) * gh) - np.sum(xl * onop.up_backward(gh))) < 1e-12
    # pooling an up-sampled field returns it; a constant pools to itself
    assert np.allclose(onop.pool(onop.up(xl)), xl)
    assert np.allclose(onop.pool(np.full((1, 4, 4, 2), 3.5)), 3.5)


def test_layer_shapes_and_count():
    sh = onop.layer_shapes(3, 4, (32, 64, 96, 128))
    assert len(sh) == 15
    assert sh[0] == (3, 32) and sh[7] == (128, 128) and sh[8] == (128, 96) and sh[-1] == (32, 4)
    assert onop.param_count(3, 4, (32, 64, 96, 128)) == sum(co * 9 * ci + co for ci, co in sh)


@pytest.fixture(scope="module")
def small_net():
    rng = _rng(4)
    n = onop.param_count(IN, OUT, CH)
    theta = 0.3 * rng.standard_normal(n)
    x = rng.standard_normal((2, 8, 8, IN))
    gy = rng.standard_normal((2, 8, 8, OUT))
    return theta, x, gy


def test_network_backward_matches_finite_differences(small_net):
    theta, x, gy = small_net
    y, cache = onop.forward(theta, x, IN, OUT, CH)
    gtheta, gx = onop.backward(theta, cache, gy, IN, OUT, CH)
    f = lambda th, xx: float(np.sum(onop.forward(th, xx, IN, OUT, CH)[0] * gy))
    rng = _rng(5)
    h = 1e-6
    # parameters from every layer (first weight, last bias of each layer, random ones)
    idx = []
    off = 0
    for ci, co in onop.layer_shapes(IN, OUT, CH):
        idx += [off, off + co * 9 * ci + co - 1, off + int(rng.integers(0, co * 9 * ci))]
        off += co * 9 * ci + co
    for i in idx:
        e = np.zeros_like(theta); e[i] = h
        fd = (f(theta + e, x) - f(theta - e, x)) / (2 * h)
        assert abs(fd - gtheta[i]) <= 1e-6 * max(1.0, abs(fd)), (i, fd, gtheta[i])
    for _ in range(8):
        j = tuple(int(rng.integers(0, s)) for s in x.shape)
        e = np.zeros_like(x); e[j] = h
        fd = (f(theta, x + e) - f(theta, x - e)) / (2 * h)
        assert abs(fd - gx[j]) <= 1e-6 * max(1.0, abs(fd)), (j, fd, gx[j])


def test_mse_gradient():
    rng = _rng(6)
    y, t = rng.standard_normal((2, 4, 4, 3)), rng.standard_normal((2, 4, 4, 3))
    L, g = onop.mse(y, t)
    assert abs(L - np.sum((y - t) ** 2) / y.size) < 1e-14
    h = 1e-6
    e = np.zeros_like(y); e[1, 2, 3, 0] = h
    fd = (onop.mse(y + e, t)[0] - onop.mse(y - e, t)[0]) / (2 * h)
    assert abs(fd - g[1, 2, 3, 0]) < 1e-8


def test_first_adam_step_closed_form():
    # after one step m_hat = g and v_hat = g^2, so the update is lr g / (|g| + eps)
    g = np.array([0.5, -2.0, 1e-3, 0.0])
    th = np.array([1.0, 1.0, 1.0, 1.0])
    new, m, v = onop.adam_step(th, g, np.zeros(4), np.zeros(4), 1, lr=0.01)
    assert np.allclose(new, th - 0.01 * g / (np.abs(g) + 1e-8), rtol=0, atol=1e-15)
    assert np.allclose(m, 0.1 * g) and np.allclose(v, 0.001 * g * g)


def test_bf16_rounding_cases():
    r = onop.to_bf16(np.array([1.0, 1.0 + 2 ** -8, 1.0 + 2 ** -8 + 2 ** -20, 1.0 + 3 * 2 ** -8, -0.15625, 3.0]))
    assert list(r) == [1.0, 1.0, 1.0 + 2 ** -7, 1.0 + 2 ** -6, -0.15625, 3.0]


def test_identity_weights_give_multiscale_sum():
    # centre-tap identity weights, zero biases and a positive input make every
    # convolution + ReLU the identity, so the U-Net reduces to
    # y = x + up(pool x) + up^2(pool^2 x) + up^3(pool^3 x)
    C = 4
    parts = []
    for ci, co in onop.layer_shapes(C, C, (C, C, C, C)):
        W = np.zeros((co, 3, 3, ci))
        W[:, 1, 1, :] = np.eye(co, ci)
        parts += [W.ravel(), np.zeros(co)]
    theta = np.concatenate(parts)
    x = 1.0 + _rng(7).random((1, 16, 8, C))
    y, _ = onop.forward(theta, x, C, C, (C, C, C, C))
    ref = x.copy()
    p = x
    for k in range(1, 4):
        p = onop.pool(p)
        q = p
        for _ in range(k):
            q = onop.up(q)
        ref = ref + q
    assert np.allclose(y, ref, rtol=0, atol=1e-12)
