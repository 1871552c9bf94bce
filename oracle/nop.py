"""Warm-start neural operator, plain numpy FP64 (oracle).

TEST INFRASTRUCTURE ONLY (see the package docstring).  The paper has no
learned component; this is the plain definition of the U-Net that the
library's tensor-core kernels implement, used to check their forward
pass, their input gradient (dgrad) and their weight gradient (wgrad).

Definition (the same network the C ABI documents):
  conv(x; W, b)[p, o] = b[o] + sum_{ky, kx, i} W[o, ky, kx, i] x[p + (ky - 1, kx - 1), i]
      with zero padding outside the image (3x3, stride 1)
  pool(x)[y, x] = mean of the 2x2 children;  up(x)[y, x] = x[y // 2, x // 2]
  encoder  a_l = relu(conv(in_l)), e_l = relu(conv(a_l)),
           in_0 = x, in_l = pool(e_{l-1})                       (l = 0..3)
  decoder  s_l = relu(conv(up(g_{l+1}))), t_l = s_l + e_l,
           g_l = relu(conv(t_l)), g_3 = e_3                      (l = 2, 1, 0)
  output   y = conv(g_0)
  loss     L = mean over batch, pixels and output channels of (y - target)^2
  Adam     bias-corrected, beta1 0.9, beta2 0.999, eps 1e-8.
Parameters are one flat vector, layer after layer (a0 e0 a1 e1 a2 e2 a3 e3
s2 g2 s1 g1 s0 g0 y), each layer W[c_out, 3, 3, c_in] then b[c_out].
Tensors are NHWC [B, H, W, C].

Pinned by tests/test_oracle_nop.py: the convolution against a scalar loop
over the definition, pooling / up-sampling against their adjoint identity,
the full reverse pass against central finite differences, and the first
Adam step against its closed form.

``bf16=True`` rounds every convolution operand (weights, input activations
and, in the reverse pass, output gradients) to the nearest BF16 before the
FP64 products, which is the operand precision the tensor-core path states;
accumulation stays FP64.
"""
import numpy as np

LAYER_NAMES = ["a0", "e0", "a1", "e1", "a2", "e2", "a3", "e3", "s2", "g2", "s1", "g1", "s0", "g0", "y"]


def layer_shapes(in_channels, out_channels, channels):
    """(c_in, c_out) of the 15 convolutions, in parameter order."""
    c = list(channels)
    sh = []
    cin = in_channels
    for l in range(4):
        if l > 0:
            cin = c[l - 1]
        sh.append((cin, c[l]))
        sh.append((c[l], c[l]))
    for l in (2, 1, 0):
        sh.append((c[l + 1], c[l]))
        sh.append((c[l], c[l]))
    sh.append((c[0], out_channels))
    return sh


def param_count(in_channels, out_channels, channels):
    return sum(co * 9 * ci + co for ci, co in layer_shapes(in_channels, out_channels, channels))


def unpack(theta, in_channels, out_channels, channels):
    """Flat vector -> list of (W[c_out, 3, 3, c_in], b[c_out])."""
    out, off = [], 0
    for ci, co in layer_shapes(in_channels, out_channels, channels):
        nw = co * 9 * ci
        W = np.asarray(theta[off:off + nw], dtype=np.float64).reshape(co, 3, 3, ci)
        b = np.asarray(theta[off + nw:off + nw + co], dtype=np.float64)
        out.append((W, b))
        off += nw + co
    return out


def pack(grads):
    return np.concatenate([np.concatenate([dW.ravel(), db.ravel()]) for dW, db in grads])


def to_bf16(a):
    """Round FP64 values to the nearest BF16 (ties to even), via FP32."""
    f = np.asarray(a, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    r = ((u + 0x7FFF + lsb) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


# -- layers ----------------------------------------------------------------
def _shift(x, dy, dx):
    """s[:, y, x] = x[:, y + dy, x + dx] with zeros outside."""
    B, H, W, C = x.shape
    s = np.zeros_like(x)
    ys, yd = (slice(dy, H), slice(0, H - dy)) if dy >= 0 else (slice(0, H + dy), slice(-dy, H))
    xs, xd = (slice(dx, W), slice(0, W - dx)) if dx >= 0 else (slice(0, W + dx), slice(-dx, W))
    s[:, yd, xd, :] = x[:, ys, xs, :]
    return s


def conv(x, W, b, bf16=False):
    if bf16:
        x, W = to_bf16(x), to_bf16(W)
    B, H, Wd, _ = x.shape
    y = np.zeros((B, H, Wd, W.shape[0])) + b
    for ky in range(3):
        for kx in range(3):
            y += _shift(x, ky - 1, kx - 1) @ W[:, ky, kx, :].T
    return y


def conv_backward(x, W, gy, bf16=False):
    """Gradients of conv w.r.t. its input, weights and bias for the output
    gradient gy.  With bf16 every product takes BF16 operands, as on the
    tensor cores: x and W as in the forward pass, and gy too (the bias
    gradient is a plain sum of the unrounded gy)."""
    gb = gy.sum(axis=(0, 1, 2))
    if bf16:
        x, W, gy = to_bf16(x), to_bf16(W), to_bf16(gy)
    gx = np.zeros_like(x)
    gW = np.zeros_like(W)
    for ky in range(3):
        for kx in range(3):
            xs = _shift(x, ky - 1, kx - 1)
            gW[:, ky, kx, :] = np.einsum("bhwo,bhwi->oi", gy, xs)
            # y[p] gets x[p + s] W: x[q] feeds y[q - s]
            gx += _shift(gy @ W[:, ky, kx, :], -(ky - 1), -(kx - 1))
    return gx, gW, gb


def relu(x):
    return np.where(x > 0, x, 0.0)


def pool(x):
    B, H, W, C = x.shape
    return x.reshape(B, H // 2, 2, W // 2, 2, C).mean(axis=(2, 4))


def pool_backward(g):
    return np.repeat(np.repeat(g, 2, axis=1), 2, axis=2) / 4.0


def up(x):
    return np.repeat(np.repeat(x, 2, axis=1), 2, axis=2)


def up_backward(g):
    B, H, W, C = g.shape
    return g.reshape(B, H // 2, 2, W // 2, 2, C).sum(axis=(2, 4))


# -- network ---------------------------------------------------------------
def forward(theta, x, in_channels, out_channels, channels, bf16=False):
    """Returns (y, cache) for x [B, H, W, in_channels]."""
    P = unpack(theta, in_channels, out_channels, channels)
    cache = {}
    k = 0

    def cv(name, inp, act):
        nonlocal k
        W, b = P[k]
        k += 1
        pre = conv(inp, W, b, bf16)
        out = relu(pre) if act else pre
        cache[name] = (inp, pre, out)
        return out

    e = []
    inp = np.asarray(x, dtype=np.float64)
    for l in range(4):
        if l > 0:
            inp = pool(e[l - 1])
        a = cv("a%d" % l, inp, True)
        e.append(cv("e%d" % l, a, True))
    g = e[3]
    for l in (2, 1, 0):
        s = cv("s%d" % l, up(g), True)
        t = s + e[l]
        g = cv("g%d" % l, t, True)
    y = cv("y", g, False)
    return y, cache


def backward(theta, cache, gy, in_channels, out_channels, channels, bf16=False):
    """Reverse pass: returns (flat dL/dtheta, dL/dx) for dL/dy = gy."""
    P = unpack(theta, in_channels, out_channels, channels)
    idx = {n: i for i, n in enumerate(LAYER_NAMES)}
    grads = [None] * len(LAYER_NAMES)

    def cv_back(name, gout, act):
        inp, pre, _ = cache[name]
        W, _ = P[idx[name]]
        gpre = np.where(pre > 0, gout, 0.0) if act else gout
        gin, gW, gb = conv_backward(inp, W, gpre, bf16)
        grads[idx[name]] = (gW, gb)
        return gin

    gg = cv_back("y", gy, False)
    ge = [None] * 4
    for l in (0, 1, 2):
        gt = cv_back("g%d" % l, gg, True)
        ge[l] = gt                                  # t_l = s_l + e_l
        gu = cv_back("s%d" % l, gt, True)
        gg = up_backward(gu)                        # gradient of g_{l+1}
    ge[3] = gg
    gx = None
    for l in (3, 2, 1, 0):
        ga = cv_back("e%d" % l, ge[l], True)
        gin = cv_back("a%d" % l, ga, True)
        if l > 0:
            ge[l - 1] = ge[l - 1] + pool_backward(gin)
        else:
            gx = gin
    return pack(grads), gx


def mse(y, target):
    d = y - target
    return float(np.mean(d * d)), 2.0 * d / d.size


def adam_step(theta, g, m, v, t, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One bias-corrected Adam step (t counts from 1); returns new
    (theta, m, v)."""
    m = b1 * m + (1.0 - b1) * g
    v = b2 * v + (1.0 - b2) * g * g
    mh = m / (1.0 - b1 ** t)
    vh = v / (1.0 - b2 ** t)
    return theta - lr * mh / (np.sqrt(vh) + eps), m, v
