"""FP64 oracle of the learned warm start: a 3-level encoder/decoder CNN that
maps (div u*/dt, 1/rho) to a pressure guess, with its backward pass, loss and
Adam update.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).  Plain numpy in float64:
every layer is its definition written out (a 3x3 convolution is nine shifted
products summed), so it can be checked by eye and by finite differences.

Layout: activations NHWC, arrays of shape (B, H, W, C); conv weights
(Cout, 3, 3, Cin) (tap (dy, dx) multiplies x[i + dy - 1, j + dx - 1]); bias
(Cout,).  Zero padding, stride 1.

Network (channel counts c1 = 16, c2 = 32):
  x (2) -> conv 2->c1, ReLU -> conv c1->c1, ReLU = s1           (N)
  pool2 -> conv c1->c2, ReLU -> conv c2->c2, ReLU = s2           (N/2)
  pool2 -> conv c2->c2, ReLU -> conv c2->c2, ReLU = t3           (N/4)
  up2(t3) ++ s2 -> conv 2c2->c2, ReLU = t4                        (N/2)
  up2(t4) ++ s1 -> conv (c2+c1)->c1, ReLU -> conv c1->1 = y      (N)
pool2 = mean of 2x2 blocks; up2 = nearest (each value to a 2x2 block);
++ = channel concatenation, upsampled tensor first.
"""
from __future__ import annotations

import numpy as np

LAYERS = [  # (name, cin, cout, relu)
    ("c1a", 2, 16, True), ("c1b", 16, 16, True),
    ("c2a", 16, 32, True), ("c2b", 32, 32, True),
    ("c3a", 32, 32, True), ("c3b", 32, 32, True),
    ("c4", 64, 32, True),
    ("c5", 48, 16, True), ("c6", 16, 1, False),
]


def layer_shapes(c1=16, c2=32):
    m = {16: c1, 32: c2, 64: 2 * c2, 48: c2 + c1, 2: 2, 1: 1}
    return [(n, m[ci], m[co], r) for n, ci, co, r in LAYERS]


def init_params(seed=0, c1=16, c2=32):
    """He-normal weights, zero biases (float64)."""
    rng = np.random.default_rng(seed)
    P = {}
    for name, ci, co, _ in layer_shapes(c1, c2):
        P[name + ".w"] = rng.standard_normal((co, 3, 3, ci)) * np.sqrt(2.0 / (9 * ci))
        P[name + ".b"] = np.zeros(co)
    return P


def conv3x3(x, w, b):
    B, H, W, _ = x.shape
    xp = np.pad(x, ((0, 0), (1, 1), (1, 1), (0, 0)))
    y = np.broadcast_to(b, (B, H, W, w.shape[0])).copy()
    for dy in range(3):
        for dx in range(3):
            y += np.einsum("bhwc,oc->bhwo", xp[:, dy:dy + H, dx:dx + W, :], w[:, dy, dx, :])
    return y


def conv3x3_bwd(x, w, gy):
    """Gradients of sum(gy * conv3x3(x, w, b)) w.r.t. x, w, b."""
    B, H, W, _ = x.shape
    xp = np.pad(x, ((0, 0), (1, 1), (1, 1), (0, 0)))
    gxp = np.zeros_like(xp)
    gw = np.zeros_like(w)
    for dy in range(3):
        for dx in range(3):
            gw[:, dy, dx, :] = np.einsum("bhwo,bhwc->oc", gy, xp[:, dy:dy + H, dx:dx + W, :])
            gxp[:, dy:dy + H, dx:dx + W, :] += np.einsum("bhwo,oc->bhwc", gy, w[:, dy, dx, :])
    return gxp[:, 1:-1, 1:-1, :], gw, gy.sum(axis=(0, 1, 2))


def pool2(x):
    B, H, W, C = x.shape
    return x.reshape(B, H // 2, 2, W // 2, 2, C).mean(axis=(2, 4))


def pool2_bwd(g):
    return np.repeat(np.repeat(g, 2, axis=1), 2, axis=2) / 4.0


def up2(x):
    return np.repeat(np.repeat(x, 2, axis=1), 2, axis=2)


def up2_bwd(g):
    B, H, W, C = g.shape
    return g.reshape(B, H // 2, 2, W // 2, 2, C).sum(axis=(2, 4))


def bf16_round(a):
    """The nearest bfloat16 value (8-bit significand, round to nearest, ties
    to even) of each element, after rounding to binary32 (the storage of a
    binary32 value as bfloat16); returned as float64."""
    f = np.ascontiguousarray(a, np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def _ident(a):
    return a


def forward(P, x, keep=False, bf16=False):
    """x (B, N, N, 2) -> y (B, N, N, 1); with keep=True also the cache.

    bf16=True evaluates the network as BF16 activations with wider
    accumulation (the precision the learned part is specified in): every
    stored activation -- each hidden layer's output after bias and ReLU, and
    each pooled tensor -- is rounded to BF16 (bf16_round); the sums inside a
    convolution stay FP64 and the last layer's output is not rounded."""
    cache = {}
    r = bf16_round if bf16 else _ident

    def conv(name, inp, relu):
        z = conv3x3(inp, P[name + ".w"], P[name + ".b"])
        out = r(np.maximum(z, 0.0)) if relu else z
        cache[name] = (inp, z)
        return out

    a = conv("c1a", x, True)
    s1 = conv("c1b", a, True)
    a = conv("c2a", r(pool2(s1)), True)
    s2 = conv("c2b", a, True)
    a = conv("c3a", r(pool2(s2)), True)
    t3 = conv("c3b", a, True)
    t4 = conv("c4", np.concatenate([up2(t3), s2], axis=3), True)
    a = conv("c5", np.concatenate([up2(t4), s1], axis=3), True)
    y = conv("c6", a, False)
    return (y, cache) if keep else y


def backward(P, cache, gy, bf16=False):
    """Gradients of sum(gy * forward(P, x)) w.r.t. every parameter and x.

    bf16=True: the BF16 counterpart of forward(bf16=True) -- every stored
    gradient tensor (gy itself, each layer's input gradient, the folded
    up-sampling gradients and the skip sums) is rounded to BF16; parameter
    gradients stay FP64 sums."""
    G = {}
    r = bf16_round if bf16 else _ident

    def conv_b(name, g, relu):
        inp, z = cache[name]
        if relu:
            g = g * (z > 0)
        gx, gw, gb = conv3x3_bwd(inp, P[name + ".w"], g)
        G[name + ".w"], G[name + ".b"] = gw, gb
        return r(gx)

    c2 = P["c4.w"].shape[0]
    g = conv_b("c6", r(gy), False)
    g = conv_b("c5", g, True)
    g_up4, g_s1 = g[..., :c2], g[..., c2:]
    g = conv_b("c4", r(up2_bwd(g_up4)), True)
    g_up3, g_s2 = g[..., :c2], g[..., c2:]
    g = conv_b("c3b", r(up2_bwd(g_up3)), True)
    g = conv_b("c3a", g, True)
    g = conv_b("c2b", r(pool2_bwd(g) + g_s2), True)
    g = conv_b("c2a", g, True)
    g = conv_b("c1b", r(pool2_bwd(g) + g_s1), True)
    gx = conv_b("c1a", g, True)
    return G, gx


def loss(y, t):
    """Mean-removed squared error per sample (the pressure is defined up to a
    constant), averaged over the batch: mean over b of mean over pixels of
    ((y - mean y) - (t - mean t))^2.  Returns (L, dL/dy)."""
    B = y.shape[0]
    n = y[0].size
    d = (y - y.mean(axis=(1, 2, 3), keepdims=True)) - (t - t.mean(axis=(1, 2, 3), keepdims=True))
    L = float((d * d).sum() / (B * n))
    g = 2.0 * d / (B * n)
    g = g - g.mean(axis=(1, 2, 3), keepdims=True)
    return L, g


def adam(P, G, M, V, step, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam step (Kingma & Ba) with bias correction; updates P, M, V."""
    for k in P:
        M[k] = b1 * M[k] + (1 - b1) * G[k]
        V[k] = b2 * V[k] + (1 - b2) * G[k] * G[k]
        mh = M[k] / (1 - b1 ** step)
        vh = V[k] / (1 - b2 ** step)
        P[k] = P[k] - lr * mh / (np.sqrt(vh) + eps)


def features(b, beta_cell):
    """Network input from a right-hand side b and cell-centred 1/rho: channel
    0 = b / s with s = rms(b - mean b), channel 1 = beta / max(beta).
    Returns (x (1, N, N, 2), s)."""
    b0 = b - b.mean()
    s = float(np.sqrt((b0 * b0).mean()))
    s = s if s > 0 else 1.0
    return np.stack([b0 / s, beta_cell / beta_cell.max()], axis=-1)[None], s
