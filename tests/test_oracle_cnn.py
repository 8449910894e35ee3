"""Pins of the CNN oracle (oracle/cnn.py): convolution against scipy's
correlation, adjoint pairs, the whole network's gradients against central
finite differences, loss invariances and the first Adam step."""
import numpy as np
import pytest

from oracle import cnn


def test_conv3x3_matches_library_correlation():
    sig = pytest.importorskip("scipy.signal")
    rng = np.random.default_rng(0)
    x = rng.standard_normal((2, 7, 9, 3))
    w = rng.standard_normal((4, 3, 3, 3))
    b = rng.standard_normal(4)
    y = cnn.conv3x3(x, w, b)
    for bb in range(2):
        for o in range(4):
            ref = b[o] + sum(sig.correlate2d(x[bb, :, :, c], w[o, :, :, c], mode="same",
                                             boundary="fill") for c in range(3))
            assert np.abs(y[bb, :, :, o] - ref).max() < 1e-12


def test_adjoint_pairs():
    rng = np.random.default_rng(1)
    x = rng.standard_normal((2, 8, 6, 3))
    g = rng.standard_normal((2, 4, 3, 3))
    assert abs((cnn.pool2(x) * g).sum() - (x * cnn.pool2_bwd(g)).sum()) < 1e-12
    xs = rng.standard_normal((2, 4, 3, 3))
    gs = rng.standard_normal((2, 8, 6, 3))
    assert abs((cnn.up2(xs) * gs).sum() - (xs * cnn.up2_bwd(gs)).sum()) < 1e-12
    w = rng.standard_normal((5, 3, 3, 3))
    gy = rng.standard_normal((2, 8, 6, 5))
    gx, gw, gb = cnn.conv3x3_bwd(x, w, gy)
    # linearity in x: <conv(x), gy> - <conv(0), gy> = <x, gx>
    lhs = (cnn.conv3x3(x, w, np.zeros(5)) * gy).sum()
    assert abs(lhs - (x * gx).sum()) < 1e-10 * abs(lhs)
    assert abs(lhs - (w * gw).sum()) < 1e-10 * abs(lhs)


def _tiny():
    P = cnn.init_params(seed=3, c1=4, c2=6)
    for q, k in enumerate(sorted(P)):
        if k.endswith(".b"):  # nonzero biases, seeded by position (str hashes vary per process)
            P[k] = np.random.default_rng(100 + q).standard_normal(P[k].shape) * 0.1
    rng = np.random.default_rng(4)
    x = rng.standard_normal((2, 8, 8, 2))
    t = rng.standard_normal((2, 8, 8, 1))
    return P, x, t


def test_network_gradients_match_finite_differences():
    P, x, t = _tiny()
    y, cache = cnn.forward(P, x, keep=True)
    L, gy = cnn.loss(y, t)
    G, gx = cnn.backward(P, cache, gy)
    rng = np.random.default_rng(5)
    eps = 1e-6

    def Lof(P_, x_):
        return cnn.loss(cnn.forward(P_, x_), t)[0]

    for k in P:
        for _ in range(3):
            idx = tuple(rng.integers(0, s) for s in P[k].shape)
            Pp = {q: v.copy() for q, v in P.items()}
            Pm = {q: v.copy() for q, v in P.items()}
            Pp[k][idx] += eps
            Pm[k][idx] -= eps
            fd = (Lof(Pp, x) - Lof(Pm, x)) / (2 * eps)
            assert abs(fd - G[k][idx]) <= 1e-7 * max(1.0, abs(fd)) + 1e-9, (k, idx, fd, G[k][idx])
    for _ in range(5):
        idx = tuple(rng.integers(0, s) for s in x.shape)
        xp, xm = x.copy(), x.copy()
        xp[idx] += eps
        xm[idx] -= eps
        fd = (Lof(P, xp) - Lof(P, xm)) / (2 * eps)
        assert abs(fd - gx[idx]) <= 1e-7 * max(1.0, abs(fd)) + 1e-9


def test_loss_ignores_constant_shifts():
    rng = np.random.default_rng(6)
    y, t = rng.standard_normal((3, 4, 4, 1)), rng.standard_normal((3, 4, 4, 1))
    L1, g1 = cnn.loss(y, t)
    L2, g2 = cnn.loss(y + np.array([1.0, -2.0, 3.0])[:, None, None, None], t - 5.0)
    assert abs(L1 - L2) < 1e-12 and np.abs(g1 - g2).max() < 1e-14
    assert np.abs(g1.sum(axis=(1, 2, 3))).max() < 1e-14
    assert cnn.loss(t + 7.0, t)[0] < 1e-24


def test_first_adam_step_is_a_sign_step():
    P = {"a": np.array([1.0, -2.0, 0.5])}
    G = {"a": np.array([0.3, -4.0, 1e-3])}
    M = {"a": np.zeros(3)}
    V = {"a": np.zeros(3)}
    cnn.adam(P, G, M, V, 1, lr=0.1, eps=0.0)
    assert np.allclose(P["a"], [0.9, -1.9, 0.4], rtol=0, atol=1e-14)


def test_bf16_rounding_matches_the_format():
    # bfloat16 is binary32 with the significand cut to 8 bits, rounded to
    # nearest with ties to even: the library's conversion is the reference
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(3)
    a = np.concatenate([rng.standard_normal(20000) * 10.0 ** rng.uniform(-30, 30, 20000),
                        [1.0 + 2 ** -8, 1.0 + 3 * 2 ** -8, -(1.0 + 2 ** -8), 0.0, -0.0]])
    ref = torch.from_numpy(a.astype(np.float32)).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(cnn.bf16_round(a), ref)


def test_bf16_replay_stores_bf16_and_stays_near_the_fp64_network():
    # the BF16 replay's stored activations are BF16 values, its output is
    # within BF16's relative precision of the FP64 network, and its gradients
    # within BF16-storage error of the FP64 gradients (15 % in norm: the
    # relative error grows towards the input layers)
    P = cnn.init_params(seed=4)
    x = np.random.default_rng(5).standard_normal((2, 16, 16, 2))
    x = cnn.bf16_round(x)
    y64, c64 = cnn.forward(P, x, keep=True)
    y16, c16 = cnn.forward(P, x, keep=True, bf16=True)
    for name in ("c1b", "c2a", "c4", "c5", "c6"):
        inp = c16[name][0]
        assert np.array_equal(cnn.bf16_round(inp), inp), name
    assert np.linalg.norm(y16 - y64) / np.linalg.norm(y64) < 2e-2
    t = np.random.default_rng(6).standard_normal(y64.shape)
    _, g64 = cnn.loss(y64, t)
    _, g16 = cnn.loss(y16, t)
    G64, _ = cnn.backward(P, c64, g64)
    G16, _ = cnn.backward(P, c16, g16, bf16=True)
    for k in G64:
        if k == "c6.b":
            continue
        assert np.linalg.norm(G16[k] - G64[k]) <= 0.15 * np.linalg.norm(G64[k]), k
