"""Pins of the surrogate network's FP64 oracle against things other than itself: a library
convolution, a Kronecker product, finite differences of its own loss, the closed form of AdamW
under a constant gradient, and torch's bfloat16 conversion."""
import numpy as np
import pytest
from scipy import signal

from oracle import surrogate_oracle as so


def test_param_count_matches_layer_list():
    # 12*512+512 + 3*(512*512+512) + 512+1 + 32*288+32 + 16*288+16 + 8*144+8 + 1*72+1
    assert so.param_count() == 810242


def test_conv3x3_is_scipy_correlate2d_same():
    rng = np.random.default_rng(3)
    u = rng.standard_normal((2, 6, 6, 3))
    W = rng.standard_normal((4, 27))
    b = rng.standard_normal(4)
    z = so.conv3x3(u, W, b)
    K = W.reshape(4, 3, 3, 3)
    for bi in range(2):
        for o in range(4):
            want = b[o] + sum(signal.correlate2d(u[bi, :, :, c], K[o, c], mode="same")
                              for c in range(3))
            np.testing.assert_allclose(z[bi, :, :, o], want, rtol=0, atol=1e-12)


def test_upsample_is_kronecker_with_ones():
    rng = np.random.default_rng(4)
    a = rng.standard_normal((2, 3, 3, 2))
    u = so.upsample2(a)
    for bi in range(2):
        for c in range(2):
            np.testing.assert_array_equal(u[bi, :, :, c], np.kron(a[bi, :, :, c], np.ones((2, 2))))


def _batch(seed, B=2):
    rng = np.random.default_rng(seed)
    X = rng.uniform(-1, 1, (B, so.NIN))
    T = rng.uniform(-1, 1, (B, 64, 64))
    TS = rng.uniform(-2, 2, B)
    return X, T, TS


def test_gradients_match_central_differences():
    """Every weight and bias block, sampled: the hand-written chain rule against (L(p + e) -
    L(p - e)) / 2e in FP64 (a dropped term, a transposed operand or a wrong tap index in any layer
    fails here)."""
    p = so.init_params(11)
    X, T, TS = _batch(5)
    w = 0.7
    L, g = so.backward(p, X, T, TS, w_scale=w)
    assert np.isclose(L, so.loss(*so.forward(p, X)[:2], T, TS, w))
    rng = np.random.default_rng(9)
    q = 0
    eps = 1e-5
    for (n, k), nb in so.layer_shapes():
        idx = list(q + rng.choice(n * k, size=min(6, n * k), replace=False))
        idx += list(q + n * k + rng.choice(nb, size=min(2, nb), replace=False))
        block = g[q:q + n * k + nb]
        scale = np.abs(block).max()
        for i in idx:
            pp, pm = p.copy(), p.copy()
            pp[i] += eps
            pm[i] -= eps
            Lp = so.loss(*so.forward(pp, X)[:2], T, TS, w)
            Lm = so.loss(*so.forward(pm, X)[:2], T, TS, w)
            fd = (Lp - Lm) / (2 * eps)
            assert abs(fd - g[i]) <= 1e-6 * scale + 1e-9, (i, fd, g[i])
        q += n * k + nb


def test_adamw_constant_gradient_closed_form():
    """Under a constant gradient the bias-corrected moments are exactly g and g^2, so each step
    moves by lr g / (|g| + eps); decoupled decay multiplies by (1 - lr wd) first."""
    rng = np.random.default_rng(2)
    p0 = rng.standard_normal(50)
    g = rng.standard_normal(50)
    lr, wd, steps = 1e-2, 0.1, 10
    p, m, v = p0.copy(), np.zeros(50), np.zeros(50)
    for t in range(1, steps + 1):
        p, m, v = so.adamw(p, g, m, v, t, lr, wd)
    u = g / (np.abs(g) + 1e-8)
    r = 1 - lr * wd
    want = r ** steps * p0 - lr * u * sum(r ** j for j in range(steps))
    np.testing.assert_allclose(p, want, rtol=1e-12, atol=1e-13)


def test_bf16_rounding_matches_torch():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(1)
    x = np.concatenate([rng.standard_normal(4000) * 10.0 ** rng.integers(-8, 8, 4000),
                        [0.0, -0.0, 1.0, -3.5, 1e-40]])
    # exact ties between two bfloat16 values, both parities of the kept bit
    ties = np.array([0x3F808000, 0x3F818000, 0xBF808000, 0x40490000 | 0x8000], dtype=np.uint32)
    x = np.concatenate([x, ties.view(np.float32).astype(np.float64)])
    want = torch.tensor(x, dtype=torch.float32).to(torch.bfloat16).to(torch.float64).numpy()
    np.testing.assert_array_equal(so.bf16_round(x), want)
