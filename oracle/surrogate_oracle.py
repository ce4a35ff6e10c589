"""FP64 numpy restatement of the learned R2 surrogate -- TEST INFRASTRUCTURE.

The surrogate is this library's own network (the paper has none): 12 standardised model
parameters -> a normalised R2 on a 64 x 64 (t1, t2) grid plus log10 of its scale.  This module
states it from its definition, for checking the CUDA kernels against:

  linear 1..4   z = h W^T + b,  h <- silu(z) = z / (1 + exp(-z))
  scale head    s = h4 w_h + b_h
  decoder       h4 read as an NHWC image [4, 4, 32] (feature f -> row f // 128, column
                f // 32 % 4, channel f % 32); four times: nearest-neighbour upsampling by 2, then
                a 3x3 cross-correlation with zero padding 1,
                    z[y, x, o] = b[o] + sum_{c, ky, kx} u[y + ky - 1, x + kx - 1, c] K[o, c, ky, kx],
                SiLU after all but the last; channels 32 -> 32 -> 16 -> 8 -> 1
  loss          mean over pixels (y - t)^2 + w_s mean over the batch (s - t_s)^2
  AdamW         m <- b1 m + (1 - b1) g,  v <- b2 v + (1 - b2) g^2,
                p <- p - lr (m / (1 - b1^t) / (sqrt(v / (1 - b2^t)) + eps) + wd p)

The convolution is written as a sum over its nine taps on a zero-padded image (no im2col), the
gradients by hand from the chain rule.  ``emulate_bf16=True`` rounds every operand of a
contraction to bfloat16 (round to nearest even) at the points where the CUDA kernels hold BF16
copies, so that the two sides take the same rounding decisions.

Pins (tests/test_surrogate_oracle.py): the convolution against scipy.signal.correlate2d, the
upsampling against a Kronecker product, every gradient block against central finite
differences of the loss, AdamW's bias correction against its constant-gradient closed form,
the bfloat16 rounding against torch's float32 -> bfloat16 conversion.

Only the tests, the smoke check and the benchmark's CPU-baseline leg may import this module.
"""
from __future__ import annotations

import numpy as np

NIN, WID, NPIX = 12, 512, 64 * 64
CONV_IN = (32, 32, 16, 8)
CONV_OUT = (32, 16, 8, 1)
CONV_HIN = (4, 8, 16, 32)


def layer_shapes():
    """(weight shape, bias length) of the nine layers in the host parameter order: linear 1..4,
    scale head, conv 1..4 (a conv weight is [out, in * 9], in-index c * 9 + ky * 3 + kx)."""
    shapes = [((WID, NIN), WID)] + [((WID, WID), WID)] * 3 + [((1, WID), 1)]
    shapes += [((o, c * 9), o) for c, o in zip(CONV_IN, CONV_OUT)]
    return shapes


def param_count() -> int:
    return sum(w[0] * w[1] + b for w, b in layer_shapes())


def unpack(flat):
    """Flat host layout -> list of (W, b) (views)."""
    flat = np.asarray(flat)
    out, q = [], 0
    for (n, k), nb in layer_shapes():
        W = flat[q:q + n * k].reshape(n, k)
        q += n * k
        b = flat[q:q + nb]
        q += nb
        out.append((W, b))
    assert q == flat.size
    return out


def pack(layers) -> np.ndarray:
    return np.concatenate([np.concatenate([np.ravel(W), np.ravel(b)]) for W, b in layers])


def init_params(seed: int) -> np.ndarray:
    """Seeded random parameters for tests (numpy generator; biases small and non-zero so that
    the bias gradients are exercised)."""
    rng = np.random.default_rng(seed)
    layers = []
    for i, ((n, k), nb) in enumerate(layer_shapes()):
        a = np.sqrt((1.5 if i in (4, 8) else 6.0) / k)
        layers.append((rng.uniform(-a, a, (n, k)), rng.uniform(-0.1, 0.1, nb)))
    return pack(layers)


def bf16_round(x):
    """Round to the nearest bfloat16 (ties to even), returned as float64.  Values first round
    to float32 (as the kernels hold them), then to the upper 16 bits of the float32 pattern."""
    f = np.ascontiguousarray(np.asarray(x, dtype=np.float32))
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    r = ((u + 0x7FFF + lsb) & 0xFFFF0000).astype(np.uint32)
    return r.view(np.float32).astype(np.float64)


def silu(z):
    return z / (1.0 + np.exp(-z))


def silu_grad(z):
    s = 1.0 / (1.0 + np.exp(-z))
    return s * (1.0 + z * (1.0 - s))


def upsample2(a):
    """Nearest-neighbour upsampling by 2 of an NHWC image."""
    return a.repeat(2, axis=1).repeat(2, axis=2)


def conv3x3(u, W, b):
    """3x3 cross-correlation with zero padding 1 of NHWC u [B, H, H, C] with W [O, C * 9]."""
    B, H, _, C = u.shape
    K = W.reshape(W.shape[0], C, 3, 3)
    up = np.zeros((B, H + 2, H + 2, C))
    up[:, 1:-1, 1:-1, :] = u
    z = np.zeros((B, H, H, W.shape[0])) + b
    for ky in range(3):
        for kx in range(3):
            z += np.einsum("bhwc,oc->bhwo", up[:, ky:ky + H, kx:kx + H, :], K[:, :, ky, kx])
    return z


def conv3x3_backward(u, W, dz):
    """Gradients of conv3x3 with respect to u and W for the output gradient dz."""
    B, H, _, C = u.shape
    K = W.reshape(W.shape[0], C, 3, 3)
    up = np.zeros((B, H + 2, H + 2, C))
    up[:, 1:-1, 1:-1, :] = u
    dup = np.zeros_like(up)
    dK = np.zeros_like(K)
    for ky in range(3):
        for kx in range(3):
            dK[:, :, ky, kx] = np.einsum("bhwo,bhwc->oc", dz, up[:, ky:ky + H, kx:kx + H, :])
            dup[:, ky:ky + H, kx:kx + H, :] += np.einsum("bhwo,oc->bhwc", dz, K[:, :, ky, kx])
    return dup[:, 1:-1, 1:-1, :], dK.reshape(W.shape)


def upsample2_backward(du):
    """Adjoint of upsample2: each input pixel collects its 2 x 2 block."""
    B, H, _, C = du.shape
    return du.reshape(B, H // 2, 2, H // 2, 2, C).sum(axis=(2, 4))


def forward(flat, X, emulate_bf16: bool = False):
    """Image [B, 64, 64], scale [B] and the cache for backward."""
    q = bf16_round if emulate_bf16 else (lambda a: np.asarray(a, dtype=np.float64))
    layers = unpack(np.asarray(flat, dtype=np.float64))
    h = np.asarray(X, dtype=np.float64)
    cache = {"h": [], "z": [], "u": [], "zc": []}
    for l in range(4):
        W, b = layers[l]
        cache["h"].append(q(h))
        z = q(h) @ q(W).T + b
        cache["z"].append(z)
        h = silu(z)
    h4 = q(h)                       # the kernels keep silu outputs in BF16
    cache["h"].append(h4)
    Wh, bh = layers[4]
    s = (h4 @ q(Wh).T + bh)[:, 0]
    a = h4.reshape(-1, 4, 4, 32)
    for c in range(4):
        W, b = layers[5 + c]
        u = q(upsample2(a))
        cache["u"].append(u)
        z = conv3x3(u, q(W), b)
        cache["zc"].append(z)
        if c < 3:
            a = silu(z)
    return z[..., 0], s, cache


def loss(Y, S, T, TS, w_scale: float = 1.0) -> float:
    T = np.asarray(T, dtype=np.float64).reshape(Y.shape)
    return float(np.mean((Y - T) ** 2) + w_scale * np.mean((S - np.asarray(TS, dtype=np.float64)) ** 2))


def backward(flat, X, T, TS, w_scale: float = 1.0, emulate_bf16: bool = False):
    """(loss, gradient in the flat host layout).  With emulate_bf16 the output gradients of
    every layer are rounded to BF16 before the contractions that take them, as in the kernels;
    the bias gradients and the scale head's term of dh4 use the unrounded values."""
    q = bf16_round if emulate_bf16 else (lambda a: np.asarray(a, dtype=np.float64))
    layers = unpack(np.asarray(flat, dtype=np.float64))
    Y, S, cache = forward(flat, X, emulate_bf16)
    B = Y.shape[0]
    T = np.asarray(T, dtype=np.float64).reshape(Y.shape)
    TS = np.asarray(TS, dtype=np.float64)
    L = loss(Y, S, T, TS, w_scale)
    grads = [None] * 9
    dz = (2.0 / Y.size * (Y - T))[..., None]             # [B, 64, 64, 1]
    dS = 2.0 * w_scale / B * (S - TS)                    # [B]
    for c in range(3, -1, -1):
        W, b = layers[5 + c]
        du, dW = conv3x3_backward(cache["u"][c], q(W), q(dz))
        grads[5 + c] = (dW, dz.sum(axis=(0, 1, 2)))
        da = upsample2_backward(du)
        if c > 0:
            dz = da * silu_grad(cache["zc"][c - 1])
    dh = da.reshape(B, WID)
    Wh, bh = layers[4]
    grads[4] = (q(dS)[None, :] @ cache["h"][4], np.array([dS.sum()]))
    dh = dh + dS[:, None] * Wh                           # FP32 master weights in the kernels
    for l in range(3, -1, -1):
        W, b = layers[l]
        dz = dh * silu_grad(cache["z"][l])
        grads[l] = (q(dz).T @ cache["h"][l], dz.sum(axis=0))
        dh = q(dz) @ q(W)
    return L, pack(grads)


def adamw(p, g, m, v, t: int, lr: float, wd: float = 0.0, b1: float = 0.9, b2: float = 0.999,
          eps: float = 1e-8):
    """One AdamW step at step number t (1-based); returns (p, m, v)."""
    m = b1 * m + (1.0 - b1) * g
    v = b2 * v + (1.0 - b2) * g * g
    mh = m / (1.0 - b1 ** t)
    vh = v / (1.0 - b2 ** t)
    return p - lr * (mh / (np.sqrt(vh) + eps) + wd * p), m, v
