"""FP64 CPU oracle for the spectra of sampled response functions -- TEST INFRASTRUCTURE.

Only the tests, the smoke check and the benchmark's CPU legs may import this module; the CUDA
library never does.  It restates Eqs. 1DIR_Raman, 2DThz_Raman and noncorrelation (Sec. II C) as
plain direct sums, one output frequency at a time, in FP64.

Discretisation (the paper gives the continuous integrals only; the readings are listed in the
design notes): a response sampled at t_k = k dtau, k = 0..N-1, stands for the integral over
[0, (N-1) dtau] by the trapezoid rule, weights c_k = dtau (1/2 at k = 0 and k = N-1), times an
optional damping exp(-eta t_k) (eta = 0: none), with R = 0 beyond the last sample.  The
frequency grid of a transform of length L >= N is centred,
    omega_j = 2 pi (j - L/2) / (L dtau),  j = 0..L-1   (omega = 0 at j = L/2),
and each sign of the exponent is the one its equation prints:
    I(omega_1)           = omega_1 Im sum_k c_k e^{+i omega_1 t_k} R1(t_k)            (1DIR_Raman)
    I(omega_1, omega_2)  = Im sum_{a,b} c_a c_b e^{-i omega_1 t_a - i omega_2 t_b} R2(t_b, t_a)
                                                                                       (2DThz_Raman)
    I(omega_3, t2, omega_1) = Im sum_{a,c} c_a c_c e^{-i omega_1 t_a + i omega_3 t_c} R3(t_c, t2, t_a)
                                                                                  (noncorrelation)
R2 arrays are indexed [t1][t2] and R3 arrays [t1][t3] (fixed t2), as the library returns them.

Parity status: pinned by the geometric-series closed form of damped complex exponentials
(exact for the discrete sums, any N, L, eta), by the continuum Fourier integral of a damped
sinusoid (second order in dtau), and by separable products (2D = product of 1D transforms);
tests/test_oracle_spectra.py.
"""
from __future__ import annotations

import numpy as np


def frequencies(L: int, dtau: float) -> np.ndarray:
    """The centred grid omega_j = 2 pi (j - L/2) / (L dtau)."""
    return 2.0 * np.pi * (np.arange(L) - L // 2) / (L * dtau)


def weights(N: int, dtau: float, eta: float = 0.0) -> np.ndarray:
    """Trapezoid weights on [0, (N-1) dtau] times exp(-eta t_k)."""
    if N < 2:
        raise ValueError("at least two samples")
    c = np.full(N, dtau)
    c[0] = c[-1] = 0.5 * dtau
    return c * np.exp(-eta * dtau * np.arange(N))


def transform(R: np.ndarray, dtau: float, L: int, sign: int, eta: float = 0.0) -> np.ndarray:
    """F(omega_j) = sum_k c_k exp(sign i omega_j t_k) R_k for a 1D array (complex result).
    The phase omega_j t_k = 2 pi (j - L/2) k / L is reduced modulo 2 pi exactly in integers."""
    R = np.asarray(R)
    N = R.shape[0]
    c = weights(N, dtau, eta)
    out = np.zeros(L, dtype=np.complex128)
    k = np.arange(N, dtype=np.int64)
    for j in range(L):
        m = ((j - L // 2) * k) % L
        out[j] = np.sum(c * R * np.exp(sign * 2j * np.pi * m / L))
    return out


def spectrum1(R1, dtau: float, L: int, eta: float = 0.0) -> np.ndarray:
    """I(omega_1) of Eq. 1DIR_Raman on the centred grid of length L."""
    F = transform(np.asarray(R1, dtype=np.float64), dtau, L, +1, eta)
    return frequencies(L, dtau) * F.imag


def spectrum2(R2, dtau: float, L1: int, L2: int, eta: float = 0.0) -> np.ndarray:
    """I(omega_1, omega_2) of Eq. 2DThz_Raman, [L1][L2], from R2[t1][t2]: the t2 sum first,
    then the t1 sum (the order does not matter in exact arithmetic)."""
    R2 = np.asarray(R2, dtype=np.float64)
    N1 = R2.shape[0]
    inner = np.stack([transform(R2[a], dtau, L2, -1, eta) for a in range(N1)])    # [N1][L2]
    out = np.zeros((L1, L2))
    for b in range(L2):
        out[:, b] = transform(inner[:, b], dtau, L1, -1, eta).imag
    return out


def spectrum3(R3, dtau: float, L1: int, L3: int, eta: float = 0.0) -> np.ndarray:
    """I(omega_3, t2, omega_1) of Eq. noncorrelation at one t2, [L1][L3], from R3[t1][t3]."""
    R3 = np.asarray(R3, dtype=np.float64)
    N1 = R3.shape[0]
    inner = np.stack([transform(R3[a], dtau, L3, +1, eta) for a in range(N1)])    # [N1][L3]
    out = np.zeros((L1, L3))
    for b in range(L3):
        out[:, b] = transform(inner[:, b], dtau, L1, -1, eta).imag
    return out
