"""Pins of the spectra oracle (Eqs. 1DIR_Raman, 2DThz_Raman, noncorrelation) against closed
forms that do not go through it: the geometric series of damped complex exponentials (exact for
the trapezoid sums), the Fourier integral of a damped sinusoid (second order in dtau), separable
2D products, and the harmonic Brownian oscillator's susceptibility."""
import numpy as np
import pytest

from oracle import spectra
import references as ref


def _geom(z, N, dtau, L, sign, eta):
    """sum_k c_k exp(sign i omega_j t_k) exp(z t_k), trapezoid weights, by the geometric series."""
    j = np.arange(L)
    w = 2.0 * np.pi * (j - L // 2) / (L * dtau)
    r = np.exp((z - eta + sign * 1j * w) * dtau)
    full = (1.0 - r ** N) / (1.0 - r)
    return dtau * (full - 0.5 * (1.0 + r ** (N - 1)))


@pytest.mark.parametrize("sign", [+1, -1])
@pytest.mark.parametrize("N,L,eta", [(2, 8, 0.0), (37, 64, 0.0), (64, 256, 0.3), (100, 100, 0.05)])
def test_transform_equals_geometric_series(sign, N, L, eta):
    dtau = 0.17
    z = -0.4 + 1.3j
    R = np.exp(z * dtau * np.arange(N))
    got = spectra.transform(R, dtau, L, sign, eta)
    want = _geom(z, N, dtau, L, sign, eta)
    np.testing.assert_allclose(got, want, rtol=0, atol=1e-12 * np.abs(want).max())


def test_frequency_grid_is_centred():
    w = spectra.frequencies(8, 0.5)
    assert w[4] == 0.0 and w[5] == pytest.approx(2 * np.pi / 4.0) and w[0] == pytest.approx(-np.pi / 0.5)


def test_spectrum1_converges_to_the_fourier_integral():
    """R1 = exp(-g t) sin(w0 t): integral_0^inf e^{i w t} R1 dt = w0 / ((g - i w)^2 + w0^2).
    The trapezoid rule's dtau^2 term is real here (R1(0) = 0), so Im converges at fourth order."""
    g, w0 = 0.5, 1.7
    errs = []
    for dtau in (0.04, 0.02):
        N = int(80.0 / dtau)
        t = dtau * np.arange(N)
        R1 = np.exp(-g * t) * np.sin(w0 * t)
        L = 2 * N
        w = spectra.frequencies(L, dtau)
        sel = np.abs(w) < 6.0
        want = w * (w0 / ((g - 1j * w) ** 2 + w0 ** 2)).imag
        got = spectra.spectrum1(R1, dtau, L)
        errs.append(np.abs(got - want)[sel].max() / np.abs(want).max())
    assert errs[0] < 1e-5 and errs[0] / errs[1] > 3.5, errs


def test_spectrum2_of_a_separable_response_is_the_product_of_closed_forms():
    """R2[t1][t2] = Re(e^{z1 t1}) Im(e^{z2 t2}): the 2D sum factorises, each factor a geometric
    series; I = Im(F1 F2), both with the minus sign of Eq. 2DThz_Raman."""
    dtau, N1, N2, L1, L2, eta = 0.2, 24, 31, 32, 64, 0.1
    z1, z2 = -0.3 + 0.9j, -0.2 + 2.1j
    t1, t2 = dtau * np.arange(N1), dtau * np.arange(N2)
    R2 = np.outer(np.exp(z1 * t1).real, np.exp(z2 * t2).imag)
    F1 = 0.5 * (_geom(z1, N1, dtau, L1, -1, eta) + _geom(np.conj(z1), N1, dtau, L1, -1, eta))
    F2 = (_geom(z2, N2, dtau, L2, -1, eta) - _geom(np.conj(z2), N2, dtau, L2, -1, eta)) / 2j
    want = np.outer(F1, F2).imag
    got = spectra.spectrum2(R2, dtau, L1, L2, eta)
    np.testing.assert_allclose(got, want, rtol=0, atol=1e-12 * np.abs(want).max())


def test_spectrum3_signs_differ_on_the_two_axes():
    """Eq. noncorrelation: e^{-i w1 t1} on t1 and e^{+i w3 t3} on t3 (separable product)."""
    dtau, N1, N3, L1, L3 = 0.25, 16, 20, 32, 32
    z1, z3 = -0.3 + 1.1j, -0.25 + 0.7j
    R3 = np.outer(np.exp(z1 * dtau * np.arange(N1)).real, np.exp(z3 * dtau * np.arange(N3)).real)
    F1 = 0.5 * (_geom(z1, N1, dtau, L1, -1, 0.0) + _geom(np.conj(z1), N1, dtau, L1, -1, 0.0))
    F3 = 0.5 * (_geom(z3, N3, dtau, L3, +1, 0.0) + _geom(np.conj(z3), N3, dtau, L3, +1, 0.0))
    want = np.outer(F1, F3).imag
    np.testing.assert_allclose(spectra.spectrum3(R3, dtau, L1, L3), want, rtol=0,
                               atol=1e-12 * np.abs(want).max())


def test_brownian_oscillator_spectrum_is_omega_im_chi():
    """R1 of the harmonic Brownian oscillator (Drude bath) = -[e^{At}]_01; with the damping
    window e^{-eta t} its Fourier-Laplace transform is [(A - eta + i w)^{-1}]_01, so
    I(w) = w Im of that (to second order in dtau)."""
    m, omega, zeta, gamma, V = 1.0, 1.0, 0.2, 1.0, 1.0
    A = ref.brownian_matrix(m, omega, zeta, gamma, V)
    dtau, eta = 0.025, 0.2
    N = int(160.0 / dtau)
    t = dtau * np.arange(N)
    R1 = ref.brownian_r1_continuum(m, omega, zeta, gamma, V, t)
    L = 2 * N
    w = spectra.frequencies(L, dtau)
    sel = np.abs(w) < 4.0
    chi = np.array([np.linalg.inv(A - eta * np.eye(3) + 1j * x * np.eye(3))[0, 1] for x in w[sel]])
    want = w[sel] * chi.imag
    got = spectra.spectrum1(R1, dtau, L, eta)[sel]
    assert np.abs(got - want).max() < 1e-4 * np.abs(want).max()
    # the absorption peak sits near the oscillator frequency
    assert abs(abs(w[sel][np.argmax(np.abs(want))]) - omega) < 0.1
