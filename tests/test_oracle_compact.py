"""Pins of the oracle's compact (Pade) q-derivative of Sec. III B, and of the Hermite
representation propagated with it, against things other than the oracle itself.

The scheme: A f' = B f / h, A = tridiag(1/3, 1, 1/3), (B f)_i = a (f_{i+1} - f_{i-1}) +
b (f_{i+2} - f_{i-2}) with zero values outside the line, a = 7/9, b = 1/36 (the paper prints
a = 7/18; that value is inconsistent, see the first test).  Pins:

* exactness on polynomials of degree <= 6 where the two ends' influence has decayed, and a
  non-zero error for degree 7 (sixth order, not higher);
* the scheme's closed-form Fourier symbol  k' h = (2a sin kh + 2b sin 2kh) / (1 + 2 alpha cos kh)
  at the middle of a long line;
* its leading error is 1/15 of the explicit 7-point stencil's (theta^6/2100 against
  theta^6/140 in the symbol), measured on a Gaussian;
* the ends' influence decays by the factor r = (sqrt(1 - 4 alpha^2) - 1) / (2 alpha) per point
  (the decay rate of A's Green's function), which fixes alpha;
* with the Hermite momenta: the Brownian oscillator's closed-form R1, and Boltzmann
  stationarity at sixth order.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2509_25840_b300 import inputs
import references as ref

ALPHA, A, B = 1.0 / 3.0, 7.0 / 9.0, 1.0 / 36.0


def test_the_printed_constant_is_inconsistent_and_the_reading_is_not():
    """Consistency on f = x at an interior row needs 2a + 4b = 1 + 2 alpha (the same derivative on
    both sides); the printed a = 7/18 gives 8/9 against 5/3, the reading a = 7/9 gives 5/3."""
    assert 2 * (7.0 / 18.0) + 4 * B != pytest.approx(1 + 2 * ALPHA)
    assert 2 * A + 4 * B == pytest.approx(1 + 2 * ALPHA, abs=1e-15)


@pytest.mark.parametrize("deg", range(9))
def test_exact_on_polynomials_up_to_degree_six_away_from_the_ends(deg):
    rng = np.random.default_rng(100 + deg)
    c = rng.normal(size=deg + 1)
    p = np.polynomial.Polynomial(c)
    x = np.linspace(-1.0, 1.0, 160)
    h = x[1] - x[0]
    got = oracle.compact_deriv1d(p(x), h)
    want = p.deriv()(x)
    scale = max(np.abs(want).max(), 1.0)
    err = np.abs(got - want)[70:90].max() / scale        # 70 points from either end
    if deg <= 6:
        assert err < 5e-14, err
    else:
        assert err > 1e-13, err                          # the h^6 f^(7) term shows


@pytest.mark.parametrize("theta", [0.3, 1.0, 2.0, 2.8])
def test_fourier_symbol(theta):
    n, h = 240, 0.05
    x = h * np.arange(n)
    kappa = theta / h
    got = oracle.compact_deriv1d(np.sin(kappa * x), h)
    ksym = (2 * A * math.sin(theta) + 2 * B * math.sin(2 * theta)) / (1 + 2 * ALPHA * math.cos(theta)) / h
    mid = slice(100, 140)
    np.testing.assert_allclose(got[mid], ksym * np.cos(kappa * x[mid]), rtol=0, atol=1e-12 * ksym)


def test_error_constant_is_one_fifteenth_of_the_explicit_stencil():
    ratios = []
    for n in (200, 400):
        x = np.linspace(-9.0, 9.0, n)
        h = x[1] - x[0]
        f = np.exp(-x * x / 2.0)
        exact = -x * f
        ec = np.abs(oracle.compact_deriv1d(f, h) - exact).max()
        ee = np.abs(oracle.deriv1d(f, h) - exact).max()
        ratios.append(ec / ee)
    assert ratios[-1] == pytest.approx(1.0 / 15.0, rel=0.05), ratios


def test_end_effect_decays_at_the_green_function_rate():
    """For f = x^2 (B f / h exact in the interior rows), the error comes from the two boundary
    rows and spreads through A^{-1}: e_j ~ C r^j from the left end."""
    n = 80
    x = np.linspace(0.0, 1.0, n)
    h = x[1] - x[0]
    e = oracle.compact_deriv1d(x * x, h) - 2 * x
    r = (math.sqrt(1 - 4 * ALPHA * ALPHA) - 1) / (2 * ALPHA)
    ratio = e[3:12] / e[2:11]                             # until rounding shows (e_12 ~ 1e-5 e_0)
    np.testing.assert_allclose(ratio, r, rtol=1e-6)


def _harmonic():
    m, w, kT, zeta, gamma, V = 1.3, 0.9, 0.7, 0.4, 1.2, 0.8
    model = inputs.Model(nmodes=1, kT=kT, m=(m,), omega=(w,), zeta=(zeta,), gamma=(gamma,), V_LL=(V,))
    return model, (m, w, kT, zeta, gamma, V)


def _hgrid(n, K, L):
    return inputs.Grid(nq=tuple(n), np=tuple(K), qmin=tuple(-x for x in L), qmax=tuple(L),
                       pmin=tuple(0.0 for _ in n), pmax=tuple(1.0 for _ in n))


def test_hermite_compact_r1_brownian_closed_form():
    """R1 (mu = q) of the harmonic Brownian oscillator with compact q-derivatives: the RK4-discrete
    closed form -[R4(dt A)^k]_01 to sixth order in h_q, with a smaller error than the explicit
    stencil on the same grid."""
    model, (m, w, kT, zeta, gamma, V) = _harmonic()
    dt, nt, stride = 0.01, 11, 20
    want = -ref.g_discrete(ref.brownian_matrix(m, w, zeta, gamma, V), dt, [k * stride for k in range(nt)])
    mu = inputs.Optical(lin=(1.0,))
    sq = math.sqrt(kT / (m * w * w))
    errs, errs_explicit = [], []
    for n in (48, 96):
        for qs, out in ((1, errs), (0, errs_explicit)):
            pb = oracle.Problem(model, _hgrid([n], [4], [8 * sq]), 3, qscheme=qs)
            R = oracle.h_response1(pb, mu, mu, oracle.h_boltzmann(pb), dt, nt, stride)
            out.append(np.abs(R - want).max() / np.abs(want).max())
    assert errs[1] < 1e-7 and math.log2(errs[0] / errs[1]) > 5.5, errs
    assert errs[0] < errs_explicit[0] / 4, (errs, errs_explicit)


@pytest.mark.parametrize("d,ns,K,L", [(1, (40, 80), [8], 7.5), (2, (20, 28), [4, 5], 5.5)])
def test_hermite_compact_boltzmann_stationary_at_sixth_order(d, ns, K, L):
    model = inputs.Model(nmodes=d, kT=0.9, m=(1.2, 0.8), omega=(1.1, 1.3), g3=(0.2, -0.1),
                         g4=(0.05, 0.04), g2=[[0, 0.1], [0, 0]], g_ss2=[[0, 0.12], [0, 0]],
                         zeta=(0.5, 0.3), gamma=(1.0, 1.5), V_LL=(1.0, 0.7), V_SL=(0.3, -0.2))
    res = []
    for n in ns:
        pb = oracle.Problem(model, _hgrid([n] * d, K, [L] * d), 3 if d == 1 else 2, qscheme=1)
        c = oracle.h_boltzmann(pb)
        res.append(np.abs(oracle.h_rhs(pb, c)).max() / np.abs(c).max())
    order = math.log(res[0] / res[1]) / math.log(ns[1] / ns[0])
    assert res[1] < 1e-3 and order > 4.5, (res, order)


def _generator(pb):
    N = pb.M * pb.P
    M = np.zeros((N, N))
    for j in range(N):
        e = np.zeros(N)
        e[j] = 1.0
        M[:, j] = oracle.h_rhs(pb, e.reshape(pb.state_shape)).ravel()
    return M


def _anharmonic_sl():
    return inputs.Model(nmodes=1, kT=1.0, m=(1.0,), omega=(1.0,), g4=(0.05,), zeta=(0.2,),
                        gamma=(1.0,), V_LL=(1.0,), V_SL=(0.3,))


def test_printed_end_rows_give_a_growing_mode_and_the_skew_part_does_not():
    """With the printed (truncated) end rows, A^{-1} B is not antisymmetric; inside the Hermite
    generator (anharmonic mode, square-linear coupling, 32 q points, K = 6, depth 3) that gives an
    eigenvalue with Re > 0.01, i.e. a mode that grows over a spectrum's t ~ 25.  The skew-symmetric
    part (qscheme 2) makes the generator antisymmetric minus the damping, like the explicit
    stencil: M + M^T = -2 diag(sum_s n_s gamma_s)."""
    model = _anharmonic_sl()
    L = inputs.default_grid(model, [32]).qmax[0]
    grid = _hgrid([32], [6], [L])
    M1 = _generator(oracle.Problem(model, grid, 3, qscheme=1))
    assert np.linalg.eigvals(M1).real.max() > 1e-2
    pb2 = oracle.Problem(model, grid, 3, qscheme=2)
    M2 = _generator(pb2)
    damp = np.repeat([n[0] * model.gamma[0] for n in oracle.members(1, 3)], pb2.P)
    np.testing.assert_allclose(M2 + M2.T, -2.0 * np.diag(damp), atol=1e-12)
    assert np.linalg.eigvals(M2).real.max() < 1e-9


def test_three_mode_skew_generator_is_antisymmetric_minus_damping_bilinear():
    """Three modes (the water-like model) with the skew-symmetric compact part on every q axis:
    u.(M v) + v.(M u) = -2 sum u D v for seeded u, v (M + M^T = -2 diag(sum_s n_s gamma_s)
    without forming M); with the printed end rows the same form is off by far more."""
    model = inputs.three_mode_model()
    grid = _hgrid([9, 8, 10], [3, 2, 2], [4.0, 4.0, 4.0])
    pb = oracle.Problem(model, grid, 2, qscheme=2)
    pb1 = oracle.Problem(model, grid, 2, qscheme=1)
    damp = np.repeat([sum(nn[s] * model.gamma[s] for s in range(3)) for nn in oracle.members(3, 2)], pb.P)
    rng = np.random.default_rng(5)
    N = pb.M * pb.P
    for _ in range(2):
        u, v = rng.normal(size=N), rng.normal(size=N)
        errs = []
        for p_ in (pb, pb1):
            Mu = oracle.h_rhs(p_, u.reshape(p_.state_shape)).ravel()
            Mv = oracle.h_rhs(p_, v.reshape(p_.state_shape)).ravel()
            scale = np.abs(u) @ np.abs(Mv) + np.abs(v) @ np.abs(Mu)
            errs.append(abs(u @ Mv + v @ Mu + 2.0 * np.sum(u * damp * v)) / scale)
        assert errs[0] < 1e-13 and errs[1] > 1e-6, errs


def test_skew_part_is_antisymmetric_and_equals_the_compact_derivative_inside():
    n, h = 64, 0.1
    D = np.stack([oracle.compact_skew_deriv1d(np.eye(n)[j], h) for j in range(n)], axis=1)
    np.testing.assert_allclose(D + D.T, 0.0, atol=1e-13)
    x = np.linspace(-1.0, 1.0, 160)
    p = np.polynomial.Polynomial(np.random.default_rng(7).normal(size=7))
    ds = oracle.compact_skew_deriv1d(p(x), x[1] - x[0])
    dc = oracle.compact_deriv1d(p(x), x[1] - x[0])
    scale = np.abs(p.deriv()(x)).max()
    assert np.abs(ds - p.deriv()(x))[70:90].max() < 5e-14 * scale   # sixth order, away from the ends
    assert np.abs(ds - dc)[70:90].max() < 5e-14 * scale


def test_hermite_skew_compact_r1_brownian_closed_form():
    model, (m, w, kT, zeta, gamma, V) = _harmonic()
    dt, nt, stride = 0.01, 11, 20
    want = -ref.g_discrete(ref.brownian_matrix(m, w, zeta, gamma, V), dt, [k * stride for k in range(nt)])
    mu = inputs.Optical(lin=(1.0,))
    sq = math.sqrt(kT / (m * w * w))
    errs = []
    for n in (48, 96):
        pb = oracle.Problem(model, _hgrid([n], [4], [8 * sq]), 3, qscheme=2)
        R = oracle.h_response1(pb, mu, mu, oracle.h_boltzmann(pb), dt, nt, stride)
        errs.append(np.abs(R - want).max() / np.abs(want).max())
    assert errs[1] < 1e-7 and math.log2(errs[0] / errs[1]) > 5.5, errs
