"""Pins of the oracle's Hermite-function momentum representation (Sec. III A, Appendix A,
Eq. HEOM2FP-H) against things other than itself: the antisymmetry of the ladder generator (the
dense matrix extracted column by column), Boltzmann stationarity at sixth order in h_q, the
Brownian oscillator's closed-form R1, the exact moment closure for R2, and the grid
representation's R2 on the same anharmonic model."""
import math

import numpy as np
import pytest

import oracle
from paper_2509_25840_b300 import inputs
import references as ref


def _hgrid(n, K, L):
    n = list(n)
    K = list(K)
    L = list(L)
    return inputs.Grid(nq=tuple(n), np=tuple(K), qmin=tuple(-x for x in L), qmax=tuple(L),
                       pmin=tuple(0.0 for _ in n), pmax=tuple(1.0 for _ in n))


def _anharmonic(d):
    return inputs.Model(nmodes=d, kT=0.9, m=(1.2, 0.8), omega=(1.1, 1.3), g3=(0.2, -0.1),
                        g4=(0.05, 0.04), g2=[[0, 0.1], [0, 0]], g_ss2=[[0, 0.12], [0, 0]],
                        zeta=(0.5, 0.3), gamma=(1.0, 1.5), V_LL=(1.0, 0.7), V_SL=(0.3, -0.2))


@pytest.mark.parametrize("d,n,K,depth", [(1, [9], [5], 2), (2, [7, 8], [3, 4], 2)])
def test_ladder_generator_is_antisymmetric_minus_damping(d, n, K, depth):
    """D+ and -D- are transposes of each other (d/dq antisymmetric), and the two hierarchy links
    are negative transposes: M + M^T = -2 diag(sum_s n_s gamma_s)."""
    model = _anharmonic(d)
    pb = oracle.Problem(model, _hgrid(n, K, [4.0] * d), depth)
    N = pb.M * pb.P
    M = np.zeros((N, N))
    for j in range(N):
        e = np.zeros(N)
        e[j] = 1.0
        M[:, j] = oracle.h_rhs(pb, e.reshape(pb.state_shape)).ravel()
    damp = np.repeat([sum(nn[s] * model.gamma[s] for s in range(d)) for nn in oracle.members(d, depth)], pb.P)
    np.testing.assert_allclose(M + M.T, -2.0 * np.diag(damp), atol=1e-13)
    assert np.abs(M).max() > 1.0          # the operator is not trivially zero


def test_three_mode_generator_is_antisymmetric_minus_damping_bilinear():
    """Three modes (the water-like model: pair couplings, square-linear bath coupling), without
    forming the matrix: for seeded u, v the bilinear form u.(M v) + v.(M u) equals
    -2 sum_i u_i D_i v_i, D = sum_s n_s gamma_s per member, i.e. M + M^T = -2 D (a wrong sign,
    index or factor on one of the q_3 / k_3 terms or links breaks the symmetry)."""
    model = inputs.three_mode_model()
    pb = oracle.Problem(model, _hgrid([7, 8, 7], [3, 2, 4], [4.0, 4.0, 4.0]), 2)
    damp = np.repeat([sum(nn[s] * model.gamma[s] for s in range(3)) for nn in oracle.members(3, 2)], pb.P)
    rng = np.random.default_rng(11)
    N = pb.M * pb.P
    for _ in range(3):
        u, v = rng.normal(size=N), rng.normal(size=N)
        Mu = oracle.h_rhs(pb, u.reshape(pb.state_shape)).ravel()
        Mv = oracle.h_rhs(pb, v.reshape(pb.state_shape)).ravel()
        lhs = u @ Mv + v @ Mu
        rhs = -2.0 * np.sum(u * damp * v)
        scale = np.abs(u) @ np.abs(Mv) + np.abs(v) @ np.abs(Mu)
        assert abs(lhs - rhs) <= 1e-13 * scale, (lhs, rhs, scale)
        assert np.abs(Mu).max() > 1.0        # the operator is not trivially zero


def test_three_mode_boltzmann_is_stationary_at_sixth_order():
    """The water-like model on q-domains where exp(-U/2kT) < 1e-7 at the ends: the residual of the
    equilibrium coefficients falls at about sixth order in h_q."""
    model = inputs.three_mode_model()
    res = []
    ns = (24, 32)
    for n in ns:
        g = inputs.default_grid(model, [n], cut=32.0)
        pb = oracle.Problem(model, _hgrid([n] * 3, [2, 2, 2], list(g.qmax)), 1)
        c = oracle.h_boltzmann(pb)
        res.append(np.abs(oracle.h_rhs(pb, c)).max() / np.abs(c).max())
    order = math.log(res[0] / res[1]) / math.log(ns[1] / ns[0])
    assert res[1] < 1e-3 and order > 4.5, (res, order)


@pytest.mark.parametrize("d,ns,K,L", [(1, (40, 80), [8], 7.5), (2, (24, 32), [4, 5], 5.5)])
def test_boltzmann_is_stationary_at_sixth_order(d, ns, K, L):
    """(The q-domain reaches exp(-U/2kT) < 1e-7 at its ends, below the stencil error.)"""
    model = _anharmonic(d)
    res = []
    for n in ns:
        pb = oracle.Problem(model, _hgrid([n] * d, K, [L] * d), 3 if d == 1 else 2)
        c = oracle.h_boltzmann(pb)
        res.append(np.abs(oracle.h_rhs(pb, c)).max() / np.abs(c).max())
    order = math.log(res[0] / res[1]) / math.log(ns[1] / ns[0])
    assert res[1] < 1e-3 and order > 4.5, (res, order)


def test_boltzmann_moments():
    """<q^2> of the sampled equilibrium of a harmonic mode is kT / (m w^2), the Gaussian value."""
    m, w, kT = 1.3, 0.9, 0.7
    model = inputs.Model(nmodes=1, kT=kT, m=(m,), omega=(w,), zeta=(0.4,), gamma=(1.2,), V_LL=(0.8,))
    sq = math.sqrt(kT / (m * w * w))
    pb = oracle.Problem(model, _hgrid([96], [4], [8 * sq]), 2)
    c = oracle.h_boltzmann(pb)
    q2 = oracle.h_observe(pb, inputs.Optical(lin=(0.0,), quad=[[2.0]]), c)
    q1 = oracle.h_observe(pb, inputs.Optical(lin=(1.0,)), c)
    assert q2 == pytest.approx(kT / (m * w * w), rel=1e-12) and abs(q1) < 1e-14


def test_r1_brownian_closed_form_sixth_order():
    """R1 with mu = q of the harmonic Brownian oscillator: -[R4(dt A)^k]_01 (the RK4-discrete
    closed form; A the 3 x 3 first-moment matrix) to sixth order in h_q -- the momenta are
    exact with K = 4 Hermite functions."""
    m, w, kT, zeta, gamma, V = 1.3, 0.9, 0.7, 0.4, 1.2, 0.8
    model = inputs.Model(nmodes=1, kT=kT, m=(m,), omega=(w,), zeta=(zeta,), gamma=(gamma,), V_LL=(V,))
    dt, nt, stride = 0.01, 11, 20
    want = -ref.g_discrete(ref.brownian_matrix(m, w, zeta, gamma, V), dt, [k * stride for k in range(nt)])
    mu = inputs.Optical(lin=(1.0,))
    sq = math.sqrt(kT / (m * w * w))
    errs = []
    for n in (64, 128):
        pb = oracle.Problem(model, _hgrid([n], [4], [8 * sq]), 3)
        R = oracle.h_response1(pb, mu, mu, oracle.h_boltzmann(pb), dt, nt, stride)
        errs.append(np.abs(R - want).max() / np.abs(want).max())
    assert errs[1] < 1e-7 and math.log2(errs[0] / errs[1]) > 5.5, errs


def test_r2_moment_closure_one_mode():
    """R2 with quadratic optics (TRT, RTT, TTR orders) of a harmonic mode with a Drude bath at
    depth 4 against the exact moment closure; K = 6 Hermite functions carry every polynomial
    moment the closure needs, so only the q-stencil error (1e-7 at 128 points) remains."""
    m, w, kT = 0.9, 1.1, 1.2
    model = inputs.Model(nmodes=1, kT=kT, m=(m,), omega=(w,), zeta=(0.6,), gamma=(1.3,), V_LL=(0.9,))
    depth = 4
    mc = ref.MomentClosure(model, depth, K=2)
    mu = inputs.Optical(lin=(1.0,), quad=[[0.4]])
    Pi = inputs.Optical(lin=(0.5,), quad=[[1.1]])
    dt, nt, stride = 0.01, 6, 20
    sq = math.sqrt(kT / (m * w * w))
    grid = _hgrid([128], [6], [8 * sq])
    pb = oracle.Problem(model, grid, depth)
    c = oracle.h_boltzmann(pb)
    qgrid = inputs.Grid(nq=(128,), np=(128,), qmin=(-8 * sq,), qmax=(8 * sq,), pmin=(-8.0,), pmax=(8.0,))
    W0 = ref.boltzmann_grid(model, qgrid)
    for (A, B, C) in [(mu, Pi, mu), (Pi, mu, mu), (mu, mu, Pi)]:
        R = oracle.h_response2(pb, A, B, C, c, dt, nt, nt, stride)
        want = mc.response2(A, B, C, W0, qgrid, dt, nt, nt, stride)
        np.testing.assert_allclose(R, want, rtol=0, atol=1e-6 * np.abs(want).max())


def test_r2_agrees_with_the_grid_representation():
    """The same anharmonic mode with linear + square-linear coupling in both representations
    (Hermite K = 8 against a 96 x 96 (q, p) grid, same q nodes): R2 agrees to the grid
    representation's own discretisation error (2e-7 measured)."""
    model = _anharmonic(1)
    gridp = inputs.default_grid(model, [96])
    mu = inputs.Optical(lin=(1.0,))
    Pi = inputs.Optical(lin=(0.5,), quad=[[0.8]])
    pbg = oracle.Problem(model, gridp, 3)
    Rg = oracle.response2(pbg, mu, Pi, mu, oracle.boltzmann(pbg), 0.005, 6, 6, 40)
    gh = inputs.Grid(nq=(96,), np=(8,), qmin=gridp.qmin, qmax=gridp.qmax, pmin=(0.0,), pmax=(1.0,))
    pbh = oracle.Problem(model, gh, 3)
    Rh = oracle.h_response2(pbh, mu, Pi, mu, oracle.h_boltzmann(pbh), 0.005, 6, 6, 40)
    assert np.abs(Rh - Rg).max() / np.abs(Rg).max() < 2e-6
