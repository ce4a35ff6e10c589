"""Pins of the FP64 oracle against things other than itself (CPU only).

Each test names what fixes the expected value: a Taylor identity, a closed form of the harmonic
Brownian oscillator, the exact moment closure of the adjoint hierarchy, classical trajectories,
Boltzmann stationarity, conservation, separability or reciprocity of equilibrium correlations.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2509_25840_b300 import inputs
import references as ref


# ------------------------------------------------------------------------------------------
# P1 -- the 6th-order central difference
# ------------------------------------------------------------------------------------------

def test_deriv_exact_on_polynomials_up_to_degree_6():
    n, h = 16, 0.37
    x = (np.arange(n) - 7.3) * h
    for k in range(7):
        f = x ** k
        want = k * x ** (k - 1) if k else np.zeros(n)
        got = oracle.deriv1d(f, h)
        np.testing.assert_allclose(got[3:n - 3], want[3:n - 3], rtol=1e-11, atol=1e-11)
    # degree 7 is not differentiated exactly: the scheme is 6th order, no better
    f = x ** 7
    err = np.abs(oracle.deriv1d(f, h)[3:n - 3] - 7 * x[3:n - 3] ** 6).max()
    assert err > 1e-6


def test_deriv_antisymmetric_with_zero_ghosts():
    n, h = 16, 0.5
    D = np.stack([oracle.deriv1d(np.eye(n)[j], h) for j in range(n)], axis=1)
    np.testing.assert_allclose(D, -D.T, atol=1e-15)
    # the interior row is (-1, 9, -45, 0, 45, -9, 1) / (60 h)
    np.testing.assert_allclose(D[8, 5:12] * 60 * h, [-1, 9, -45, 0, 45, -9, 1], atol=1e-12)


def test_deriv_sixth_order_convergence():
    errs = []
    for n in (41, 81, 161):
        x = np.linspace(-1.0, 1.0, n)
        h = x[1] - x[0]
        d = oracle.deriv1d(np.sin(3 * x), h)
        sl = slice(n // 4, 3 * n // 4)
        errs.append(np.abs(d[sl] - 3 * np.cos(3 * x[sl])).max())
    orders = [math.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert all(5.6 < o < 6.4 for o in orders), orders


# ------------------------------------------------------------------------------------------
# potential and its gradient: sympy differentiation of the paper's polynomial
# ------------------------------------------------------------------------------------------

def test_potential_and_gradient_against_symbolic():
    sp = pytest.importorskip("sympy")
    rng = np.random.default_rng(3)
    model = inputs.Model(nmodes=3, m=(1.2, 0.8, 1.5), omega=(0.7, 1.1, 1.9), g3=(0.3, -0.2, 0.1),
                         g4=(0.05, 0.02, 0.07), g2=rng.normal(size=(3, 3)),
                         g_s2s=rng.normal(size=(3, 3)), g_ss2=rng.normal(size=(3, 3)))
    pb = oracle.Problem(model, inputs.default_grid(model, [8]), 0)
    q = sp.symbols("q1:4")
    U = 0
    for s in range(3):
        U += sp.Rational(1, 2) * model.m[s] * model.omega[s] ** 2 * q[s] ** 2 \
            + model.g3[s] * q[s] ** 3 / sp.factorial(3) + model.g4[s] * q[s] ** 4 / sp.factorial(4)
    for a in range(3):
        for b in range(a + 1, 3):
            U += model.g2[a, b] * q[a] * q[b] + sp.Rational(1, 6) * (
                model.g_s2s[a, b] * q[a] ** 2 * q[b] + model.g_ss2[a, b] * q[a] * q[b] ** 2)
    grads = [sp.lambdify(q, sp.diff(U, qs)) for qs in q]
    Uf = sp.lambdify(q, U)
    for _ in range(20):
        x = rng.uniform(-2, 2, size=3)
        assert oracle.potential(pb, x) == pytest.approx(float(Uf(*x)), rel=1e-13, abs=1e-13)
        for s in range(3):
            assert oracle.dUdq(pb, x, s) == pytest.approx(float(grads[s](*x)), rel=1e-12, abs=1e-12)


# ------------------------------------------------------------------------------------------
# P2 -- RK4 stepping: the stability polynomial applied to the extracted generator
# ------------------------------------------------------------------------------------------

def _generator(pb):
    n = pb.M * pb.P
    cols = []
    for j in range(n):
        e = np.zeros(n)
        e[j] = 1.0
        cols.append(oracle.rhs(pb, e).ravel())
    return np.stack(cols, axis=1)


@pytest.mark.parametrize("d,n,depth", [(1, 9, 3), (2, 5, 2)])
def test_rk4_equals_stability_polynomial(d, n, depth):
    model = inputs.Model(nmodes=d, kT=0.8, m=(1.1, 0.9), omega=(1.0, 1.3), g3=(0.2, -0.1),
                         g4=(0.05, 0.03), g_ss2=[[0, 0.2], [0, 0]], g2=[[0, 0.1], [0, 0]],
                         zeta=(0.5, 0.3), gamma=(1.0, 1.5), V_LL=(1.0, 0.7), V_SL=(0.3, 0.2))
    grid = inputs.default_grid(model, [n])
    pb = oracle.Problem(model, grid, depth)
    Mgen = _generator(pb)
    w0 = inputs.random_state(grid, pb.M, seed=11, smooth=False)
    # linearity of the right-hand side
    w1 = inputs.random_state(grid, pb.M, seed=12, smooth=False)
    np.testing.assert_allclose(oracle.rhs(pb, 2.0 * w0 - 0.5 * w1),
                               2.0 * oracle.rhs(pb, w0) - 0.5 * oracle.rhs(pb, w1), atol=1e-11)
    dt, k = 0.01, 7
    want = np.linalg.matrix_power(ref.rk4_poly(dt * Mgen), k) @ w0.ravel()
    got = oracle.rk4(pb, w0, dt, k).ravel()
    np.testing.assert_allclose(got, want, rtol=0, atol=1e-12 * np.abs(want).max())


# ------------------------------------------------------------------------------------------
# P3/P4 -- R1 of the harmonic Brownian oscillator (closed form)
#
# States are symmetrised (g = W exp(H/2kT)), so the moment identities that make the closed forms
# exact for a W-grid hold here up to the O(h^6) error of the stencil: each closed-form pin checks
# that the grid result converges to the closed form at (close to) sixth order.
# ------------------------------------------------------------------------------------------

def _scaled_grid1(m, w, kT, n=64, c=8.0):
    sq, sp_ = math.sqrt(kT / (m * w * w)), math.sqrt(m * kT)
    return inputs.Grid(nq=(n,), np=(n,), qmin=(-c * sq,), qmax=(c * sq,), pmin=(-c * sp_,),
                       pmax=(c * sp_,))


def _converges(run, want, tol, ns=(64, 128), min_order=4.3, scale=None):
    """run(n) -> result on an n x n grid; errors relative to max|want| (or scale)."""
    scale = np.abs(want).max() if scale is None else scale
    errs = [np.abs(run(n) - want).max() / scale for n in ns]
    if errs[-1] < 1e-13:          # exact up to rounding on both grids
        return errs
    order = math.log(errs[0] / errs[1]) / math.log(ns[1] / ns[0])
    assert errs[-1] < tol and order > min_order, (errs, order)
    return errs


def test_r1_brownian_closed_form_discrete_and_continuum():
    m, w, kT, zeta, gamma, V = 1.3, 0.9, 0.7, 0.4, 1.2, 0.8
    model = inputs.Model(nmodes=1, kT=kT, m=(m,), omega=(w,), zeta=(zeta,), gamma=(gamma,),
                         V_LL=(V,))
    depth, dt, nt, stride = 3, 0.01, 60, 10
    mu = inputs.Optical(lin=(1.7,))

    def run(n):
        grid = _scaled_grid1(m, w, kT, n)
        pb = oracle.Problem(model, grid, depth)
        Weq = ref.hierarchy_state(ref.boltzmann_sym(model, grid), pb.M)
        return oracle.response1(pb, mu, mu, Weq, dt, nt, stride)

    A = ref.brownian_matrix(m, w, zeta, gamma, V)
    want = -1.7 ** 2 * ref.g_discrete(A, dt, [k * stride for k in range(nt)])
    _converges(run, want, 5e-7)
    # the continuum Brownian-oscillator formula agrees with the discrete one to the RK4 error
    t = dt * stride * np.arange(nt)
    cont = 1.7 ** 2 * ref.brownian_r1_continuum(m, w, zeta, gamma, V, t)
    np.testing.assert_allclose(want, cont, rtol=0, atol=1e-7 * np.abs(cont).max())


def test_r1_free_oscillator_is_minus_sine():
    m, w = 0.8, 1.4
    model = inputs.Model(nmodes=1, kT=1.0, m=(m,), omega=(w,), zeta=(0.0,), gamma=(1.0,),
                         V_LL=(1.0,))
    mu = inputs.Optical(lin=(1.0,))
    dt, nt, stride = 0.005, 40, 20

    def run(n):
        grid = _scaled_grid1(m, w, 1.0, n)
        pb = oracle.Problem(model, grid, 1)
        Weq = ref.hierarchy_state(ref.boltzmann_sym(model, grid), pb.M)
        return oracle.response1(pb, mu, mu, Weq, dt, nt, stride)

    t = dt * stride * np.arange(nt)
    _converges(run, -np.sin(w * t) / (m * w), 5e-7)


# ------------------------------------------------------------------------------------------
# P5 -- R2 of the harmonic Brownian oscillator (closed forms)
# ------------------------------------------------------------------------------------------

BO = dict(m=1.1, w=1.0, kT=0.9, zeta=0.5, gamma=0.8, V=1.0)


def _bo_r2(A, B, C, depth, dt, nt, stride):
    model = inputs.Model(nmodes=1, kT=BO["kT"], m=(BO["m"],), omega=(BO["w"],),
                         zeta=(BO["zeta"],), gamma=(BO["gamma"],), V_LL=(BO["V"],))

    def run(n):
        grid = _scaled_grid1(BO["m"], BO["w"], BO["kT"], n)
        pb = oracle.Problem(model, grid, depth)
        Weq = ref.hierarchy_state(ref.boltzmann_sym(model, grid), pb.M)
        return oracle.response2(pb, A, B, C, Weq, dt, nt, nt, stride)

    return run


def _bo_matrix():
    return ref.brownian_matrix(BO["m"], BO["w"], BO["zeta"], BO["gamma"], BO["V"])


def test_r2_trt_quadratic_raman_closed_form():
    mu1, Pi1, Pi2 = 1.3, 0.7, 0.9
    mu = inputs.Optical(lin=(mu1,))
    Pi = inputs.Optical(lin=(Pi1,), quad=[[Pi2]])
    dt, nt, stride = 0.01, 8, 25
    g = ref.g_discrete(_bo_matrix(), dt, [k * stride for k in range(nt)])
    want = mu1 ** 2 * Pi2 * np.outer(g, g)
    _converges(_bo_r2(mu, Pi, mu, 3, dt, nt, stride), want, 1e-6)


def test_r2_all_linear_and_rtt_vanish():
    mu = inputs.Optical(lin=(1.0,))
    Pi = inputs.Optical(lin=(0.6,), quad=[[1.5]])
    dt, nt, stride = 0.01, 6, 25
    scale = np.abs(_bo_r2(mu, Pi, mu, 3, dt, nt, stride)(64)).max()
    zero = np.zeros((nt, nt))
    _converges(_bo_r2(mu, mu, mu, 3, dt, nt, stride), zero, 1e-6, scale=scale)
    _converges(_bo_r2(Pi, mu, mu, 3, dt, nt, stride), zero, 1e-6, scale=scale)


def test_r2_ttr_closed_form_pins_theta_factor():
    # R2 = mu^2 Pi2 g(t2) g(t1 + t2) needs members up to tier 2 with the n_s factor on Theta
    mu1, Pi2 = 1.0, 1.2
    mu = inputs.Optical(lin=(mu1,))
    Pi = inputs.Optical(lin=(0.0,), quad=[[Pi2]])
    dt, nt, stride = 0.005, 6, 50
    t = dt * stride * np.arange(nt)
    g = lambda tt: -ref.brownian_r1_continuum(BO["m"], BO["w"], BO["zeta"], BO["gamma"], BO["V"], tt)
    want = mu1 ** 2 * Pi2 * g(t)[None, :] * g(t[:, None] + t[None, :])
    # continuum-time formula: the RK4 time error (~1e-7) is the floor at the finer grid
    _converges(_bo_r2(mu, mu, Pi, 3, dt, nt, stride), want, 1e-6, min_order=3.0)


# ------------------------------------------------------------------------------------------
# moment closure: several modes, bilinear coupling, quadratic optics, RK4 mirrored exactly
# ------------------------------------------------------------------------------------------

def test_moment_closure_one_mode_deep_hierarchy():
    m, w, kT = 0.9, 1.1, 1.2
    model = inputs.Model(nmodes=1, kT=kT, m=(m,), omega=(w,), zeta=(0.6,), gamma=(1.3,),
                         V_LL=(0.9,))
    depth = 4
    mc = ref.MomentClosure(model, depth, K=2)
    mu = inputs.Optical(lin=(1.0,), quad=[[0.4]])
    Pi = inputs.Optical(lin=(0.5,), quad=[[1.1]])
    dt, nt, stride = 0.01, 6, 20
    for (A, B, C) in [(mu, Pi, mu), (Pi, mu, mu), (mu, mu, Pi), (Pi, Pi, Pi)]:
        grid = _scaled_grid1(m, w, kT, 128)
        pb = oracle.Problem(model, grid, depth)
        Weq = ref.hierarchy_state(ref.boltzmann_sym(model, grid), pb.M)
        R = oracle.response2(pb, A, B, C, Weq, dt, nt, nt, stride)
        want = mc.response2(A, B, C, ref.boltzmann_grid(model, grid), grid, dt, nt, nt, stride)
        np.testing.assert_allclose(R, want, rtol=0, atol=1e-6 * np.abs(want).max())


def test_r3_moment_closure_one_mode_deep_hierarchy():
    """Eq. 3Dresponse against the exact moment closure: one harmonic mode with a Drude bath at
    depth 4, linear and quadratic optics in several orders, waiting time 0.15."""
    m, w, kT = 0.9, 1.1, 1.2
    model = inputs.Model(nmodes=1, kT=kT, m=(m,), omega=(w,), zeta=(0.6,), gamma=(1.3,),
                         V_LL=(0.9,))
    depth = 4
    mc = ref.MomentClosure(model, depth, K=2)
    mu = inputs.Optical(lin=(1.0,), quad=[[0.4]])
    Pi = inputs.Optical(lin=(0.5,), quad=[[1.1]])
    dt, nt, stride, n2 = 0.01, 5, 20, 15
    grid = _scaled_grid1(m, w, kT, 128)
    pb = oracle.Problem(model, grid, depth)
    Weq = ref.hierarchy_state(ref.boltzmann_sym(model, grid), pb.M)
    W0 = ref.boltzmann_grid(model, grid)
    for ops in [(mu, Pi, Pi, mu), (Pi, mu, mu, Pi), (mu, mu, Pi, Pi), (Pi, Pi, Pi, Pi)]:
        R = oracle.response3(pb, *ops, Weq, dt, nt, n2, nt, stride)
        want = mc.response3(*ops, W0, grid, dt, nt, n2, nt, stride)
        assert np.abs(want).max() > 1e-3
        np.testing.assert_allclose(R, want, rtol=0, atol=1e-6 * np.abs(want).max())


def test_r3_all_linear_vanishes():
    """Harmonic mode, linear A, B, C, D: the third-order response is zero (each linear insertion
    lowers the polynomial degree of the adjoint observable by one)."""
    model = inputs.Model(nmodes=1, kT=BO["kT"], m=(BO["m"],), omega=(BO["w"],),
                         zeta=(BO["zeta"],), gamma=(BO["gamma"],), V_LL=(BO["V"],))
    mu = inputs.Optical(lin=(1.0,))
    Pi = inputs.Optical(lin=(0.6,), quad=[[1.5]])
    dt, nt, stride, n2 = 0.01, 4, 25, 10

    def run(ops):
        def f(n):
            grid = _scaled_grid1(BO["m"], BO["w"], BO["kT"], n)
            pb = oracle.Problem(model, grid, 3)
            Weq = ref.hierarchy_state(ref.boltzmann_sym(model, grid), pb.M)
            return oracle.response3(pb, *ops, Weq, dt, nt, n2, nt, stride)
        return f

    scale = np.abs(run((mu, Pi, Pi, mu))(64)).max()
    # sixth-order convergence to zero (2.5e-6 of the quadratic-optics R3 at 128 points)
    _converges(run((mu, mu, mu, mu)), np.zeros((nt, nt)), 1e-5, scale=scale)


@pytest.mark.slow
def test_moment_closure_two_coupled_modes():
    # 4D grids are coarse (h ~ 0.5 sigma at 28 points), so the O(h^6) error of the stencil is
    # ~5e-4 of R2 there; the pin is convergence towards the moment closure between 20^4 and 28^4
    # (the bilinear coupling itself moves R2 by 1e-2, halving zeta_2 by 5e-3).
    model = inputs.Model(nmodes=2, kT=1.0, m=(1.0, 1.3), omega=(1.0, 1.4), g2=[[0, 0.25], [0, 0]],
                         zeta=(0.4, 0.7), gamma=(1.0, 1.6), V_LL=(1.0, 0.8))
    depth = 2
    mc = ref.MomentClosure(model, depth, K=2)
    mu = inputs.Optical(lin=(1.0, 0.6), quad=[[0.0, 0.3], [0.3, 0.0]])
    Pi = inputs.Optical(lin=(0.4, 1.0), quad=[[0.5, 0.2], [0.2, -0.3]])
    dt, nt, stride = 0.02, 3, 8
    grid_of = lambda n: inputs.default_grid(model, [n], nsigma=6.5, cut=6.5 ** 2 / 2)

    def run(n):
        grid = grid_of(n)
        pb = oracle.Problem(model, grid, depth)
        Weq = ref.hierarchy_state(ref.boltzmann_sym(model, grid), pb.M)
        return oracle.response2(pb, mu, Pi, mu, Weq, dt, nt, nt, stride)

    # the closure's equilibrium moments depend on the grid only at the 1e-12 level here
    want = mc.response2(mu, Pi, mu, ref.boltzmann_grid(model, grid_of(28)), grid_of(28), dt, nt,
                        nt, stride)
    _converges(run, want, 1e-3, ns=(20, 28), min_order=4.0)


# ------------------------------------------------------------------------------------------
# P9 -- anharmonic potential, zeta = 0: classical trajectories
# ------------------------------------------------------------------------------------------

@pytest.mark.slow
def test_r1_anharmonic_free_mode_matches_trajectories():
    model = inputs.Model(nmodes=1, kT=1.0, m=(1.0,), omega=(1.0,), g3=(0.35,), g4=(0.15,),
                         zeta=(0.0,), gamma=(1.0,), V_LL=(1.0,))
    grid = inputs.default_grid(model, [128], nsigma=7.0, cut=24.0)
    pb = oracle.Problem(model, grid, 0)
    Weq = ref.hierarchy_state(ref.boltzmann_sym(model, grid), pb.M)
    mu = inputs.Optical(lin=(1.0,))
    dt, nt, stride = 0.004, 13, 125
    R = oracle.response1(pb, mu, mu, Weq, dt, nt, stride)
    t = dt * stride * np.arange(nt)
    want = ref.trajectory_r1(model, 1.0, t, nq=44, npq=32)
    # the anharmonic terms move R1 by 3e-2 over t <= 6; the grid result agrees to 1.5e-7
    assert np.abs(want + np.sin(t)).max() > 2e-2
    np.testing.assert_allclose(R, want, rtol=0, atol=5e-7)


# ------------------------------------------------------------------------------------------
# P6/P7 -- Boltzmann stationarity, norm conservation
# ------------------------------------------------------------------------------------------

def _anharmonic_sl_model(d):
    return inputs.Model(nmodes=d, kT=0.9, m=(1.2, 0.8, 1.0), omega=(1.0, 1.3, 0.7),
                        g3=(0.2, -0.15, 0.1), g4=(0.05, 0.04, 0.06),
                        g2=[[0, 0.1, 0.05], [0, 0, -0.1]], g_s2s=[[0, 0.2, 0.1], [0, 0, 0.1]],
                        g_ss2=[[0, 0.12, 0.1], [0, 0, 0.05]], zeta=(0.5, 0.3, 0.4),
                        gamma=(1.0, 1.5, 0.8), V_LL=(1.0, 0.7, 0.9), V_SL=(0.3, -0.4, 0.2))


def test_boltzmann_is_stationary_to_sixth_order():
    # residual of the distribution W = exp(-H/2kT) g, relative to max |W|
    model = _anharmonic_sl_model(1)
    res = []
    ns = (32, 48, 64)
    for n in ns:
        grid = inputs.default_grid(model, [n])
        pb = oracle.Problem(model, grid, 3)
        w = ref.sym_weight(model, grid)[None]
        G = ref.hierarchy_state(ref.boltzmann_sym(model, grid), pb.M)
        res.append(np.abs(oracle.rhs(pb, G) * w).max() / np.abs(G * w).max())
    orders = [math.log(res[i] / res[i + 1]) / math.log(ns[i + 1] / ns[i]) for i in range(2)]
    assert res[-1] < 1e-5
    assert all(5.0 < o < 7.5 for o in orders), (res, orders)
    # the wrong temperature is not stationary at any resolution
    hot = ref.hierarchy_state(ref.boltzmann_sym(model.replace(kT=1.2 * model.kT), grid), pb.M)
    assert np.abs(oracle.rhs(pb, hot) * w).max() / np.abs(hot * w).max() > 1e3 * res[-1]


@pytest.mark.parametrize("d,ns,depth,min_order", [(2, (14, 20, 26), 2, 4.5), (3, (8, 11), 1, 4.5)])
def test_boltzmann_stationary_multimode(d, ns, depth, min_order):
    # mode couplings (bilinear and cubic), square-linear bath coupling: the residual of the
    # distribution W = exp(-H/2kT) g must fall at the order of the stencil
    model = _anharmonic_sl_model(d)
    res = []
    for n in ns:
        grid = inputs.default_grid(model, [n], cut=12.0, nsigma=5.0)
        pb = oracle.Problem(model, grid, depth)
        w = ref.sym_weight(model, grid)[None]
        G = ref.hierarchy_state(ref.boltzmann_sym(model, grid), pb.M)
        res.append(np.abs(oracle.rhs(pb, G) * w).max() / np.abs(G * w).max())
    orders = [math.log(res[i] / res[i + 1]) / math.log(ns[i + 1] / ns[i]) for i in range(len(ns) - 1)]
    assert all(o > min_order for o in orders), (res, orders)


def test_norm_conserved_and_insertion_has_zero_mass():
    model = _anharmonic_sl_model(1)
    grid = inputs.default_grid(model, [96], nsigma=8.0, cut=32.0)
    pb = oracle.Problem(model, grid, 3)
    vol = ref.cell_volume(grid)
    w = ref.sym_weight(model, grid)
    G = ref.hierarchy_state(ref.boltzmann_sym(model, grid), pb.M)
    X = inputs.Optical(lin=(1.0,), quad=[[0.7]])
    Gx = oracle.insert(pb, X, G)
    assert abs(vol * np.sum(w * Gx[0])) < 1e-9
    # a displaced distribution moves; integral W^(0) stays (every term of its equation is a
    # derivative; on the grid it holds to the O(h^6) error of the symmetrised operators)
    G1 = ref.hierarchy_state(ref.boltzmann_sym(model, grid) * np.exp(0.4 * np.linspace(-1, 1, 96))[:, None], pb.M)
    n0 = vol * np.sum(w * G1[0])
    G2 = oracle.rk4(pb, G1, 0.005, 200)
    assert abs(vol * np.sum(w * G2[0]) - n0) < 1e-8 * abs(n0)
    assert np.abs(G2[0] - G1[0]).max() > 1e-3 * np.abs(G1[0]).max()


def test_observe_gaussian_moments():
    m, w, kT = 1.3, 0.8, 0.6
    model = inputs.Model(nmodes=2, kT=kT, m=(m, 1.0), omega=(w, 1.0))
    grid = inputs.default_grid(model, [40], nsigma=8.0, cut=32.0)
    pb = oracle.Problem(model, grid, 1)
    W = ref.hierarchy_state(ref.boltzmann_sym(model, grid), pb.M)
    C = inputs.Optical(lin=(0.3, -0.2), quad=[[2.0, 0.5], [0.5, 4.0]])
    # <C> = 1/2 (2 <q1^2> + 4 <q2^2>) with <q_s^2> = kT / (m_s w_s^2); odd and cross moments vanish
    want = 0.5 * (2.0 * kT / (m * w * w) + 4.0 * kT / 1.0)
    assert oracle.observe(pb, C, W) == pytest.approx(want, rel=1e-10)


def test_insert_matches_analytic_derivative_of_boltzmann():
    # X^x W_B = sum_s dX/dq_s (-p_s / (m_s kT)) W_B; the p axes are fine, the q axes coarse
    model = inputs.Model(nmodes=2, kT=0.8, m=(1.0, 1.4), omega=(1.0, 0.9), g4=(0.05, 0.02))
    base = inputs.default_grid(model, [12, 12, 72, 72], nsigma=8.0, cut=18.0)
    pb = oracle.Problem(model, base, 1)
    wgt = ref.sym_weight(model, base)
    W0 = ref.boltzmann_grid(model, base)
    G = ref.hierarchy_state(W0 / wgt, pb.M)
    X = inputs.Optical(lin=(0.7, -1.1), quad=[[0.4, 0.9], [0.1, -0.6]])
    got = oracle.insert(pb, X, G)
    mesh = np.meshgrid(*ref.grid_axes(base), indexing="ij")
    q, p = mesh[:2], mesh[2:]
    Qs = 0.5 * (X.quad[:2, :2] + X.quad[:2, :2].T)
    want = np.zeros_like(W0)
    for s in range(2):
        grad = X.lin[s] + Qs[s, 0] * q[0] + Qs[s, 1] * q[1]
        want += grad * (-p[s] / (model.m[s] * model.kT)) * W0
    np.testing.assert_allclose(got[0] * wgt, want, rtol=0, atol=1e-5 * np.abs(want).max())
    assert np.abs(got[1:]).max() == 0.0


# ------------------------------------------------------------------------------------------
# P8 -- separability: uncoupled modes respond as the sum of single modes
# ------------------------------------------------------------------------------------------

@pytest.mark.slow
def test_separable_two_modes_equal_sum_of_single_modes():
    """Uncoupled modes: the 4D operator is a Kronecker sum of 2D ones, so R1 for a sum of
    per-mode linear dipoles is the sum of the single-mode R1s.  The sum-truncation of the 4D
    hierarchy cuts product members (n1, n2) with n1 + n2 > depth, which only the O(h^6)
    non-stationarity of each mode's sampled Boltzmann reaches: agreement to 1e-8."""
    kw = dict(zeta=(0.4, 0.6), gamma=(1.0, 1.5), V_LL=(1.0, 0.8), V_SL=(0.3, 0.2),
              g3=(0.1, -0.2), g4=(0.05, 0.03), m=(1.0, 1.2), omega=(1.0, 1.4))
    model2 = inputs.Model(nmodes=2, kT=0.9, **kw)
    grid2 = inputs.default_grid(model2, [22])
    depth = 2
    pb2 = oracle.Problem(model2, grid2, depth)
    W2 = ref.hierarchy_state(ref.boltzmann_sym(model2, grid2), pb2.M)
    mu2 = inputs.Optical(lin=(0.8, 1.3))
    dt, nt, stride = 0.01, 5, 10
    R2 = oracle.response1(pb2, mu2, mu2, W2, dt, nt, stride)
    total = np.zeros(nt)
    for s, mus in ((0, 0.8), (1, 1.3)):
        m1 = inputs.Model(nmodes=1, kT=0.9, **{k: (v[s],) for k, v in kw.items()})
        g1 = inputs.Grid(nq=(grid2.nq[s],), np=(grid2.np[s],), qmin=(grid2.qmin[s],),
                         qmax=(grid2.qmax[s],), pmin=(grid2.pmin[s],), pmax=(grid2.pmax[s],))
        pb1 = oracle.Problem(m1, g1, depth)
        W1 = ref.hierarchy_state(ref.boltzmann_sym(m1, g1), pb1.M)
        mu1 = inputs.Optical(lin=(mus,))
        total += oracle.response1(pb1, mu1, mu1, W1, dt, nt, stride)
    np.testing.assert_allclose(R2, total, rtol=0, atol=1e-7 * np.abs(total).max())


# ------------------------------------------------------------------------------------------
# reciprocity of equilibrium correlations: <q(t) p(0)> = -<p(t) q(0)>  (any U, LL + SL)
# ------------------------------------------------------------------------------------------

@pytest.mark.slow
def test_reciprocity_square_linear_coupling():
    """The hierarchy is the exact reduction of a Hamiltonian system + harmonic bath (Sec. II A),
    and its plain truncation is a Galerkin projection that keeps the time-reversal structure, so
    equilibrium cross-correlations of an even (q) and an odd (p) observable are antisymmetric.
    A wrong sign or weight on the square-linear part of Phi or Theta breaks it."""
    model = inputs.Model(nmodes=1, kT=1.0, m=(1.0,), omega=(1.0,), g3=(0.3,), g4=(0.1,),
                         zeta=(0.8,), gamma=(1.2,), V_LL=(0.6,), V_SL=(0.5,))
    grid = inputs.default_grid(model, [72], nsigma=7.0, cut=24.0)
    depth = 4
    pb = oracle.Problem(model, grid, depth)
    Geq, steps, res = oracle.equilibrate(pb, 0.004, 4000, 1e-11, 500)
    q, p = np.meshgrid(*ref.grid_axes(grid), indexing="ij")
    w = ref.sym_weight(model, grid)
    vol = ref.cell_volume(grid)
    pG, qG = Geq * p[None], Geq * q[None]
    qp, pq = [], []
    for _ in range(6):
        pG = oracle.rk4(pb, pG, 0.004, 125)
        qG = oracle.rk4(pb, qG, 0.004, 125)
        qp.append(vol * np.sum(q * w * pG[0]))
        pq.append(vol * np.sum(p * w * qG[0]))
    qp, pq = np.array(qp), np.array(pq)
    scale = max(np.abs(qp).max(), np.abs(pq).max())
    assert scale > 0.1
    np.testing.assert_allclose(qp, -pq, rtol=0, atol=2e-6 * scale)


# ------------------------------------------------------------------------------------------
# equilibration: stationary result, O(h^6) from the sampled Boltzmann
# ------------------------------------------------------------------------------------------

def test_equilibrate_reaches_discrete_steady_state():
    wl = inputs.one_mode_64()
    pb = oracle.Problem(wl.model, wl.grid, wl.depth)
    G_B = oracle.boltzmann(pb)
    np.testing.assert_allclose(G_B[0], ref.boltzmann_sym(wl.model, wl.grid), rtol=1e-12,
                               atol=1e-15)
    np.testing.assert_allclose(oracle.to_density(pb, G_B)[0], ref.boltzmann_grid(wl.model, wl.grid),
                               rtol=1e-12, atol=1e-15)
    r0 = oracle.residual(pb, G_B)
    G, steps, r = oracle.equilibrate(pb, wl.dt, 3000, 1e-9, 100)
    assert r < r0 / 20
    assert np.abs(G - G_B).max() < 1e-3 * np.abs(G_B).max()


def test_residual_pins():
    """orc_residual (max |M g| / max |g|, the equilibration's stop criterion, Sec. IV B): zero on
    an exact null vector of the generator (extracted column by column and solved for with numpy),
    invariant under scaling and sign, and O(h^6) on the sampled Boltzmann state (the ratio between
    two resolutions close to the ratio of h^6)."""
    model = inputs.Model(nmodes=1, kT=0.8, m=(1.1,), omega=(0.9,), g4=(0.05,), zeta=(0.3,),
                         gamma=(1.2,), V_LL=(1.0,), V_SL=(0.2,))
    grid = inputs.default_grid(model, [9])
    pb = oracle.Problem(model, grid, 2)
    N = pb.M * pb.P
    M = np.stack([oracle.rhs(pb, np.eye(N)[j].reshape(pb.state_shape)).ravel() for j in range(N)], axis=1)
    w, V = np.linalg.eig(M)
    j = int(np.argmin(np.abs(w)))
    assert abs(w[j]) < 1e-10                       # the generator has a null vector (stationary state)
    v = np.real(V[:, j] * np.exp(-1j * np.angle(V[np.argmax(np.abs(V[:, j])), j])))
    assert oracle.residual(pb, v.reshape(pb.state_shape)) < 1e-10
    W = inputs.random_state(grid, pb.M, seed=3, smooth=True)
    r = oracle.residual(pb, W)
    assert r > 1e-3
    assert oracle.residual(pb, -3.7 * W) == pytest.approx(r, rel=1e-14)
    res = []
    for n in (64, 96):   # a domain wide enough (U = 32 kT, 8 sigma in p) that the ends do not show
        pbn = oracle.Problem(model, inputs.default_grid(model, [n], cut=32.0, nsigma=8.0), 2)
        res.append(oracle.residual(pbn, oracle.boltzmann(pbn)))
    assert 0.7 * (96 / 64) ** 6 < res[0] / res[1] < 1.4 * (96 / 64) ** 6, res
