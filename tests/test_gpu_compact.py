"""GPU parity of the compact q-derivatives of Sec. III B (tridiagonal systems solved by parallel
cyclic reduction, Sec. III C) in the Hermite representation: libchfpe with p_basis = 1,
q_scheme = 1, through its C ABI, against the oracle's h_* functions with qscheme = 1 (which
solves every line by forward elimination and back substitution) on the same seeded inputs.
Tolerances as for the other representations: operators 1e-13 (FP64) / 3e-6 (FP32) of max, RK4
1e-12 / 2e-5, responses 1e-10 / 1e-4 of max|R|."""
import math

import numpy as np
import pytest

import oracle
from paper_2509_25840_b300 import inputs
import references as ref

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2509_25840_b300 import build
    build.build()


def _chfpe():
    from paper_2509_25840_b300 import chfpe
    return chfpe


def _model(d):
    return inputs.Model(nmodes=d, kT=0.9, m=(1.2, 0.8, 1.0), omega=(1.0, 1.3, 0.7),
                        g3=(0.2, -0.15, 0.1), g4=(0.05, 0.04, 0.06),
                        g2=[[0, 0.1, 0.05], [0, 0, -0.1]], g_s2s=[[0, 0.2, 0.1], [0, 0, 0.1]],
                        g_ss2=[[0, 0.12, 0.1], [0, 0, 0.05]], zeta=(0.5, 0.3, 0.4),
                        gamma=(1.0, 1.5, 0.8), V_LL=(1.0, 0.7, 0.9), V_SL=(0.3, -0.4, 0.2))


def _hgrid(nq, K, L=5.0):
    d = len(nq)
    return inputs.Grid(nq=tuple(nq), np=tuple(K), qmin=(-L,) * d, qmax=(L,) * d,
                       pmin=(0.0,) * d, pmax=(1.0,) * d)


def _dtype(prec):
    return torch.float64 if prec == 64 else torch.float32


def _rounded(W, prec):
    return W if prec == 64 else W.astype(np.float32).astype(np.float64)


# (modes, q points, Hermite functions, depth): line lengths that are and are not powers of two
# (PCR levels ceil(log2 n)), a line longer than a 32-column tile's rows, K = 1, odd K
CASES = [
    (1, [37], [9], 5),
    (1, [64], [1], 3),
    (1, [200], [3], 2),
    (2, [11, 16], [5, 6], 4),
    (2, [9, 10], [7, 3], 2),
    (3, [7, 8, 9], [3, 4, 2], 2),
    (2, [8, 32], [6, 6], 4),       # the row kernel reading the derivative arrays (3 pairs per thread)
]


def _handle(d, nq, K, depth, prec, max_batch=1, dt=0.003, qs=1):
    chfpe = _chfpe()
    model = _model(d)
    grid = _hgrid(nq, K)
    h = chfpe.Handle(model, grid, depth=depth, dt=dt, precision=prec, max_batch=max_batch,
                     p_basis=1, q_scheme=qs)
    return h, oracle.Problem(model, grid, depth, qscheme=qs)


def _random(pb, seed):
    return inputs.uniform_array(seed, pb.M * pb.P).reshape(pb.state_shape)


@pytest.mark.parametrize("qs", [1, 2])
@pytest.mark.parametrize("prec", [64, 32])
@pytest.mark.parametrize("d,nq,K,depth", CASES)
def test_compact_rhs_matches_oracle(d, nq, K, depth, prec, qs):
    """The right-hand side of three seeded states at once (more states than the handle's
    derivative arrays hold: the library works through them in chunks), for the compact scheme
    (qs = 1) and its skew-symmetric part (qs = 2)."""
    h, pb = _handle(d, nq, K, depth, prec, max_batch=2, qs=qs)
    with h:
        C = [_rounded(_random(pb, 31 + 7 * b + d), prec) for b in range(3)]
        want = [oracle.h_rhs(pb, c) for c in C]
        x = torch.tensor(np.stack(C), dtype=_dtype(prec), device="cuda")
        y = torch.empty_like(x)
        h.rhs_device(x.data_ptr(), y.data_ptr(), 3)
        got = y.double().cpu().numpy()
    tol = 1e-13 if prec == 64 else 3e-6
    for b in range(3):
        assert np.abs(got[b] - want[b]).max() <= tol * np.abs(want[b]).max(), b


@pytest.mark.parametrize("qs", [1, 2])
@pytest.mark.parametrize("prec", [64, 32])
@pytest.mark.parametrize("d,nq,K,depth", [CASES[0], CASES[3], CASES[5], CASES[6]])
def test_compact_rk4_matches_oracle(d, nq, K, depth, prec, qs):
    h, pb = _handle(d, nq, K, depth, prec, max_batch=2, qs=qs)
    with h:
        C = _rounded(_random(pb, 5) * 1e-2 + oracle.h_boltzmann(pb), prec)
        want = oracle.h_rk4(pb, C, 0.003, 20)
        x = torch.tensor(np.stack([C, -C]), dtype=_dtype(prec), device="cuda")
        h.rk4_device(x.data_ptr(), 2, 20)
        got = x.double().cpu().numpy()
    tol = 1e-12 if prec == 64 else 2e-5
    scale = np.abs(want).max()
    assert np.abs(got[0] - want).max() <= tol * scale
    assert np.abs(got[1] + want).max() <= tol * scale


@pytest.mark.parametrize("qs", [1, 2])
@pytest.mark.parametrize("d,nq,K,depth,dt,stride,nt", [
    (1, [48], [8], 4, 0.005, 20, 12),
    (2, [12, 13], [6, 5], 3, 0.004, 30, 4),
])
def test_compact_responses_match_oracle(d, nq, K, depth, dt, stride, nt, qs):
    """R1 and R2 (batched branches, chunks of 3) with compact q-derivatives: FP64 to 1e-10, FP32
    to 1e-4 of max|R| against the oracle (every branch propagated on its own)."""
    chfpe = _chfpe()
    model = _model(d)
    grid = _hgrid(nq, K)
    pb = oracle.Problem(model, grid, depth, qscheme=qs)
    Ceq = _rounded(oracle.h_boltzmann(pb), 32)
    mu = inputs.Optical(lin=(1.0, 0.6), quad=[[0.3, 0.1], [0.1, -0.2]])
    Pi = inputs.Optical(lin=(0.5, 1.0), quad=[[0.8, 0.0], [0.0, 0.4]])
    w1 = oracle.h_response1(pb, mu, mu, Ceq, dt, nt, stride)
    w2 = oracle.h_response2(pb, mu, Pi, mu, Ceq, dt, nt, nt, stride)
    for prec, tol in ((64, 1e-10), (32, 1e-4)):
        with chfpe.Handle(model, grid, depth=depth, dt=dt, precision=prec, max_batch=3,
                          p_basis=1, q_scheme=qs) as h:
            h.set_equilibrium(Ceq)
            r1 = h.response1(mu, mu, nt, stride)
            r2 = h.response2(mu, Pi, mu, nt, nt, stride)
        assert np.abs(r1 - w1).max() < tol * np.abs(w1).max(), (prec, "R1")
        assert np.abs(r2 - w2).max() < tol * np.abs(w2).max(), (prec, "R2")


def test_compact_r1_brownian_closed_form_on_the_gpu():
    """The harmonic Brownian oscillator's R1 (mu = q) on the GPU in FP64 with both q schemes
    against the RK4-discrete closed form: the compact scheme is the more accurate on the same
    grid, and sixth order."""
    chfpe = _chfpe()
    m, w, kT, zeta, gamma, V = 1.3, 0.9, 0.7, 0.4, 1.2, 0.8
    model = inputs.Model(nmodes=1, kT=kT, m=(m,), omega=(w,), zeta=(zeta,), gamma=(gamma,), V_LL=(V,))
    dt, nt, stride = 0.01, 11, 20
    want = -ref.g_discrete(ref.brownian_matrix(m, w, zeta, gamma, V), dt, [k * stride for k in range(nt)])
    mu = inputs.Optical(lin=(1.0,))
    L = 8 * math.sqrt(kT / (m * w * w))
    err = {}
    for n in (48, 96):
        for qs in (0, 1):
            grid = inputs.Grid(nq=(n,), np=(4,), qmin=(-L,), qmax=(L,), pmin=(0.0,), pmax=(1.0,))
            with chfpe.Handle(model, grid, depth=3, dt=dt, precision=64, p_basis=1, q_scheme=qs) as h:
                h.equilibrate(0, 1.0, 1)                # the sampled Boltzmann coefficients
                R = h.response1(mu, mu, nt, stride)
            err[n, qs] = np.abs(R - want).max() / np.abs(want).max()
    assert err[96, 1] < 1e-7 and math.log2(err[48, 1] / err[96, 1]) > 5.5, err
    assert err[48, 1] < err[48, 0] / 4, err


@pytest.mark.parametrize("max_batch", [1, 4])
@pytest.mark.parametrize("qs", [1, 2])
def test_compact_fp64_equilibration_of_an_fp32_handle(qs, max_batch):
    """An FP32 handle equilibrates in FP64 through the same derivative arrays and PCR tables
    (FP64 copies of both): 100 FP64 steps from the sampled Boltzmann coefficients against the
    oracle's h_rk4; the handle keeps its equilibrium in FP32, so every value agrees to the FP32
    rounding of the FP64 result (half an ulp, 2^-24 relative, plus 1e-12 of the maximum for the
    FP64 steps)."""
    h, pb = _handle(2, [11, 16], [5, 6], 2, 32, max_batch=max_batch, qs=qs)
    with h:
        steps, res = h.equilibrate(100, 0.0, 50)
        got = h.get_equilibrium()
    want = oracle.h_rk4(pb, oracle.h_boltzmann(pb), 0.003, 100)
    assert steps == 100
    bound = 2.0 ** -24 * np.abs(want) * 1.01 + 1e-12 * np.abs(want).max()
    assert np.all(np.abs(got - want) <= bound), np.abs(got - want).max()
