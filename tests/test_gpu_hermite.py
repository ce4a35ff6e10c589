"""GPU parity of the Hermite-function momentum representation (Sec. III A, Appendix A,
Eq. HEOM2FP-H): libchfpe with p_basis = 1, through its C ABI, against the oracle's h_* functions
on the same seeded inputs; and the GPU responses of both representations of one model against
each other.  Tolerances as for the grid representation: operators 1e-13 (FP64) / 3e-6 (FP32) of
max, RK4 1e-12 / 2e-5, responses 1e-10 / 1e-4 of max|R|."""
import math

import numpy as np
import pytest

import oracle
from paper_2509_25840_b300 import inputs

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


# (modes, q points, Hermite functions, depth): ragged q extents, K = 1 (no ladder) and odd K
CASES = [
    (1, [37], [9], 5),
    (1, [64], [1], 3),
    (2, [11, 13], [5, 6], 4),
    (2, [9, 10], [7, 3], 2),
    (3, [7, 8, 9], [3, 4, 2], 2),
    (2, [11, 13], [6, 6], 5),      # row-marching kernel: 2, 2 and 8 elements per thread
    (2, [10, 7], [8, 8], 3),
    (2, [9, 40], [6, 7], 2),
    (2, [8, 32], [6, 6], 4),       # the 32-point q_2 rows of 6 x 6 functions (5 per thread)
    (2, [7, 131], [6, 6], 1),      # the shortest q extent; rows too long for it (gather kernel)
]


def _setup(d, nq, K, depth, prec, max_batch=1, dt=0.004):
    chfpe = _chfpe()
    model = _model(d)
    grid = _hgrid(nq, K)
    h = chfpe.Handle(model, grid, depth=depth, dt=dt, precision=prec, max_batch=max_batch,
                     p_basis=1)
    return model, grid, h, oracle.Problem(model, grid, depth)


def _random(pb, seed):
    return inputs.uniform_array(seed, pb.M * pb.P).reshape(pb.state_shape)


@pytest.mark.parametrize("prec", [64, 32])
@pytest.mark.parametrize("d,nq,K,depth", CASES)
def test_hermite_rhs_matches_oracle(d, nq, K, depth, prec):
    model, grid, h, pb = _setup(d, nq, K, depth, prec)
    with h:
        C = _rounded(_random(pb, 11 + d), prec)
        want = oracle.h_rhs(pb, C)
        x = torch.tensor(C, dtype=_dtype(prec), device="cuda")
        y = torch.empty_like(x)
        h.rhs_device(x.data_ptr(), y.data_ptr(), 1)
        got = y.double().cpu().numpy()
    tol = 1e-13 if prec == 64 else 3e-6
    assert np.abs(got - want).max() <= tol * np.abs(want).max()


@pytest.mark.parametrize("prec", [64, 32])
@pytest.mark.parametrize("d,nq,K,depth", [CASES[2], CASES[4], CASES[8]])
def test_hermite_rhs_with_pointers_off_the_vector_boundaries(d, nq, K, depth, prec):
    """Two states starting one element past a 16-byte boundary: the aligned paths (element pairs,
    16-byte row copies) must step aside for the scalar row kernel with element copies, or the
    gather kernel, and give the same result."""
    model, grid, h, pb = _setup(d, nq, K, depth, prec, max_batch=2)
    with h:
        C = np.stack([_rounded(_random(pb, 21), prec), _rounded(_random(pb, 22), prec)])
        want = [oracle.h_rhs(pb, C[b]) for b in range(2)]
        n = C[0].size
        x = torch.zeros(2 * n + 1, dtype=_dtype(prec), device="cuda")
        y = torch.zeros(2 * n + 1, dtype=_dtype(prec), device="cuda")
        x[1:] = torch.tensor(C.reshape(-1), dtype=_dtype(prec), device="cuda")
        es = x.element_size()
        h.rhs_device(x.data_ptr() + es, y.data_ptr() + es, 2)
        got = y[1:].double().cpu().numpy().reshape(C.shape)
    tol = 1e-13 if prec == 64 else 3e-6
    for b in range(2):
        assert np.abs(got[b] - want[b]).max() <= tol * np.abs(want[b]).max()


@pytest.mark.parametrize("prec", [64, 32])
@pytest.mark.parametrize("d,nq,K,depth", [CASES[0], CASES[2], CASES[4], CASES[5], CASES[7], CASES[8]])
def test_hermite_rk4_insert_observe_match_oracle(d, nq, K, depth, prec):
    model, grid, h, pb = _setup(d, nq, K, depth, prec, max_batch=2)
    with h:
        C = _rounded(_random(pb, 5) * 1e-2 + oracle.h_boltzmann(pb), prec)
        want = oracle.h_rk4(pb, C, 0.004, 20)
        x = torch.tensor(np.stack([C, -C]), dtype=_dtype(prec), device="cuda")
        h.rk4_device(x.data_ptr(), 2, 20)
        got = x.double().cpu().numpy()
        tol = 1e-12 if prec == 64 else 2e-5
        scale = np.abs(want).max()
        assert np.abs(got[0] - want).max() <= tol * scale
        assert np.abs(got[1] + want).max() <= tol * scale
        X = inputs.Optical(lin=(0.7, -1.1, 0.4), quad=[[0.4, 0.9, 0.1], [0.1, -0.6, 0.2], [0.3, 0.0, 0.5]])
        wi = oracle.h_insert(pb, X, C)
        xi = torch.tensor(C, dtype=_dtype(prec), device="cuda")
        yi = torch.empty_like(xi)
        h.insert_device(X, xi.data_ptr(), yi.data_ptr(), 1)
        assert np.abs(yi.double().cpu().numpy() - wi).max() <= (1e-13 if prec == 64 else 3e-6) * np.abs(wi).max()
        Rd = torch.zeros(1, dtype=torch.float64, device="cuda")
        h.observe_device(X, xi.data_ptr(), 1, Rd.data_ptr())
        assert Rd.item() == pytest.approx(oracle.h_observe(pb, X, C), rel=1e-12, abs=1e-14)


def test_hermite_equilibrate_matches_oracle():
    """FP64 equilibration from the sampled Boltzmann coefficients (c^(0)_0 = exp(-U/2kT) / Z):
    300 steps against the oracle's h_boltzmann + h_rk4."""
    model, grid, h, pb = _setup(2, [12, 11], [5, 6], 2, 64)
    with h:
        steps, res = h.equilibrate(300, 0.0, 100)
        got = h.get_equilibrium()
    want = oracle.h_rk4(pb, oracle.h_boltzmann(pb), 0.004, 300)
    assert steps == 300
    assert np.abs(got - want).max() <= 1e-12 * np.abs(want).max()


@pytest.mark.parametrize("d,nq,K,depth,dt,stride,nt", [
    (1, [48], [8], 4, 0.005, 20, 12),
    (2, [12, 12], [6, 6], 3, 0.005, 30, 4),
])
def test_hermite_responses_match_oracle(d, nq, K, depth, dt, stride, nt):
    """R1, R2 (batched branches, chunks of 3) and R3 in the Hermite representation: FP64 to 1e-10,
    FP32 to 1e-4 of max|R| against the oracle (which propagates each branch on its own)."""
    chfpe = _chfpe()
    model = _model(d)
    grid = _hgrid(nq, K)
    pb = oracle.Problem(model, grid, depth)
    Ceq = _rounded(oracle.h_boltzmann(pb), 32)
    mu = inputs.Optical(lin=(1.0, 0.6), quad=[[0.3, 0.1], [0.1, -0.2]])
    Pi = inputs.Optical(lin=(0.5, 1.0), quad=[[0.8, 0.0], [0.0, 0.4]])
    w1 = oracle.h_response1(pb, mu, mu, Ceq, dt, nt, stride)
    w2 = oracle.h_response2(pb, mu, Pi, mu, Ceq, dt, nt, nt, stride)
    for prec, tol in ((64, 1e-10), (32, 1e-4)):
        with chfpe.Handle(model, grid, depth=depth, dt=dt, precision=prec, max_batch=3,
                          p_basis=1) as h:
            h.set_equilibrium(Ceq)
            r1 = h.response1(mu, mu, nt, stride)
            r2 = h.response2(mu, Pi, mu, nt, nt, stride)
        assert np.abs(r1 - w1).max() < tol * np.abs(w1).max(), (prec, "R1")
        assert np.abs(r2 - w2).max() < tol * np.abs(w2).max(), (prec, "R2")


def test_hermite_and_grid_representations_agree_on_the_gpu():
    """One anharmonic mode with linear + square-linear coupling: R2 of the Hermite representation
    (K = 10) against the grid representation on a 96 x 96 (q, p) grid with the same q nodes, both
    on the GPU in FP64 (agreement to the grid's discretisation error, 2e-7 in the oracle pin)."""
    chfpe = _chfpe()
    model = _model(1)
    gridp = inputs.default_grid(model, [96])
    gh = inputs.Grid(nq=(96,), np=(10,), qmin=gridp.qmin, qmax=gridp.qmax, pmin=(0.0,), pmax=(1.0,))
    mu = inputs.Optical(lin=(1.0,))
    Pi = inputs.Optical(lin=(0.5,), quad=[[0.8]])
    R = {}
    for basis, grid in ((0, gridp), (1, gh)):
        with chfpe.Handle(model, grid, depth=3, dt=0.005, precision=64, max_batch=8,
                          p_basis=basis) as h:
            h.equilibrate(0, 1.0, 1)          # the sampled Boltzmann distribution
            R[basis] = h.response2(mu, Pi, mu, 8, 8, 40)
    assert np.abs(R[1] - R[0]).max() < 2e-6 * np.abs(R[0]).max()
