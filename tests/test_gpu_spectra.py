"""GPU parity of the spectra (Eqs. 1DIR_Raman, 2DThz_Raman, noncorrelation): libchfpe's FP64 DFT
kernels through the C ABI against the pinned oracle (oracle/spectra.py), on seeded responses and on
an R2 from the solver, at 1e-12 of the largest |I|."""
import numpy as np
import pytest

from oracle import spectra as ospec
from paper_2509_25840_b300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2509_25840_b300 import build
    build.build()


def _close(got, want, scale=None):
    """1e-12 of the largest |I|, or of `scale` -- the size of the sum's terms -- where every
    output is zero in exact arithmetic (the oracle's complex exponential then leaves ~1e-16)."""
    ref = np.abs(want).max() if scale is None else max(np.abs(want).max(), scale)
    assert np.abs(got - want).max() <= 1e-12 * ref


@pytest.mark.parametrize("N,L,eta", [(2, 2, 0.0), (37, 64, 0.0), (201, 1024, 0.1), (100, 100, 0.02)])
def test_spectrum1_matches_oracle(N, L, eta):
    from paper_2509_25840_b300 import chfpe
    R = inputs.uniform_array(17 + N, N)
    scale = 0.05 * np.abs(R).sum() * np.pi / 0.05
    _close(chfpe.spectrum1(R, 0.05, L, eta), ospec.spectrum1(R, 0.05, L, eta), scale)


@pytest.mark.parametrize("n1,n2,L1,L2,eta", [(2, 3, 4, 3, 0.0), (17, 23, 32, 64, 0.1), (64, 64, 128, 128, 0.05)])
def test_spectrum2_and_3_match_oracle(n1, n2, L1, L2, eta):
    from paper_2509_25840_b300 import chfpe
    R = inputs.uniform_array(5 + n1, n1 * n2).reshape(n1, n2)
    _close(chfpe.spectrum2(R, 0.2, L1, L2, eta), ospec.spectrum2(R, 0.2, L1, L2, eta))
    _close(chfpe.spectrum3(R, 0.2, L1, L2, eta), ospec.spectrum3(R, 0.2, L1, L2, eta))


def test_spectra_reject_bad_sizes():
    from paper_2509_25840_b300 import chfpe
    R = np.ones(8)
    for args in ((R[:1], 0.1, 4), (R, 0.1, 4), (R, 0.0, 16), (R, 0.1, 1 << 23)):
        with pytest.raises(chfpe.ChfpeError) as e:
            chfpe.spectrum1(*args)
        assert e.value.status == chfpe.EINVAL
    with pytest.raises(chfpe.ChfpeError):
        chfpe.spectrum1(R, 0.1, 16, -1.0)


def test_solver_r2_to_2d_spectrum():
    """R2 of a small two-mode model from chfpe_response2 (FP64), then its 2D spectrum on the GPU
    against the oracle's transform of the same array."""
    from paper_2509_25840_b300 import chfpe
    import oracle
    import references as ref
    model = inputs.two_mode_model()
    grid = inputs.default_grid(model, [12, 12, 12, 12])
    depth, dt, stride, nt = 2, 0.01, 20, 16
    pb = oracle.Problem(model, grid, depth)
    W = ref.hierarchy_state(ref.boltzmann_sym(model, grid), pb.M)
    mu = inputs.Optical(lin=(1.0, 1.0))
    with chfpe.Handle(model, grid, depth=depth, dt=dt, precision=64, max_batch=nt) as h:
        h.set_equilibrium(W)
        R2 = h.response2(mu, mu, mu, nt, nt, stride)
    dtau = dt * stride
    _close(chfpe.spectrum2(R2, dtau, 64, 64, 0.1), ospec.spectrum2(R2, dtau, 64, 64, 0.1))
