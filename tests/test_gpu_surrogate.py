"""The surrogate's kernels through the C ABI against the FP64 network oracle, and the surrogate
against the solver it learns from.

Tolerances:
  GEMM      BF16 operands multiply exactly in FP32; K FP32 additions then err by at most
            K u sum|a b| (u = 2^-24); the bar takes twice that.
  forward   against the oracle rounding the same operands to BF16: the sides differ by FP32
            versus FP64 accumulation (~sqrt(K) u: 1.6e-7 of the output's largest magnitude on a
            sample without flips) and by the BF16 rounding decisions that this difference flips.
            A flip moves one activation by one BF16 ulp (<= 2^-7 relative); inside the 512-wide
            linear layers it reaches every later unit.  Measured: about one flip per sample,
            half the samples off by 1e-3..3e-3 of max |y|, the others by ~1e-7.  Bars (relative
            to max |y|): median pixel error <= 1e-4, largest <= 1e-2 -- far below the O(0.1..1)
            errors of a wrong index, tap or operand.
  gradients the same flips, plus the BF16 rounding of each layer's output gradient and split-K
            atomics in FP32: bar 1e-2 relative (Frobenius) per weight or bias block, loss within
            1e-3.
"""
import numpy as np
import pytest

from oracle import surrogate_oracle as so
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


@pytest.mark.parametrize("path", ["tcgen05", "mma"])
@pytest.mark.parametrize("ta,tb", [(False, False), (False, True), (True, False), (True, True)])
@pytest.mark.parametrize("M,N,K,splits", [(1, 1, 1, 1), (70, 45, 33, 1), (130, 64, 300, 3),
                                          (64, 200, 16, 1), (5, 80, 4099, 7), (300, 200, 520, 3),
                                          (256, 512, 512, 1), (1000, 8, 288, 1)])
def test_gemm_bf16_matches_exact_products(ta, tb, M, N, K, splits, path, monkeypatch):
    """Both GEMM kernels (tcgen05 with TMEM accumulators, the default; warp-level mma.sync),
    every storage order, ragged tiles in M, N and K, split-K, and the surrogate's own shapes."""
    if path == "mma":
        monkeypatch.setenv("CHFPE_SURROGATE_GEMM", "mma")
    else:
        monkeypatch.delenv("CHFPE_SURROGATE_GEMM", raising=False)
    chfpe = _chfpe()
    rng = np.random.default_rng(M * 1000 + N * 10 + K)
    A = so.bf16_round(rng.standard_normal((M, K)))
    B = so.bf16_round(rng.standard_normal((N, K)))
    bias = rng.standard_normal(N)
    dA = torch.tensor(A.T.copy() if ta else A, dtype=torch.bfloat16, device="cuda")
    dB = torch.tensor(B.T.copy() if tb else B, dtype=torch.bfloat16, device="cuda")
    dbias = torch.tensor(bias, dtype=torch.float32, device="cuda")
    C = torch.zeros((M, N), dtype=torch.float32, device="cuda")
    lda = M if ta else K
    ldb = N if tb else K
    chfpe.surrogate_gemm(dA.data_ptr(), ta, lda, dB.data_ptr(), tb, ldb, C.data_ptr(),
                         dbias.data_ptr(), M, N, K, splits,
                         torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    want = A @ B.T + bias.astype(np.float32)
    bound = 2 * K * 2.0 ** -24 * (np.abs(A) @ np.abs(B).T) + 2.0 ** -24 * np.abs(bias)
    err = np.abs(C.cpu().numpy() - want)
    assert np.all(err <= bound + 1e-30), err.max()


def _dev(a, dtype=torch.float32):
    """A device copy made on torch's stream, complete before the library's own stream reads it."""
    t = torch.tensor(np.ascontiguousarray(a), dtype=dtype, device="cuda")
    torch.cuda.synchronize()
    return t


def _setup(B, seed):
    chfpe = _chfpe()
    p = so.init_params(seed)
    rng = np.random.default_rng(seed + 1)
    X = rng.uniform(-1, 1, (B, 12))
    T = rng.uniform(-1, 1, (B, 64, 64))
    TS = rng.uniform(-2, 2, B)
    sur = chfpe.Surrogate(max_batch=max(B, 8), seed=3)
    sur.set_params(p.astype(np.float32))
    return sur, p.astype(np.float32).astype(np.float64), X, T, TS


def test_params_roundtrip_and_count():
    chfpe = _chfpe()
    with chfpe.Surrogate(max_batch=4, seed=5) as sur:
        assert sur.nparam == so.param_count()
        p = sur.get_params()
        assert np.isfinite(p).all() and np.abs(p).max() > 0
        q = so.init_params(2).astype(np.float32)
        sur.set_params(q)
        np.testing.assert_array_equal(sur.get_params(), q)


@pytest.mark.parametrize("B", [1, 5, 67])
def test_forward_matches_oracle(B):
    sur, p, X, _, _ = _setup(B, 21)
    with sur:
        dX = _dev(X.astype(np.float32))
        Y = torch.empty((B, 4096), device="cuda")
        S = torch.empty(B, device="cuda")
        sur.infer(dX.data_ptr(), B, Y.data_ptr(), S.data_ptr())
        torch.cuda.synchronize()
        Xf = X.astype(np.float32).astype(np.float64)
        Ye, Se, _ = so.forward(p, Xf, emulate_bf16=True)
        Yx, Sx, _ = so.forward(p, Xf, emulate_bf16=False)
        y, s = Y.cpu().numpy().reshape(B, 64, 64), S.cpu().numpy()
        rel = np.abs(y - Ye) / np.abs(Ye).max()
        e_emul, e_50 = rel.max(), np.median(rel)
        e_s = np.abs(s - Se).max() / np.abs(Se).max()
        e_fp64 = np.abs(y - Yx).max() / np.abs(Yx).max()
        print(f"B={B}: image err vs BF16-emulating oracle max {e_emul:.2e} median {e_50:.2e}, "
              f"scale {e_s:.2e}; vs plain FP64 oracle {e_fp64:.2e}")
        assert e_50 <= 1e-4
        assert e_emul <= 1e-2
        assert e_s <= 1e-2
        assert e_fp64 <= 5e-2          # BF16 through 9 layers: reported, loosely bounded


def test_gradients_match_oracle():
    B = 3
    sur, p, X, T, TS = _setup(B, 33)
    with sur:
        Xf = X.astype(np.float32).astype(np.float64)
        Tf = T.astype(np.float32).astype(np.float64)
        TSf = TS.astype(np.float32).astype(np.float64)
        dX, dT, dTS = _dev(Xf), _dev(Tf), _dev(TSf)      # alive until the call returns
        loss, g = sur.gradients(dX.data_ptr(), dT.data_ptr(), dTS.data_ptr(), B, w_scale=0.5)
        L, want = so.backward(p, Xf, Tf, TSf, w_scale=0.5, emulate_bf16=True)
        _, exact = so.backward(p, Xf, Tf, TSf, w_scale=0.5, emulate_bf16=False)
        assert abs(loss - L) <= 1e-3 * L
        q = 0
        worst, worst_fp64 = 0.0, 0.0
        for (n, k), nb in so.layer_shapes():
            for a, b in ((q, q + n * k), (q + n * k, q + n * k + nb)):
                ref = want[a:b]
                e = np.linalg.norm(g[a:b] - ref) / np.linalg.norm(ref)
                worst = max(worst, e)
                worst_fp64 = max(worst_fp64, np.linalg.norm(g[a:b] - exact[a:b]) / np.linalg.norm(exact[a:b]))
                assert e <= 1e-2, (a, b, e)
            q += n * k + nb
        print(f"gradient blocks: worst rel err vs BF16-emulating oracle {worst:.2e}, "
              f"vs plain FP64 {worst_fp64:.2e}")


def test_train_step_is_adamw_of_the_gradient():
    B = 4
    sur, p, X, T, TS = _setup(B, 44)
    with sur:
        dX, dT, dTS = _dev(X), _dev(T), _dev(TS)
        _, g = sur.gradients(dX.data_ptr(), dT.data_ptr(), dTS.data_ptr(), B, w_scale=0.3)
        lr, wd = 1e-3, 0.05
        sur.train(dX.data_ptr(), dT.data_ptr(), dTS.data_ptr(), B, B, 1, lr, wd, 0.3, seed=1)
        p1 = sur.get_params().astype(np.float64)
        want, _, _ = so.adamw(p, g.astype(np.float64), 0.0, 0.0, 1, lr, wd)
        # split-K atomics reorder the gradient sums between the two calls; where a weight
        # gradient is small against its summands that moves g / (|g| + eps) slightly: bar 1e-3 of
        # the step (a missing bias correction is a factor 3.2, missing decay lr wd |p| ~ 5e-6)
        np.testing.assert_allclose(p1, want, rtol=0, atol=1e-3 * lr)


def test_training_fits_a_smooth_map():
    """1024 samples of a smooth 12 -> 64 x 64 map (separable Gaussians whose centres and widths
    follow the inputs): the loss falls by two orders of magnitude and held-out samples are fitted
    about as well as training ones."""
    chfpe = _chfpe()
    rng = np.random.default_rng(7)
    n, nt = 1024, 128
    X = rng.uniform(-1, 1, (n + nt, 12))
    t = np.linspace(-1, 1, 64)
    c1, c2 = 0.5 * X[:, 0], 0.5 * X[:, 1]
    w1, w2 = 0.3 + 0.1 * X[:, 2], 0.3 + 0.1 * X[:, 3]
    img = (np.exp(-((t[None, :, None] - c1[:, None, None]) / w1[:, None, None]) ** 2) *
           np.exp(-((t[None, None, :] - c2[:, None, None]) / w2[:, None, None]) ** 2))
    img *= (1 + 0.3 * X[:, 4])[:, None, None]
    T = img / np.abs(img).max(axis=(1, 2), keepdims=True)
    TS = 0.5 * X[:, 5]
    with chfpe.Surrogate(max_batch=128, seed=9) as sur:
        dX, dT, dTS = _dev(X[:n]), _dev(T[:n]), _dev(TS[:n])
        losses = sur.train(dX.data_ptr(), dT.data_ptr(), dTS.data_ptr(), n, 128, 60, 2e-3, 0.0,
                           1.0, seed=3)
        Y = torch.empty((nt, 4096), device="cuda")
        S = torch.empty(nt, device="cuda")
        dXt = _dev(X[n:])
        sur.infer(dXt.data_ptr(), nt, Y.data_ptr(), S.data_ptr())
        torch.cuda.synchronize()
        mse_test = np.mean((Y.cpu().numpy().reshape(nt, 64, 64) - T[n:]) ** 2)
    print(f"loss {losses[0]:.3e} -> {losses[-1]:.3e}, held-out image MSE {mse_test:.3e}")
    assert losses[-1] < 1e-2 * losses[0]
    assert mse_test < 5 * losses[-1] + 1e-3


@pytest.fixture(scope="module")
def solver_data():
    from paper_2509_25840_b300 import surrogate
    kw = dict(n_axis=10, depth=2, stride=10)      # t1, t2 up to 3.2 (dt 0.005)
    X, R, secs = surrogate.make_dataset(range(500, 500 + 96), **kw)
    return X, R, secs, kw


def test_surrogate_on_solver_data_and_fallback(solver_data):
    """Trained on 80 solver spectra, the surrogate beats the mean-spectrum predictor on 16
    held-out instances, is orders of magnitude faster than the solver, and hands parameter
    vectors outside the training ranges to the solver."""
    chfpe = _chfpe()
    from paper_2509_25840_b300 import surrogate
    X, R, secs, kw = solver_data
    ntr = 80
    with surrogate.make_surrogate(max_batch=256, seed=1) as sur:
        losses = surrogate.train(sur, X[:ntr], R[:ntr], epochs=200, batch=16, lr=2e-3)
        err = surrogate.rel_errors(surrogate.infer(sur, X[ntr:]), R[ntr:])
        T, TS = surrogate.targets(R[:ntr])
        mean_pred = np.repeat((T.mean(axis=0) * 10.0 ** TS.mean())[None], len(R) - ntr, axis=0)
        err_mean = surrogate.rel_errors(mean_pred, R[ntr:])
        rate = surrogate.inference_rate(sur, n=1024, reps=3)
        solver_rate = len(X) / secs
        x_out = inputs.SURROGATE_HI * 1.1
        x_in = X[-1]
        Rp, used = surrogate.Predictor(sur, **kw).predict(np.stack([x_in, x_out]))
        direct = surrogate.solve(x_out, **kw)
    print(f"loss {losses[0]:.3e} -> {losses[-1]:.3e}; held-out rel err median "
          f"{np.median(err):.3f} (mean predictor {np.median(err_mean):.3f}); "
          f"surrogate {rate:.3e} spectra/s vs solver {solver_rate:.2f} spectra/s")
    assert losses[-1] < 0.5 * losses[0]
    assert np.median(err) < np.median(err_mean)
    assert rate > 100 * solver_rate
    assert list(used) == [False, True]
    np.testing.assert_array_equal(Rp[1], direct)
