"""GPU parity: libchfpe (through its C ABI) against the FP64 oracle on the same seeded inputs.

Tolerances: FP64 path 1e-10 (normalised L-infinity on responses, relative to max |oracle| on
operator outputs); FP32 path 1e-4 on normalised responses.  Operator-level FP32 checks compare
against the oracle evaluated on the float-rounded input, so only arithmetic rounding differs; the
bound there is a few float ulps times the size of the largest single term."""
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


def _dtype(prec):
    return torch.float64 if prec == 64 else torch.float32


def _rounded(W, prec):
    return W if prec == 64 else W.astype(np.float32).astype(np.float64)


def _model(d):
    return inputs.Model(nmodes=d, kT=0.9, m=(1.2, 0.8, 1.0), omega=(1.0, 1.3, 0.7),
                        g3=(0.2, -0.15, 0.1), g4=(0.05, 0.04, 0.06),
                        g2=[[0, 0.1, 0.05], [0, 0, -0.1]], g_s2s=[[0, 0.2, 0.1], [0, 0, 0.1]],
                        g_ss2=[[0, 0.12, 0.1], [0, 0, 0.05]], zeta=(0.5, 0.3, 0.4),
                        gamma=(1.0, 1.5, 0.8), V_LL=(1.0, 0.7, 0.9), V_SL=(0.3, -0.4, 0.2))


# ragged per-axis sizes: several thread blocks plus a tail in every case; a fastest axis (p_d)
# that is a multiple of 4 runs the vectorised stage kernel (float4 / double2), others the scalar
CASES = [
    (1, [37, 45], 5),
    (1, [37, 44], 5),
    (1, [64, 64], 8),
    (2, [9, 11, 13, 15], 4),
    (2, [9, 11, 13, 12], 4),
    (2, [12, 10, 14, 8], 5),
    (3, [7, 8, 9, 7, 8, 9], 2),
    (3, [7, 8, 9, 7, 9, 8], 2),
    (3, [7, 7, 8, 8, 7, 8], 3),
]


def _setup(d, n, depth, prec, max_batch=1, dt=0.004):
    chfpe = _chfpe()
    model = _model(d)
    grid = inputs.default_grid(model, n, cut=12.0, nsigma=5.0)
    h = chfpe.Handle(model, grid, depth=depth, dt=dt, precision=prec, max_batch=max_batch)
    pb = oracle.Problem(model, grid, depth)
    return model, grid, h, pb


@pytest.mark.parametrize("prec", [64, 32])
@pytest.mark.parametrize("d,n,depth", CASES)
def test_rhs_matches_oracle(d, n, depth, prec):
    model, grid, h, pb = _setup(d, n, depth, prec)
    W = _rounded(inputs.random_state(grid, pb.M, seed=100 + d, smooth=False), prec)
    want = oracle.rhs(pb, W)
    x = torch.tensor(W, dtype=_dtype(prec), device="cuda")
    y = torch.empty_like(x)
    h.rhs_device(x.data_ptr(), y.data_ptr(), 1)
    got = y.double().cpu().numpy()
    scale = np.abs(want).max()
    tol = 1e-13 if prec == 64 else 3e-6
    assert np.abs(got - want).max() <= tol * scale


@pytest.mark.parametrize("prec", [64, 32])
@pytest.mark.parametrize("d,n,depth", CASES[::2])
def test_insert_and_observe_match_oracle(d, n, depth, prec):
    model, grid, h, pb = _setup(d, n, depth, prec)
    W = _rounded(inputs.random_state(grid, pb.M, seed=7, smooth=True), prec)
    X = inputs.Optical(lin=(0.7, -1.1, 0.4), quad=[[0.4, 0.9, 0.1], [0.1, -0.6, 0.2], [0.3, 0.0, 0.5]])
    want = oracle.insert(pb, X, W)
    x = torch.tensor(W, dtype=_dtype(prec), device="cuda")
    y = torch.empty_like(x)
    h.insert_device(X, x.data_ptr(), y.data_ptr(), 1)
    got = y.double().cpu().numpy()
    tol = 1e-13 if prec == 64 else 3e-6
    assert np.abs(got - want).max() <= tol * np.abs(want).max()
    # observable: FP64 accumulation on both sides of the same (rounded) values
    Rd = torch.zeros(2, dtype=torch.float64, device="cuda")
    xx = torch.stack([x, 2.0 * x])
    h.observe_device(X, xx.data_ptr(), 2, Rd.data_ptr())
    r = Rd.cpu().numpy()
    r0 = oracle.observe(pb, X, W)
    assert r[0] == pytest.approx(r0, rel=1e-12, abs=1e-14)
    assert r[1] == pytest.approx(2 * r0, rel=1e-12, abs=1e-14)


@pytest.mark.parametrize("prec", [64, 32])
@pytest.mark.parametrize("d,n,depth", [CASES[0], CASES[1], CASES[3], CASES[4], CASES[6], CASES[7]])
def test_rk4_matches_oracle_and_batches_are_independent(d, n, depth, prec):
    model, grid, h, pb = _setup(d, n, depth, prec, max_batch=3)
    W = _rounded(inputs.random_state(grid, pb.M, seed=5, smooth=True), prec)
    nsteps = 25
    want = oracle.rk4(pb, W, 0.004, nsteps)
    x = torch.tensor(np.stack([W, 0.5 * W, W]), dtype=_dtype(prec), device="cuda")
    h.rk4_device(x.data_ptr(), 3, nsteps)
    got = x.double().cpu().numpy()
    tol = 1e-12 if prec == 64 else 2e-5
    scale = np.abs(want).max()
    assert np.abs(got[0] - want).max() <= tol * scale
    assert np.abs(got[1] - 0.5 * want).max() <= tol * scale
    assert np.array_equal(got[0], got[2])           # batch slots do not interact


def _norm_err(got, want):
    return np.abs(got - want).max() / np.abs(want).max()


@pytest.mark.parametrize("prec,tol", [(64, 1e-10), (32, 1e-4)])
def test_response1_one_mode_matches_oracle(prec, tol):
    wl = inputs.one_mode_64(nt=201, stride=2)
    chfpe = _chfpe()
    pb = oracle.Problem(wl.model, wl.grid, wl.depth)
    Weq, _, _ = oracle.equilibrate(pb, wl.dt, 200, 0.0, 100)
    want = oracle.response1(pb, wl.A, wl.C, _rounded(Weq, prec), wl.dt, wl.nt1, wl.stride)
    with chfpe.Handle(wl.model, wl.grid, depth=wl.depth, dt=wl.dt, precision=prec) as h:
        h.set_equilibrium(Weq)
        got = h.response1(wl.A, wl.C, wl.nt1, wl.stride)
    assert _norm_err(got, want) < tol


def _workload_optics(d):
    """The optics of the named workloads: mu = q1 + q2 (two modes); water-like mu, Pi (three)."""
    if d == 2:
        mu = inputs.Optical(lin=(1.0, 1.0))
        return mu, mu, mu
    mu, Pi = inputs.three_mode_optics()
    return mu, Pi, mu


@pytest.mark.parametrize("d,n,depth,dt,stride,nt", [
    (2, [12, 11, 12, 12], 4, 0.01, 50, 4),     # vectorised stage kernel, t1, t2 <= 1.5
    (2, [12, 12, 12, 13], 3, 0.01, 50, 4),     # scalar stage kernel
    (3, [7, 7, 8, 8, 7, 8], 2, 0.004, 20, 3),  # water-like TRT optics, vectorised
])
def test_response2_matches_oracle(d, n, depth, dt, stride, nt):
    """Both precisions against one oracle run on the float-rounded equilibrium: FP64 to 1e-10,
    FP32 to 1e-4 of max|R2| (the response has developed: t1, t2 up to (nt-1) stride dt)."""
    chfpe = _chfpe()
    model = _model(d)
    grid = inputs.default_grid(model, n, cut=12.0, nsigma=5.0)
    pb = oracle.Problem(model, grid, depth)
    Weq = _rounded(ref.hierarchy_state(ref.boltzmann_sym(model, grid), pb.M), 32)
    A, B, C = _workload_optics(d)
    want = oracle.response2(pb, A, B, C, Weq, dt, nt, nt, stride)
    for prec, tol in ((64, 1e-10), (32, 1e-4)):
        with chfpe.Handle(model, grid, depth=depth, dt=dt, precision=prec, max_batch=3) as h:
            h.set_equilibrium(Weq)
            got = h.response2(A, B, C, nt, nt, stride)
        assert _norm_err(got, want) < tol, (prec, _norm_err(got, want))


def test_response2_strong_cancellation_fp64():
    """Two modes with the water-like optics on a coarse 4D grid: the linear parts of mu and Pi
    build branch states ~1e3 x larger than R2 that cancel in the observable, so FP32 rounding
    (u = 6e-8) shows at ~2e-4 of max|R2| there; the FP64 path holds 1e-10."""
    chfpe = _chfpe()
    model = _model(2)
    grid = inputs.default_grid(model, [14, 12, 16, 13], cut=12.0, nsigma=5.0)
    pb = oracle.Problem(model, grid, 3)
    Weq = ref.hierarchy_state(ref.boltzmann_sym(model, grid), pb.M)
    mu, Pi = inputs.three_mode_optics()
    dt, nt1, nt2, stride = 0.004, 5, 4, 6
    want = oracle.response2(pb, mu, Pi, mu, Weq, dt, nt1, nt2, stride)
    with chfpe.Handle(model, grid, depth=3, dt=dt, precision=64, max_batch=3) as h:
        h.set_equilibrium(Weq)
        got = h.response2(mu, Pi, mu, nt1, nt2, stride)
    assert _norm_err(got, want) < 1e-10


def test_response2_chunking_is_bitwise_invariant():
    chfpe = _chfpe()
    model = _model(2)
    grid = inputs.default_grid(model, [11, 12, 13, 10], cut=12.0, nsigma=5.0)
    pb = oracle.Problem(model, grid, 2)
    Weq = ref.hierarchy_state(ref.boltzmann_sym(model, grid), pb.M)
    mu, Pi = inputs.three_mode_optics()
    out = []
    for mb in (1, 3, 7):
        with chfpe.Handle(model, grid, depth=2, dt=0.004, precision=64, max_batch=mb) as h:
            h.set_equilibrium(Weq)
            out.append(h.response2(Pi, mu, mu, 7, 5, 4))
    assert np.array_equal(out[0], out[1]) and np.array_equal(out[0], out[2])


def test_equilibrate_matches_oracle():
    chfpe = _chfpe()
    model = _model(2)
    grid = inputs.default_grid(model, [12, 11, 13, 12], cut=12.0, nsigma=5.0)
    pb = oracle.Problem(model, grid, 2)
    want, steps_o, res_o = oracle.equilibrate(pb, 0.004, 300, 0.0, 100)
    for prec in (64, 32):
        with chfpe.Handle(model, grid, depth=2, dt=0.004, precision=prec) as h:
            steps, res = h.equilibrate(300, 0.0, 100)
            got = h.get_equilibrium()
        assert steps == steps_o == 300
        assert res == pytest.approx(res_o, rel=1e-9)
        tol = 1e-12 if prec == 64 else 1e-7      # FP32 only rounds the FP64 result once
        assert np.abs(got - want).max() <= tol * np.abs(want).max()


def test_state_roundtrip_save_load_and_errors(tmp_path):
    chfpe = _chfpe()
    wl = inputs.one_mode_64(nt=3)
    with chfpe.Handle(wl.model, wl.grid, depth=wl.depth, dt=wl.dt, precision=64) as h:
        with pytest.raises(chfpe.ChfpeError) as e:
            h.response1(wl.A, wl.C, 3, 1)
        assert e.value.status == chfpe.ESTATE
        W = inputs.random_state(wl.grid, h.members, seed=3)
        h.set_equilibrium(W)
        assert np.array_equal(h.get_equilibrium(), W)
        p = str(tmp_path / "eq.bin")
        h.save_equilibrium(p)
        h.set_equilibrium(2 * W)
        h.load_equilibrium(p)
        assert np.array_equal(h.get_equilibrium(), W)
        h.set_state(W)
        h.propagate(3)
        pb = oracle.Problem(wl.model, wl.grid, wl.depth)
        np.testing.assert_allclose(h.get_state(), oracle.rk4(pb, W, wl.dt, 3), rtol=0,
                                   atol=1e-12 * np.abs(W).max())
        # a poisoned equilibrium is reported, not propagated silently
        bad = W.copy()
        bad[0, 10, 10] = np.nan
        h.set_equilibrium(bad)
        with pytest.raises(chfpe.ChfpeError) as e:
            h.response1(wl.A, wl.C, 3, 1)
        assert e.value.status == chfpe.EUNSTABLE


@pytest.mark.parametrize("prec", [64, 32])
def test_vector_and_scalar_stage_kernels_agree(prec, monkeypatch):
    """The vectorised stage kernel (p_d a multiple of the vector width) against the scalar one
    on the same handle parameters: same arithmetic per cell, possibly another FMA grouping."""
    model = _model(2)
    grid = inputs.default_grid(model, [10, 9, 12, 16], cut=12.0, nsigma=5.0)
    W = _rounded(inputs.random_state(grid, 15, seed=9, smooth=False), prec)
    outs = []
    for scalar in ("0", "1"):
        monkeypatch.setenv("CHFPE_SCALAR_STAGE", scalar)
        chfpe = _chfpe()
        with chfpe.Handle(model, grid, depth=4, dt=0.004, precision=prec) as h:
            x = torch.tensor(W, dtype=_dtype(prec), device="cuda")
            y = torch.empty_like(x)
            h.rhs_device(x.data_ptr(), y.data_ptr(), 1)
            outs.append(y.double().cpu().numpy())
    scale = np.abs(outs[0]).max()
    assert np.abs(outs[0] - outs[1]).max() <= (1e-14 if prec == 64 else 1e-6) * scale


TUNED_CASES = [(1, [40, 48], 5), (2, [9, 11, 12, 16], 4), (2, [9, 11, 13, 12], 2),
               (3, [7, 8, 9, 7, 8, 12], 2)]


@pytest.mark.parametrize("variant", range(18))
@pytest.mark.parametrize("d,n,depth", TUNED_CASES)
def test_every_stage_launch_shape_matches_oracle(d, n, depth, variant, monkeypatch):
    """Each launch shape the autotuner can pick (forced through CHFPE_STAGE_VARIANT), FP32,
    against the oracle's RHS: same bar as the other FP32 RHS cases."""
    monkeypatch.setenv("CHFPE_STAGE_VARIANT", str(variant))
    model, grid, h, pb = _setup(d, n, depth, 32)
    with h:
        assert h.stage_tuning()[0] == variant
        W = _rounded(inputs.random_state(grid, pb.M, seed=300 + d, smooth=False), 32)
        want = oracle.rhs(pb, W)
        x = torch.tensor(W, dtype=torch.float32, device="cuda")
        y = torch.empty_like(x)
        h.rhs_device(x.data_ptr(), y.data_ptr(), 1)
        got = y.double().cpu().numpy()
    assert np.abs(got - want).max() <= 3e-6 * np.abs(want).max()


@pytest.mark.parametrize("variant", [3, 15, 16])
def test_bench_launch_shapes_match_oracle_at_full_size(variant, monkeypatch):
    """The launch shapes the autotuner picks on the benchmark workload, on that workload itself:
    its model, its 32^4 grid and domain, depth 4 (15 members), FP32, against the oracle's RHS of
    the same seeded state (every boundary case of every axis)."""
    monkeypatch.setenv("CHFPE_STAGE_VARIANT", str(variant))
    chfpe = _chfpe()
    wl = inputs.two_mode_32(nt=2)
    pb = oracle.Problem(wl.model, wl.grid, wl.depth)
    W = _rounded(inputs.random_state(wl.grid, pb.M, seed=77, smooth=False), 32)
    want = oracle.rhs(pb, W)
    with chfpe.Handle(wl.model, wl.grid, depth=wl.depth, dt=wl.dt, precision=32) as h:
        assert h.stage_tuning()[0] == variant
        x = torch.tensor(W, dtype=torch.float32, device="cuda")
        y = torch.empty_like(x)
        h.rhs_device(x.data_ptr(), y.data_ptr(), 1)
        got = y.double().cpu().numpy()
    assert np.abs(got - want).max() <= 3e-6 * np.abs(want).max()


def test_autotuner_times_the_shapes_and_keeps_the_fastest(monkeypatch):
    monkeypatch.delenv("CHFPE_STAGE_VARIANT", raising=False)
    model = _model(2)
    grid = inputs.default_grid(model, [16, 16, 16, 16], cut=12.0, nsigma=5.0)
    chfpe = _chfpe()
    with chfpe.Handle(model, grid, depth=4, dt=0.004, precision=32, max_batch=4) as h:
        v, us = h.stage_tuning()
    print(f"stage shapes (us per launch, 4 states of 16^4 x 15): {np.round(us, 1)} -> {v}")
    assert len(us) == 18
    assert np.all(us > 0)
    assert us[v] <= us.min() / 0.98 + 1e-9          # within the 2 % preference for earlier shapes
    assert all(us[w] >= 0.98 * us[v] for w in range(v))
    # a 3-mode handle has no bulk-copy shape: not timed
    model3 = _model(3)
    grid3 = inputs.default_grid(model3, [8, 8, 8, 8, 8, 8], cut=12.0, nsigma=5.0)
    with chfpe.Handle(model3, grid3, depth=2, dt=0.004, precision=32, max_batch=2) as h:
        v3, us3 = h.stage_tuning()
    others = [w for w in range(18) if w not in (4, 5)]
    assert np.all(us3[4:6] == -1) and v3 not in (4, 5) and np.all(us3[others] > 0)
    with chfpe.Handle(model, grid, depth=4, dt=0.004, precision=64) as h:   # not tuned
        v, us = h.stage_tuning()
    assert v == 0 and np.all(us == -1)


@pytest.mark.parametrize("prec", [64, 32])
def test_persistent_propagation_matches_launch_per_stage(prec, monkeypatch):
    """The one-launch persistent R1 (grid barriers between stages, in-kernel reduction) against
    the launch-per-stage path on the one-mode workload and a small two-mode case."""
    chfpe = _chfpe()
    wl = inputs.one_mode_64(nt=201, stride=2)
    W = ref.hierarchy_state(ref.boltzmann_sym(wl.model, wl.grid), inputs.member_count(1, wl.depth))
    m2 = _model(2)
    g2 = inputs.default_grid(m2, [9, 11, 12, 16], cut=12.0, nsigma=5.0)
    W2 = ref.hierarchy_state(ref.boltzmann_sym(m2, g2), inputs.member_count(2, 4))
    mu2 = inputs.Optical(lin=(1.0, 0.5), quad=[[0.2, 0.1], [0.0, -0.1]])
    for model, grid, depth, dt, Weq, A, C, nt, stride in (
            (wl.model, wl.grid, wl.depth, wl.dt, W, wl.A, wl.C, 201, 2),
            (m2, g2, 4, 0.004, W2, mu2, mu2, 12, 5)):
        got = {}
        for persistent in ("1", "0"):
            monkeypatch.setenv("CHFPE_PERSISTENT", persistent)
            with chfpe.Handle(model, grid, depth=depth, dt=dt, precision=prec) as h:
                h.set_equilibrium(Weq)
                got[persistent] = h.response1(A, C, nt, stride)
                launches = h.stats()["kernel_launches"]
            if persistent == "1":
                assert launches < 20             # set-up, insertion, one persistent launch
        scale = np.abs(got["0"]).max()
        tol = 1e-12 if prec == 64 else 1e-6
        assert np.abs(got["1"] - got["0"]).max() <= tol * scale


def test_persistent_barrier_error_reports_timeout_and_recovers(monkeypatch):
    """The grid barrier's error path: with the error word set before the launch (as if a wait had
    given up) every block leaves at its first barrier, the call returns CHFPE_ETIMEOUT, and the
    next call on the same handle runs normally."""
    chfpe = _chfpe()
    wl = inputs.one_mode_64(nt=21, stride=2)
    W = ref.hierarchy_state(ref.boltzmann_sym(wl.model, wl.grid), inputs.member_count(1, wl.depth))
    monkeypatch.setenv("CHFPE_PERSISTENT", "1")
    with chfpe.Handle(wl.model, wl.grid, depth=wl.depth, dt=wl.dt, precision=64) as h:
        h.set_equilibrium(W)
        want = h.response1(wl.A, wl.C, 21, 2)
        monkeypatch.setenv("CHFPE_TEST_PRESET_ERROR", "1")
        with pytest.raises(chfpe.ChfpeError) as e:
            h.response1(wl.A, wl.C, 21, 2)
        assert e.value.status == chfpe.ETIMEOUT
        monkeypatch.delenv("CHFPE_TEST_PRESET_ERROR")
        again = h.response1(wl.A, wl.C, 21, 2)
    np.testing.assert_array_equal(again, want)


def test_response2_bench_workload_launch_per_stage_matches_oracle():
    """The benchmark workload itself (two_mode_32: its model, 32^4 grid and domain, depth 4,
    dt 0.005, stride 40, A = B = C = q1 + q2) through chfpe_response2 on the branch the bench
    takes: stage timing on, which selects one launch per RK4 stage (no CUDA graph, no persistent
    kernel), from the float-rounded sampled Boltzmann equilibrium (Eq. 2Dresponse).

    * FP64 build against the oracle on nt1 = nt2 = 3 (t <= 0.4): 1e-10 of max|R2|.
    * FP32 against that FP64 build on 8 x 8 samples (t <= 1.4): 1e-4 of max|R2|.
    * FP32 against the oracle on the 3 x 3 window, normalised by max|R2| of the 8 x 8 window:
      1e-4.  (Over t <= 0.4 alone R2 has not developed -- max|R2| is 1 % of its value over the
      spectrum -- and FP32 rounding of the O(1) branch states shows at ~1e-4 of that small
      maximum; the normalised error of the response is taken over its t-grid.)"""
    chfpe = _chfpe()
    wl = inputs.two_mode_32(nt=3)
    pb = oracle.Problem(wl.model, wl.grid, wl.depth)
    Weq = _rounded(oracle.boltzmann(pb), 32)
    want = oracle.response2(pb, wl.A, wl.B, wl.C, Weq, wl.dt, 3, 3, wl.stride)
    got = {}
    for prec in (64, 32):
        with chfpe.Handle(wl.model, wl.grid, depth=wl.depth, dt=wl.dt, precision=prec,
                          max_batch=8) as h:
            h.set_equilibrium(Weq)
            h.stats_reset(time_stages=True)
            small = h.response2(wl.A, wl.B, wl.C, 3, 3, wl.stride)
            st = h.stats()
            # chain 2 x 40 steps, then one burst of 2 x 40 steps for the 3 branches
            assert st["stage_launches"] == 4 * (2 * wl.stride + 2 * wl.stride)
            got[prec] = (small, h.response2(wl.A, wl.B, wl.C, 8, 8, wl.stride))
    assert _norm_err(got[64][0], want) < 1e-10, _norm_err(got[64][0], want)
    assert _norm_err(got[32][1], got[64][1]) < 1e-4, _norm_err(got[32][1], got[64][1])
    scale = np.abs(got[64][1]).max()
    assert np.abs(got[32][0] - want).max() / scale < 1e-4


def test_response2_two_mode_long_times_matches_oracle():
    """The benchmark's model (two coupled anharmonic modes, LL + SL) on a reduced grid out to
    t1, t2 = 6 (11 x 11 samples at dtau = 0.6): FP64 to 1e-10 and FP32 to 1e-4 of max|R2|."""
    chfpe = _chfpe()
    model = inputs.two_mode_model()
    grid = inputs.default_grid(model, [10, 11, 12, 12])
    depth, dt, stride, nt = 4, 0.005, 120, 11
    pb = oracle.Problem(model, grid, depth)
    Weq = _rounded(oracle.boltzmann(pb), 32)
    mu = inputs.Optical(lin=(1.0, 1.0))
    want = oracle.response2(pb, mu, mu, mu, Weq, dt, nt, nt, stride)
    for prec, tol in ((64, 1e-10), (32, 1e-4)):
        with chfpe.Handle(model, grid, depth=depth, dt=dt, precision=prec, max_batch=6) as h:
            h.set_equilibrium(Weq)
            got = h.response2(mu, mu, mu, nt, nt, stride)
        assert _norm_err(got, want) < tol, (prec, _norm_err(got, want))


@pytest.mark.parametrize("mode", ["persistent", "graphs", "per_stage"])
def test_sample_device_matches_oracle(mode, monkeypatch):
    """chfpe_sample_device on caller-owned states, under each dispatch of the sampling loop:
    sample k of state b equals the oracle's observable after k * stride RK4 steps of that state."""
    chfpe = _chfpe()
    env = {"persistent": ("1", "-1"), "graphs": ("0", "1"), "per_stage": ("0", "0")}[mode]
    monkeypatch.setenv("CHFPE_PERSISTENT", env[0])
    monkeypatch.setenv("CHFPE_GRAPHS", env[1])
    model = _model(2)
    grid = inputs.default_grid(model, [9, 11, 12, 16], cut=12.0, nsigma=5.0)
    depth, dt, stride, ns, batch = 4, 0.004, 5, 6, 3
    pb = oracle.Problem(model, grid, depth)
    W = [inputs.random_state(grid, pb.M, seed=40 + b, smooth=True) for b in range(batch)]
    C = inputs.Optical(lin=(0.8, -0.5), quad=[[0.3, 0.1], [0.1, -0.2]])
    want = np.zeros((batch, ns))
    for b in range(batch):
        w = W[b]
        for k in range(ns):
            want[b, k] = oracle.observe(pb, C, w)
            if k + 1 < ns:
                w = oracle.rk4(pb, w, dt, stride)
    with chfpe.Handle(model, grid, depth=depth, dt=dt, precision=64, max_batch=batch) as h:
        x = torch.tensor(np.stack(W), dtype=torch.float64, device="cuda")
        R = torch.zeros((batch, ns + 2), dtype=torch.float64, device="cuda")
        h.sample_device(C, x.data_ptr(), batch, ns, stride, R.data_ptr(), ns + 2)
        got = R.cpu().numpy()
        launches = h.stats()["kernel_launches"]
        with pytest.raises(chfpe.ChfpeError) as e:            # batch beyond the branch arenas
            h.sample_device(C, x.data_ptr(), batch + 1, ns, stride, R.data_ptr(), ns + 2)
        assert e.value.status == chfpe.EINVAL
    if mode == "persistent":
        assert launches < 20
    np.testing.assert_allclose(got[:, :ns], want, rtol=1e-11, atol=1e-13 * np.abs(want).max())
    assert np.all(got[:, ns:] == 0)                         # ld > nsamples: the gap untouched


@pytest.mark.parametrize("d,n,depth,dt,stride,n2,nt,mb", [
    (1, [37, 44], 4, 0.005, 20, 30, 5, 2),            # chunks 2 + 2 + 1; scalar stage kernel
    (2, [12, 11, 12, 12], 3, 0.01, 25, 40, 4, 4),     # vectorised stage kernel
])
def test_response3_matches_oracle(d, n, depth, dt, stride, n2, nt, mb):
    """Eq. 3Dresponse at one waiting time: both precisions against the oracle (which propagates
    every t1 branch on its own): FP64 1e-10, FP32 1e-4 of max|R3|."""
    chfpe = _chfpe()
    model = _model(d)
    grid = inputs.default_grid(model, n, cut=12.0, nsigma=5.0)
    pb = oracle.Problem(model, grid, depth)
    Weq = _rounded(ref.hierarchy_state(ref.boltzmann_sym(model, grid), pb.M), 32)
    mu = inputs.Optical(lin=(1.0, 0.6, 0.3), quad=[[0.3, 0.1, 0.0], [0.1, -0.2, 0.0], [0, 0, 0.1]])
    Pi = inputs.Optical(lin=(0.5, 1.0, 0.2), quad=[[0.8, 0.0, 0.1], [0.0, 0.4, 0.0], [0.1, 0, 0.2]])
    want = oracle.response3(pb, mu, Pi, Pi, mu, Weq, dt, nt, n2, nt, stride)
    for prec, tol in ((64, 1e-10), (32, 1e-4)):
        with chfpe.Handle(model, grid, depth=depth, dt=dt, precision=prec, max_batch=mb) as h:
            h.set_equilibrium(Weq)
            got = h.response3(mu, Pi, Pi, mu, nt, n2, nt, stride)
        assert _norm_err(got, want) < tol, (prec, _norm_err(got, want))


def test_alu_peak_microbenchmark():
    """chfpe_alu_peak: positive FMA rates, FP32 above FP64, both below a generous physical bound
    (2 flops x 148 SMs x 256 lanes x 2.1 GHz)."""
    chfpe = _chfpe()
    p64, p32 = chfpe.alu_peak(64), chfpe.alu_peak(32)
    bound = 2 * 148 * 256 * 2.1e9
    assert 0 < p64 < p32 < bound, (p64, p32)
    with pytest.raises(chfpe.ChfpeError):
        chfpe.alu_peak(16)
