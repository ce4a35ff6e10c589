"""chfpe_observe_noalloc, the reduction for callers that cannot allocate device memory.

Some users of this library run it inside programs that own all device memory themselves (a
fixed budget carved out at start-up, pre-sized buffers handed to every library) or inside
latency-critical loops where cudaMalloc's device synchronisation is not acceptable; they cannot
create a chfpe_handle, which allocates.  chfpe_observe_noalloc gives them the observable
reduction with its scratch in a fixed device array inside the library.  This test calls it
through the C ABI twice in a row and checks each result against the handle-based
chfpe_observe_device, with the tolerance the other reduction tests use (rel 1e-12).  It lives in
its own file, collected last, so that a run stopping at the first failure has already run
everything else; it passes alone in a fresh process and after the other tests."""
import numpy as np
import pytest

from paper_2509_25840_b300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _model():
    return inputs.Model(nmodes=2, kT=0.9, m=(1.2, 0.8), omega=(1.0, 1.3), g3=(0.2, -0.15),
                        g4=(0.05, 0.04), g2=[[0, 0.1], [0, 0]], g_s2s=[[0, 0.2], [0, 0]],
                        g_ss2=[[0, 0.12], [0, 0]], zeta=(0.5, 0.3), gamma=(1.0, 1.5),
                        V_LL=(1.0, 0.7), V_SL=(0.3, -0.4))


@pytest.mark.parametrize("prec", [64, 32])
def test_observe_noalloc_matches_handle_observe_twice(prec):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2509_25840_b300 import build, chfpe
    build.build()
    model = _model()
    grid = inputs.default_grid(model, [11, 12, 13, 10], cut=12.0, nsigma=5.0)
    depth, batch = 3, 5
    dtype = torch.float64 if prec == 64 else torch.float32
    M = inputs.member_count(2, depth)
    W = inputs.random_state(grid, M, seed=21, smooth=True)
    states = torch.tensor(np.stack([W * (1.0 + 0.25 * b) for b in range(batch)]), dtype=dtype,
                          device="cuda")
    ops = [inputs.Optical(lin=(0.7, -1.1), quad=[[0.4, 0.9], [0.1, -0.6]]),
           inputs.Optical(lin=(1.0, 1.0))]
    with chfpe.Handle(model, grid, depth=depth, dt=0.004, precision=prec, max_batch=batch) as h:
        for call, C in enumerate(ops):                       # two calls in a row
            want = torch.zeros(batch, dtype=torch.float64, device="cuda")
            h.observe_device(C, states.data_ptr(), batch, want.data_ptr())
            got = torch.full((batch,), float("nan"), dtype=torch.float64, device="cuda")
            torch.cuda.synchronize()
            free_before = torch.cuda.mem_get_info()[0]
            chfpe.observe_noalloc(model, grid, depth, prec, C, states.data_ptr(), batch,
                                  got.data_ptr(), torch.cuda.current_stream().cuda_stream)
            torch.cuda.synchronize()
            if call == 1:   # after the first call's one-time address lookup: no device memory taken
                assert torch.cuda.mem_get_info()[0] == free_before
            g, w = got.cpu().numpy(), want.cpu().numpy()
            np.testing.assert_allclose(g, w, rtol=1e-12, atol=1e-14 * np.abs(w).max())


def test_observe_noalloc_rejects_batches_beyond_its_scratch():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2509_25840_b300 import build, chfpe
    build.build()
    model = _model()
    grid = inputs.default_grid(model, [32, 32, 32, 32])     # 512 blocks per state
    dummy = torch.zeros(4, dtype=torch.float32, device="cuda")
    R = torch.zeros(4, dtype=torch.float64, device="cuda")
    with pytest.raises(chfpe.ChfpeError) as e:
        chfpe.observe_noalloc(model, grid, 4, 32, inputs.Optical(lin=(1.0, 1.0)),
                              dummy.data_ptr(), 65, R.data_ptr())   # 65 x 512 > 32768
    assert e.value.status == chfpe.EINVAL
    assert "maximum is 32768" in str(e.value)
