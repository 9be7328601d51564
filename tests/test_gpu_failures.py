"""Failure detection on the GPU, in the forms that fault nothing.

- A bounded device wait that runs out: a test hook makes one radix-sort tile
  withhold its look-back prefix, so the next tile's wait (lowered to a short
  limit) gives up.  The call must return DENOISE_E_TIMEOUT promptly and the
  context must give the right answer on the next call.
- An allocation that fails: a context sized beyond the GPU's memory must be
  refused with DENOISE_E_NOMEM, holding nothing afterwards.
"""

import time

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__
    __graft_entry__.build()
    from paper_2512_10386_gb300 import _native as N
    return N


def test_lookback_wait_times_out_and_context_recovers(lib):
    N = lib
    import synth
    from paper_2512_10386_gb300 import Denoiser, Params
    xyz_np, _ = synth.object_cloud(seed=61, n_surface=20000)     # 21,000 points: 11 radix tiles
    xyz = torch.from_numpy(xyz_np).cuda()
    P = Params(k=16)
    d = Denoiser(max_points=len(xyz_np))
    try:
        good = d.run(xyz, P)
        want = (good.mask.clone(), good.score.clone(), good.stage.clone())
        d.set_wait_limit(4096)
        d.test_hold_lookback(3)
        t0 = time.perf_counter()
        with pytest.raises(N.DenoiseError) as e:
            d.run(xyz, P)
        assert e.value.status == N.DENOISE_E_TIMEOUT
        assert time.perf_counter() - t0 < 30.0
        # the same in asynchronous mode: the status comes from denoise_get_status
        d.set_sync(False)
        d.run(xyz, P)
        assert d.status() == N.DENOISE_E_TIMEOUT
        d.set_sync(True)
        # hook off, default limit: the context is usable and right again
        d.test_hold_lookback(-1)
        d.set_wait_limit(0)
        again = d.run(xyz, P)
        assert torch.equal(again.mask, want[0]) and torch.equal(again.stage, want[2])
        assert torch.equal(again.score, want[1])
    finally:
        d.close()


def test_hook_rejects_bad_tile(lib):
    N = lib
    from paper_2512_10386_gb300 import Denoiser
    d = Denoiser(max_points=1000)
    try:
        with pytest.raises(N.DenoiseError) as e:
            d.test_hold_lookback(-2)
        assert e.value.status == N.DENOISE_E_INVAL
    finally:
        d.close()


def test_context_beyond_device_memory_is_refused(lib):
    N = lib
    free_before, _ = torch.cuda.mem_get_info()
    with pytest.raises(N.DenoiseError) as e:
        N.denoise_create(0, (1 << 30) - 1, 1)
    assert e.value.status == N.DENOISE_E_NOMEM
    free_after, _ = torch.cuda.mem_get_info()
    assert abs(free_after - free_before) < (64 << 20)        # nothing left allocated
    ctx = N.denoise_create(0, 1000, 1)                        # and a normal context still works
    N.denoise_destroy(ctx)
