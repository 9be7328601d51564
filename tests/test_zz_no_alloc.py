"""The no-allocation entry point agrees with denoise_run.

denoise_run_noalloc serves callers that cannot allocate device memory (a host
framework that owns every allocation, a loop whose policy forbids cudaMalloc):
it runs the same kernels on scratch held in a fixed device array of the
library.  This file is collected last on purpose, so that a failure here comes
after every other test has run.  It builds what it needs itself and passes on
its own in a fresh process as well as after the rest of the suite.
"""

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _noalloc(N, xyz, P):
    n = xyz.shape[0]
    mask = torch.empty(n, dtype=torch.uint8, device="cuda")
    score = torch.empty(n, dtype=torch.float32, device="cuda")
    stage = torch.empty(n, dtype=torch.uint8, device="cuda")
    st = N.denoise_run_noalloc(xyz.data_ptr(), n, P.to_c(), mask.data_ptr(), score.data_ptr(), stage.data_ptr(),
                               torch.cuda.current_stream().cuda_stream)
    return st, mask, score, stage


def test_noalloc_matches_denoise_run_two_calls_in_a_row():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__
    __graft_entry__.build()
    import synth
    from paper_2512_10386_gb300 import Denoiser, Params
    from paper_2512_10386_gb300 import _native as N

    clouds = [synth.object_cloud(seed=41, n_surface=15000)[0],   # 15,750 points
              synth.object_cloud(seed=42, n_surface=6000)[0]]    # 6,300 points: a smaller second call
    assert all(len(c) <= N.DENOISE_NOALLOC_MAX_POINTS for c in clouds)
    P = Params(k=16, leaf_capacity=256)
    d = Denoiser(max_points=N.DENOISE_NOALLOC_MAX_POINTS)
    try:
        for xyz_np in clouds:                      # two calls in a row, different sizes
            xyz = torch.from_numpy(xyz_np).cuda()
            ref = d.run(xyz, P)
            st, mask, score, stage = _noalloc(N, xyz, P)
            assert st == N.DENOISE_OK, N.strerror(st)
            torch.cuda.synchronize()
            # same tolerance as the parity tests: scores within 1e-5, masks and stages identical
            sr, sg = ref.score.double().cpu().numpy(), score.double().cpu().numpy()
            scored = sr > 0
            assert np.array_equal(sr > 0, sg > 0)
            assert np.all(np.abs(sg[scored] - sr[scored]) <= 1e-5 * sr[scored])
            assert torch.equal(mask, ref.mask) and torch.equal(stage, ref.stage)
    finally:
        d.close()


def test_noalloc_spill_path_at_its_maximum_size():
    # n at the maximum, K = 64, and leaves larger than the shared-memory path: the
    # scratch array is filled to its size and the per-point spill region is used
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__
    __graft_entry__.build()
    from paper_2512_10386_gb300 import Denoiser, Params
    from paper_2512_10386_gb300 import _native as N
    n = N.DENOISE_NOALLOC_MAX_POINTS
    rng = np.random.default_rng(43)
    xyz_np = np.concatenate([rng.normal(size=(n - 1000, 3)) * 0.05,
                             rng.uniform(-1, 1, size=(1000, 3))]).astype(np.float32)
    P = Params(k=64, leaf_capacity=4096, beta=3.0)
    d = Denoiser(max_points=n)
    try:
        xyz = torch.from_numpy(xyz_np).cuda()
        for _ in range(2):
            ref = d.run(xyz, P)
            st, mask, score, stage = _noalloc(N, xyz, P)
            assert st == N.DENOISE_OK, N.strerror(st)
            torch.cuda.synchronize()
            sr, sg = ref.score.double().cpu().numpy(), score.double().cpu().numpy()
            scored = sr > 0
            assert scored.sum() > n // 2
            assert np.array_equal(sr > 0, sg > 0)
            assert np.all(np.abs(sg[scored] - sr[scored]) <= 1e-5 * sr[scored])
            assert torch.equal(mask, ref.mask) and torch.equal(stage, ref.stage)
        st = d.stats()
        assert st["n_leaves"] <= 16           # leaves of thousands of points: the spill path
    finally:
        d.close()


def test_noalloc_rejects_sizes_beyond_its_maximum():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__
    __graft_entry__.build()
    from paper_2512_10386_gb300 import Params
    from paper_2512_10386_gb300 import _native as N
    big = torch.zeros((N.DENOISE_NOALLOC_MAX_POINTS + 1, 3), device="cuda")
    st, *_ = _noalloc(N, big, Params())
    assert st == N.DENOISE_E_CAPACITY
    host = torch.zeros((10, 3))
    st = N.denoise_run_noalloc(host.data_ptr(), 10, Params().to_c(), None, None, None, 0)
    assert st == N.DENOISE_E_INVAL
