"""Autotuner of the batched path, and oracle parity on the batching workload's frames.

The tuner picks a leaf capacity and the leaf kernel's CTAs per SM by timing;
whatever it picks, the batched result must equal per-frame runs at the same
capacity, and the per-frame result must match the FP64 oracle (bit-exact gates
and neighbour sets, scores within 1e-5) at every capacity it may choose.
"""

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

from gpu_helpers import compare_with_oracle, oracle_params, to_np  # noqa: E402


@pytest.fixture(scope="module")
def env():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__
    __graft_entry__.build()
    import oracle
    return oracle


def test_tuned_batch_equals_per_frame(env, tmp_path):
    import synth
    from paper_2512_10386_gb300 import Denoiser, Params
    from paper_2512_10386_gb300.autotune import tune_batch
    frames = [synth.lidar_frame(2000 + i)[0] for i in range(4)]
    offs = np.cumsum([0] + [len(f) for f in frames]).tolist()
    xyz = torch.from_numpy(np.concatenate(frames)).cuda()
    P = Params(k=24)
    cache = str(tmp_path / "tune.json")
    best = tune_batch(xyz, offs, P, capacities=(192, 512), ctas=(0, 2), smem_points=(0, 128), threads=(0, 64),
                      reps=2, cache_path=cache)
    assert best["leaf_capacity"] in (192, 512) and best["leaf_ctas_per_sm"] in (0, 2)
    assert best["leaf_smem_points"] in (0, 128) and best["leaf_threads"] in (0, 64)
    assert len(best["table"]) == 12  # 2 capacities x (2 CTA counts x 2 smem sizes at 128 threads + 2 at 64)
    assert tune_batch(xyz, offs, P, cache_path=cache)["leaf_capacity"] == best["leaf_capacity"]  # cached
    import dataclasses
    Pt = dataclasses.replace(P, leaf_capacity=best["leaf_capacity"])
    d = Denoiser(max_points=offs[-1], max_frames=len(frames))
    d.set_tuning(best["leaf_ctas_per_sm"], best["leaf_smem_points"], best["leaf_threads"])
    d.set_graphs(True)
    rb = d.run_batch(xyz, offs, Pt)
    d.set_graphs(False)
    for f in range(len(frames)):
        a, b = offs[f], offs[f + 1]
        rs = d.run(xyz[a:b], Pt)
        assert torch.equal(rb.mask[a:b], rs.mask) and torch.equal(rb.score[a:b], rs.score)
    d.close()


@pytest.mark.parametrize("cap", [128, 256, 512])
def test_lidar_frame_parity_at_tunable_capacities(env, cap):
    import synth
    from paper_2512_10386_gb300 import Denoiser, Params
    xyz, _ = synth.lidar_frame(1000)
    P = Params(k=24, leaf_capacity=cap)
    d = Denoiser(max_points=len(xyz))
    g = to_np(d.run_debug(torch.from_numpy(xyz).cuda(), P))
    d.close()
    r = env.denoise(xyz, oracle_params(P), debug=True)
    stats = compare_with_oracle(g, r, P)
    print(f"lidar frame cap {cap}:", stats)


@pytest.mark.parametrize("smem_points", [64, 256])
def test_results_do_not_depend_on_the_shared_memory_leaf_size(env, smem_points):
    """Leaves above leaf_smem_points take the kernel's global-memory path:
    bit-identical results to the default (every leaf in shared memory)."""
    import synth
    from paper_2512_10386_gb300 import Denoiser, Params
    xyz, _ = synth.superquadric_scan(seed=3, n_surface=120_000)
    t = torch.from_numpy(xyz).cuda()
    P = Params(k=32, leaf_capacity=512)
    d = Denoiser(max_points=len(xyz))
    ref = d.run(t, P)
    ref = [x.clone() for x in (ref.mask, ref.score, ref.stage)]
    d.set_tuning(0, smem_points)
    got = d.run(t, P)
    for a, b in zip(ref, (got.mask, got.score, got.stage)):
        assert torch.equal(a, b)
    d.close()


@pytest.mark.parametrize("threads", [64, 128])
def test_results_do_not_depend_on_the_leaf_cta_size(env, threads):
    """64- or 128-thread leaf CTAs: bit-identical results (LiDAR frame, K = 24,
    capacity 256, and the dense scan subset at capacity 512)."""
    import synth
    from paper_2512_10386_gb300 import Denoiser, Params
    from paper_2512_10386_gb300 import _native as N
    for xyz, P in ((synth.lidar_frame(1001)[0], Params(k=24, leaf_capacity=256)),
                   (synth.superquadric_scan(seed=4, n_surface=80_000)[0], Params(k=32, leaf_capacity=512))):
        t = torch.from_numpy(xyz).cuda()
        d = Denoiser(max_points=len(xyz))
        ref = d.run(t, P)
        ref = [x.clone() for x in (ref.mask, ref.score, ref.stage)]
        d.set_tuning(0, 0, threads)
        got = d.run(t, P)
        for a, b in zip(ref, (got.mask, got.score, got.stage)):
            assert torch.equal(a, b)
        with pytest.raises(N.DenoiseError):
            d.set_tuning(0, 0, 96)
        d.close()
