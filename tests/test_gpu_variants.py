"""Structural variants (Sec. 4.3.2, Tables 8-9) on the GPU against the FP64 oracle.

Every combination of the three stages switched off (A1 voxel gate, A2 density
gate, A3 score selection), the score on a kNN recomputed within P_2, and the
"without octree" configuration (one leaf holding the whole cloud), with the
same element-by-element parity rule as the full method: bit-exact keys,
leaves, voxel counts, gates, neighbour sets and r_K^2; scores within 1e-5;
masks identical outside the tolerance band.
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
    from paper_2512_10386_gb300 import Denoiser
    d = Denoiser(max_points=50_000)
    yield oracle, d
    d.close()


def _run(env, xyz, **kw):
    orc, d = env
    from paper_2512_10386_gb300 import Params
    P = Params(**kw)
    g = to_np(d.run_debug(torch.from_numpy(xyz).cuda(), P))
    r = orc.denoise(xyz, oracle_params(P), debug=True)
    return compare_with_oracle(g, r, P), g, r


@pytest.mark.parametrize("stage_off", list(range(8)))
@pytest.mark.parametrize("rescore", [0, 1])
def test_stage_toggles(env, stage_off, rescore):
    import synth
    xyz, _ = synth.object_cloud(seed=70 + stage_off, n_surface=9000)
    stats, g, r = _run(env, xyz, k=16, leaf_capacity=256, rho_percentile=5.0, stage_off=stage_off,
                       rescore_p2=rescore)
    if stage_off & 1:
        assert not (g["stage"] == 1).any()
    if stage_off & 4:
        assert not (g["stage"] == 3).any() and not g["score"].any()


@pytest.mark.parametrize("mode", [0, 1])
def test_rescore_threshold_and_small_leaves(env, mode):
    # small leaves: P_2 of one point (no neighbour to score with) and lone points without the density gate
    rng = np.random.default_rng(80 + mode)
    xyz = np.concatenate([rng.normal(size=(3000, 3)) * 0.3, rng.uniform(-3, 3, size=(400, 3))]).astype(np.float32)
    for kw in (dict(rescore_p2=1, rho_percentile=20.0), dict(stage_off=2), dict(stage_off=3, rescore_p2=1)):
        _run(env, xyz, k=8, leaf_capacity=16, min_vox_count=1, select_mode=mode, tau=2.0, **kw)


def test_without_octree_single_leaf(env):
    import synth
    xyz, _ = synth.object_cloud(seed=90, n_surface=5000)
    stats, g, r = _run(env, xyz, k=16, leaf_capacity=0xFFFFFFFF)
    assert r["n_leaves"] == 1 and int(g["leaf_count"][0]) == len(xyz)
    print("without octree:", stats)


# ---------------------------------------------------------------------------
# cross-leaf kNN (candidates from the 27 same-level cells around a leaf)
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("k", [8, 16, 32])
def test_cross_leaf_knn(env, k):
    import synth
    orc, d = env
    d.set_cross_leaf(True)
    xyz, _ = synth.object_cloud(seed=95 + k, n_surface=8000)
    stats, g, r = _run(env, xyz, k=k, leaf_capacity=256, cross_leaf=1)
    print(f"cross-leaf k={k}:", stats)


def test_cross_leaf_threshold_mode_and_dense_blob(env):
    orc, d = env
    d.set_cross_leaf(True)
    rng = np.random.default_rng(96)
    xyz = np.concatenate([rng.normal(size=(6000, 3)) * 0.2, rng.uniform(-2, 2, size=(600, 3))]).astype(np.float32)
    _run(env, xyz, k=12, leaf_capacity=128, cross_leaf=1, select_mode=1, tau=5.0, rho_percentile=5.0)


def test_cross_leaf_requires_its_tables_and_excludes_other_variants():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2512_10386_gb300 import Denoiser, Params
    from paper_2512_10386_gb300 import _native as N
    d = Denoiser(max_points=1000)
    try:
        x = torch.rand((1000, 3), device="cuda")
        with pytest.raises(N.DenoiseError) as e:
            d.run(x, Params(k=8, cross_leaf=1))
        assert e.value.status == N.DENOISE_E_STATE
        d.set_cross_leaf(True)
        d.run(x, Params(k=8, cross_leaf=1))
        with pytest.raises(N.DenoiseError) as e:
            d.run(x, Params(k=8, cross_leaf=1, stage_off=1))
        assert e.value.status == N.DENOISE_E_INVAL
    finally:
        d.close()
