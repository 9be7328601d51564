"""CUDA path vs the FP64 oracle, element by element, through the C ABI.

Bit-exact: Morton keys, leaf partition, voxel size h, voxel counts, both
gates, neighbour lists, neighbour distances and r_K^2.  Scores within 1e-5
relative.  Masks identical except for points whose score is within that
tolerance of the selection cut (counted, and bounded by the band).
"""

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

from gpu_helpers import compare_with_oracle, oracle_params, to_np  # noqa: E402


@pytest.fixture(scope="module")
def dn():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__
    __graft_entry__.build()
    from paper_2512_10386_gb300 import Denoiser
    d = Denoiser(max_points=600_000, max_frames=64)
    yield d
    d.close()


@pytest.fixture(scope="module")
def orc():
    import oracle
    oracle.build()
    return oracle


def run_both(dn, orc, xyz, P):
    g = to_np(dn.run_debug(torch.from_numpy(xyz).cuda(), P))
    r = orc.denoise(xyz, oracle_params(P), debug=True)
    return g, r


def P_(**kw):
    from paper_2512_10386_gb300 import Params
    return Params(**kw)


# ---------------------------------------------------------------------------
# the small object workload (36,750 points, K = 16, leaf capacity 512)
# ---------------------------------------------------------------------------
def test_object_workload_full_parity(dn, orc):
    import synth
    xyz, _ = synth.object_cloud(seed=0)
    P = P_(k=16, leaf_capacity=512)
    g, r = run_both(dn, orc, xyz, P)
    stats = compare_with_oracle(g, r, P)
    print("object workload:", stats)
    assert stats["mismatch"] <= max(4, stats["ambiguous"])


@pytest.mark.parametrize("k", [1, 8, 12, 24, 32, 64])
def test_k_variants(dn, orc, k):
    import synth
    xyz, _ = synth.object_cloud(seed=k, n_surface=9000)
    P = P_(k=k, leaf_capacity=300)
    g, r = run_both(dn, orc, xyz, P)
    compare_with_oracle(g, r, P)


def test_threshold_mode_and_parameters(dn, orc):
    import synth
    xyz, _ = synth.object_cloud(seed=5, n_surface=12000)
    for kw in (dict(select_mode=1, tau=7.5), dict(alpha=2.0, sigma=0.6, gamma=3.0, select_mode=1, tau=6.0),
               dict(alpha=-0.5, sigma=1.7, gamma=1.0, eps_k=1e-3, lam=0.7), dict(rho_percentile=10.0, lam=0.9)):
        P = P_(k=12, **kw)
        g, r = run_both(dn, orc, xyz, P)
        compare_with_oracle(g, r, P)


@pytest.mark.parametrize("n", [2, 3, 17, 4095, 4096, 4097, 12289])
def test_ragged_sizes_multi_tile(dn, orc, n):
    rng = np.random.default_rng(n)
    xyz = np.concatenate([rng.normal(size=(n - n // 5, 3)) * 0.2,
                          rng.uniform(-1, 1, size=(n // 5, 3))]).astype(np.float32)
    P = P_(k=8, leaf_capacity=64, beta=2.0, min_vox_count=2)
    g, r = run_both(dn, orc, xyz, P)
    compare_with_oracle(g, r, P)


def test_duplicates_and_oversized_leaf(dn, orc):
    # 2,000 identical points form one max-depth leaf larger than the shared-memory
    # path: it runs on the global spill area, with every distance tie broken by index
    rng = np.random.default_rng(1)
    dup = np.repeat(np.array([[0.25, -0.5, 0.125]], np.float32), 2000, axis=0)
    rest = rng.uniform(-1, 1, size=(3000, 3)).astype(np.float32)
    xyz = np.concatenate([rest[:1500], dup, rest[1500:]])
    P = P_(k=16, leaf_capacity=256)
    g, r = run_both(dn, orc, xyz, P)
    assert r["leaf_count"].max() == 2000
    compare_with_oracle(g, r, P)


@pytest.mark.parametrize("n_cluster", [1500, 5000])
def test_dense_cluster_below_sorted_depth(dn, orc, n_cluster):
    """A cluster far smaller than a level-10 cell of the root cube: its leaves lie
    deeper than the levels the radix passes order, so its cell is brought into full
    octree order on its own (in shared memory up to 2,048 points, else by digit
    passes); with identical points too."""
    rng = np.random.default_rng(n_cluster)
    rest = rng.uniform(-1, 1, size=(4000, 3)).astype(np.float32)
    cl = (np.float32([0.3, -0.2, 0.1]) + rng.uniform(0, 1e-4, size=(n_cluster, 3))).astype(np.float32)
    dup = np.repeat(np.float32([[-0.6, 0.4, 0.7]]), n_cluster // 2, axis=0)
    xyz = np.concatenate([rest[:1000], cl[: n_cluster // 2], dup, rest[1000:], cl[n_cluster // 2:]])
    P = P_(k=16, leaf_capacity=64, min_vox_count=1)
    g, r = run_both(dn, orc, xyz, P)
    assert r["leaf_level"].max() > 10
    compare_with_oracle(g, r, P)


@pytest.mark.parametrize("max_depth", [12, 15])
def test_cluster_below_sorted_depth_limited_depth(dn, orc, max_depth):
    """As above with a depth limit below 21: the sorted key bits start above bit 0
    and the cells needing full order are sorted by the key bits the limit keeps
    (ties in them by input index)."""
    rng = np.random.default_rng(max_depth)
    rest = rng.uniform(-1, 1, size=(3000, 3)).astype(np.float32)
    cl = (np.float32([0.3, -0.2, 0.1]) + rng.uniform(0, 3e-4, size=(2600, 3))).astype(np.float32)
    xyz = np.concatenate([rest[:1000], cl, rest[1000:]])
    P = P_(k=16, leaf_capacity=48, max_depth=max_depth, min_vox_count=1)
    g, r = run_both(dn, orc, xyz, P)
    assert r["leaf_level"].max() > 9
    compare_with_oracle(g, r, P)


def test_shallow_octree_large_leaves(dn, orc):
    import synth
    xyz, _ = synth.object_cloud(seed=7, n_surface=6000)
    P = P_(k=16, leaf_capacity=256, max_depth=2)
    g, r = run_both(dn, orc, xyz, P)
    assert r["leaf_count"].max() > 256    # above the shared-memory path (capacity 256)
    compare_with_oracle(g, r, P)


def test_large_leaf_capacity_global_paths(dn, orc):
    # capacity 3,000: the leaf finder searches global memory (its shared-memory
    # key window holds capacities up to 2,543) and the leaf kernel's CTAs hold
    # 2,048-point leaves (11-bit packed neighbour positions)
    import synth
    xyz, _ = synth.object_cloud(seed=11, n_surface=12000)
    P = P_(k=16, leaf_capacity=3000)
    g, r = run_both(dn, orc, xyz, P)
    assert r["leaf_count"].max() > 1024
    compare_with_oracle(g, r, P)


def test_max_depth_zero_single_leaf(dn, orc):
    rng = np.random.default_rng(2)
    xyz = rng.normal(size=(700, 3)).astype(np.float32)
    P = P_(k=10, leaf_capacity=8, max_depth=0, min_vox_count=1)
    g, r = run_both(dn, orc, xyz, P)
    assert r["n_leaves"] == 1
    compare_with_oracle(g, r, P)


@pytest.mark.parametrize("n", [2, 32, 33, 34, 35, 37, 64, 65, 97, 130])
def test_single_leaf_scan_edges(dn, orc, n):
    """One leaf of n points at K = 32: the whole leaf as the seed window (n <= 33),
    one forward step into the NaN padding (34..37), backward steps that start
    below position 0, and several query rounds."""
    rng = np.random.default_rng(n)
    xyz = rng.normal(size=(n, 3)).astype(np.float32)
    P = P_(k=32, leaf_capacity=n, max_depth=0, min_vox_count=1)
    g, r = run_both(dn, orc, xyz, P)
    assert r["n_leaves"] == 1
    compare_with_oracle(g, r, P)


def test_degenerate_clouds(dn, orc):
    for xyz in (np.zeros((1, 3), np.float32), np.ones((2, 3), np.float32), np.ones((700, 3), np.float32),
                np.stack([np.arange(300, dtype=np.float32), np.zeros(300, np.float32),
                          np.zeros(300, np.float32)], 1)):
        P = P_(k=8, leaf_capacity=64, min_vox_count=1)
        g, r = run_both(dn, orc, xyz, P)
        compare_with_oracle(g, r, P)


@pytest.mark.parametrize("k", [8, 32])
def test_lattice_ties(dn, orc, k):
    """Exact distance ties everywhere; k = 32 also takes the warp-shared seed window."""
    g1 = np.arange(9, dtype=np.float32) * 0.5
    xyz = np.stack(np.meshgrid(g1, g1, g1, indexing="ij"), -1).reshape(-1, 3)
    xyz = xyz[np.random.default_rng(3).permutation(len(xyz))]
    P = P_(k=k, leaf_capacity=100, min_vox_count=1)
    g, r = run_both(dn, orc, xyz, P)
    compare_with_oracle(g, r, P)


def test_topratio_cut_through_exact_score_ties(dn):
    """Two translated copies of one cluster in one leaf (max_depth 0: input
    order is the leaf order) give bit-identical scores pairwise, so the Top-lambda
    cut falls between points of equal F: the kept set must still be the
    ceil(lambda m) largest by (F descending, input index ascending) (Eq. 22)."""
    rng = np.random.default_rng(21)
    a = rng.integers(0, 512, size=(150, 3)).astype(np.float32) / 64.0  # exact in FP32
    a = np.unique(a, axis=0)
    b = a + np.float32(64.0)                                           # exact translation, far apart
    xyz = np.concatenate([a, b]).astype(np.float32)
    n = len(xyz)
    split_a_tie = False
    for lam in (0.5, 0.9, 0.95):
        P = P_(k=8, max_depth=0, leaf_capacity=n, min_vox_count=1, lam=lam)
        res = dn.run(torch.from_numpy(xyz).cuda(), P)
        mask, score, stage = (t.cpu().numpy() for t in (res.mask, res.score, res.stage))
        p2 = np.where((stage == 0) | (stage == 3))[0]
        m = len(p2)
        keep_n = min(m, int(np.ceil(np.float64(lam) * m)))
        F = score[p2]
        order = np.lexsort((p2, -F.astype(np.float64)))  # F descending, then input index
        want = np.zeros(n, np.uint8)
        want[p2[order[:keep_n]]] = 1
        assert np.array_equal(mask, want), lam
        # the cut really splits a group of equal scores for at least one lambda
        split_a_tie |= bool(keep_n < m and F[order[keep_n]] == F[order[keep_n - 1]])
    assert split_a_tie


# ---------------------------------------------------------------------------
# the dense scan workload at full size (560,000 points, K = 32), as benchmarked
# ---------------------------------------------------------------------------
def test_dense_scan_workload_full_parity(dn, orc):
    import synth
    xyz, _ = synth.superquadric_scan(seed=1)
    P = P_(k=32)
    g, r = run_both(dn, orc, xyz, P)
    stats = compare_with_oracle(g, r, P)
    print("dense scan workload:", stats)


# ---------------------------------------------------------------------------
# API behaviour
# ---------------------------------------------------------------------------
def test_host_buffers_match_device_buffers(dn):
    import synth
    xyz, _ = synth.object_cloud(seed=9, n_surface=5000)
    P = P_(k=16)
    rd = dn.run(torch.from_numpy(xyz).cuda(), P)
    rh = dn.run(torch.from_numpy(xyz).pin_memory(), P)
    assert rh.mask.device.type == "cpu"
    assert torch.equal(rd.mask.cpu(), rh.mask) and torch.equal(rd.score.cpu(), rh.score)
    assert torch.equal(rd.stage.cpu(), rh.stage)


def test_pageable_host_input_matches_device_input(dn):
    """Pinned host input is read in place by the bounding-box pass; pageable host
    memory takes the copy-first path: both give the device-input results."""
    import synth
    xyz, _ = synth.object_cloud(seed=11, n_surface=5000)
    P = P_(k=16)
    rd = dn.run(torch.from_numpy(xyz).cuda(), P)
    src = torch.from_numpy(xyz.copy())  # pageable
    assert not src.is_pinned()
    rp = dn.run(src, P)
    assert torch.equal(rd.mask.cpu(), rp.mask.cpu()) and torch.equal(rd.score.cpu(), rp.score.cpu())
    assert torch.equal(rd.stage.cpu(), rp.stage.cpu())


def test_host_outputs_any_alignment_and_pageable(dn):
    """Results into pinned host buffers are written by one kernel through their
    mapped addresses (16-byte stores where source and destination offsets agree,
    bytes elsewhere); pageable ones go through the copy engine.  Every placement
    gives the device results, and no byte outside a result buffer changes."""
    import synth
    xyz, _ = synth.object_cloud(seed=12, n_surface=7001)
    n = xyz.shape[0]
    P = P_(k=16)
    rd = dn.run(torch.from_numpy(xyz).cuda(), P)
    want = (rd.mask.cpu(), rd.score.cpu(), rd.stage.cpu())
    xh = torch.from_numpy(xyz).pin_memory()
    for off in (0, 1, 3, 16, 17):
        bm = torch.full((n + 64,), 0xA5, dtype=torch.uint8).pin_memory()
        bs = torch.full((n + 64,), -7.0, dtype=torch.float32).pin_memory()
        bg = torch.full((n + 64,), 0x5A, dtype=torch.uint8).pin_memory()
        r = dn.run(xh, P, mask=bm[off:off + n], score=bs[off:off + n], stage=bg[off:off + n])
        for got, exp in zip((r.mask, r.score, r.stage), want):
            assert torch.equal(got, exp), off
        for b, fill in ((bm, 0xA5), (bs, -7.0), (bg, 0x5A)):
            assert bool((b[:off] == fill).all()) and bool((b[off + n:] == fill).all()), off
    # pageable outputs (copy engine), alone and mixed with pinned ones
    pm, ps, pg = torch.empty(n, dtype=torch.uint8), torch.empty(n), torch.empty(n, dtype=torch.uint8)
    assert not pm.is_pinned()
    r = dn.run(xh, P, mask=pm, score=ps, stage=pg)
    assert torch.equal(pm, want[0]) and torch.equal(ps, want[1]) and torch.equal(pg, want[2])
    qm = torch.empty(n, dtype=torch.uint8).pin_memory()
    ps2 = torch.empty(n)
    r = dn.run(xh, P, mask=qm, score=ps2)
    assert torch.equal(qm, want[0]) and torch.equal(ps2, want[1]) and torch.equal(r.stage.cpu(), want[2])


def test_input_at_any_point_offset(dn):
    """The bounding-box pass reads 16-byte words where the input (and its device
    copy) allow and single values elsewhere: device and pinned host input that
    start 1, 2 or 3 points into a buffer give the aligned input's results."""
    import synth
    xyz, _ = synth.object_cloud(seed=13, n_surface=9001)
    n = xyz.shape[0]
    P = P_(k=16)
    rd = dn.run(torch.from_numpy(xyz).cuda(), P)
    for off in (1, 2, 3):
        buf = torch.zeros((n + 4, 3), dtype=torch.float32)
        buf[off:off + n] = torch.from_numpy(xyz)
        for src in (buf.cuda(), buf.pin_memory()):
            r = dn.run(src[off:off + n], P)
            assert torch.equal(r.mask.cpu(), rd.mask.cpu()) and torch.equal(r.score.cpu(), rd.score.cpu()), off
            assert torch.equal(r.stage.cpu(), rd.stage.cpu()), off


def test_deterministic_bytes(dn):
    import synth
    xyz, _ = synth.object_cloud(seed=10, n_surface=20000)
    t = torch.from_numpy(xyz).cuda()
    a = dn.run(t, P_(k=16))
    b = dn.run(t, P_(k=16))
    assert torch.equal(a.mask, b.mask) and torch.equal(a.score, b.score) and torch.equal(a.stage, b.stage)


def test_batch_equals_single_frames(dn, orc):
    import synth
    frames = [synth.object_cloud(seed=s, n_surface=ns)[0] for s, ns in ((20, 3000), (21, 9000), (22, 1))]
    frames.insert(1, np.zeros((0, 3), np.float32))
    offs = np.cumsum([0] + [len(f) for f in frames]).tolist()
    xyz = np.concatenate(frames)
    P = P_(k=12)
    rb = dn.run_batch(torch.from_numpy(xyz).cuda(), offs, P)
    for f, fr in enumerate(frames):
        a, b = offs[f], offs[f + 1]
        if b == a:
            continue
        rs = dn.run(torch.from_numpy(fr).cuda(), P)
        assert torch.equal(rb.mask[a:b], rs.mask) and torch.equal(rb.score[a:b], rs.score)
        ref = orc.denoise(fr, oracle_params(P), debug=True)
        compare_with_oracle({"mask": rs.mask.cpu().numpy(), "score": rs.score.cpu().numpy(),
                             "stage": rs.stage.cpu().numpy()}, ref, P, check_debug=False)


def test_async_calls_with_changing_layouts(dn):
    # back-to-back asynchronous calls on one context, each with a new frame
    # layout: the pinned tile tables are staged through a ring of slots, so a
    # call never overwrites a table that an earlier call is still copying
    import synth
    from paper_2512_10386_gb300 import Params
    from paper_2512_10386_gb300 import _native as N
    P = Params(k=16)
    clouds = [torch.from_numpy(synth.object_cloud(seed=300 + i, n_surface=n)[0]).cuda()
              for i, n in enumerate((3000, 9000, 1500, 20000, 6000, 12000, 2500))]
    ref = [[x.clone() for x in (r.mask, r.score, r.stage)] for r in (dn.run(c, P) for c in clouds)]
    s = torch.cuda.Stream()
    outs = [(torch.empty(len(c), dtype=torch.uint8, device="cuda"), torch.empty(len(c), device="cuda"),
             torch.empty(len(c), dtype=torch.uint8, device="cuda")) for c in clouds]
    dn.set_sync(False)
    try:
        for rep in range(2):
            for c, (m, sc, st) in zip(clouds, outs):
                dn.run(c, P, mask=m, score=sc, stage=st, stream=s)
        s.synchronize()
        assert dn.status(s) == N.DENOISE_OK
    finally:
        dn.set_sync(True)
    for r, o in zip(ref, outs):
        for a_, b_ in zip(r, o):
            assert torch.equal(a_, b_)


def test_graph_mode_matches_direct(dn):
    import synth
    xyz, _ = synth.object_cloud(seed=11, n_surface=8000)
    t = torch.from_numpy(xyz).cuda()
    ref = dn.run(t, P_(k=16))
    dn.set_graphs(True)
    try:
        for _ in range(3):   # first call captures, the others replay
            r = dn.run(t, P_(k=16))
            assert torch.equal(r.mask, ref.mask) and torch.equal(r.score, ref.score)
        r2 = dn.run(t, P_(k=8))  # new parameters: re-capture
    finally:
        dn.set_graphs(False)
    ref2 = dn.run(t, P_(k=8))
    assert torch.equal(r2.mask, ref2.mask) and torch.equal(r2.score, ref2.score)


def test_layout_changes_direct_and_graph(dn):
    """The tile and frame tables are uploaded only when the frame layout changes
    (repeated layouts reuse the device copy), and a captured graph is replayed
    only while the staging slot its table copies read still holds its layout:
    alternating sizes, repeats, and a graph replay after the staging ring has
    wrapped through other layouts all give the direct results."""
    import synth
    xyz, _ = synth.object_cloud(seed=14, n_surface=12000)
    t = torch.from_numpy(xyz).cuda()
    sizes = [t.shape[0], 9000, 7001, 5003, 3000, 2001]
    P = P_(k=16)
    ref = {n: dn.run(t[:n], P) for n in sizes}
    ref = {n: (r.mask.clone(), r.score.clone()) for n, r in ref.items()}

    def same(n, r):
        return torch.equal(r.mask, ref[n][0]) and torch.equal(r.score, ref[n][1])

    for n in (sizes[1], sizes[1], sizes[2], sizes[1], sizes[1], sizes[0]):
        assert same(n, dn.run(t[:n], P)), n
    dn.set_graphs(True)
    try:
        assert same(sizes[0], dn.run(t[:sizes[0]], P))          # captured
        dn.set_graphs(False)
        for n in sizes[1:]:                                       # the ring of staging slots wraps
            assert same(n, dn.run(t[:n], P)), n
        dn.set_graphs(True)
        for _ in range(2):
            assert same(sizes[0], dn.run(t[:sizes[0]], P))      # re-captured, then replayed
    finally:
        dn.set_graphs(False)


def test_errors(dn):
    from paper_2512_10386_gb300 import _native as N
    bad = torch.zeros((10, 3), device="cuda")
    bad[3, 1] = float("nan")
    with pytest.raises(N.DenoiseError) as e:
        dn.run(bad, P_())
    assert e.value.status == N.DENOISE_E_NONFINITE
    inf = torch.zeros((10, 3), device="cuda")
    inf[0, 0] = float("inf")
    with pytest.raises(N.DenoiseError) as e:
        dn.run(inf, P_())
    assert e.value.status == N.DENOISE_E_NONFINITE
    with pytest.raises(N.DenoiseError) as e:
        dn.run(torch.zeros((10, 3), device="cuda"), P_(k=0))
    assert e.value.status == N.DENOISE_E_INVAL
    with pytest.raises(N.DenoiseError) as e:
        dn.run(torch.zeros((dn.max_points + 1, 3), device="cuda"), P_())
    assert e.value.status == N.DENOISE_E_CAPACITY
    r = dn.run(torch.zeros((0, 3), device="cuda"), P_())
    assert r.mask.numel() == 0
    # the context stays usable after errors
    xyz = torch.rand((1000, 3), device="cuda")
    dn.run(xyz, P_(k=8))


def test_stats_count_pairs(dn, orc):
    import synth
    xyz, _ = synth.object_cloud(seed=0)
    P = P_(k=16)
    dn.run(torch.from_numpy(xyz).cuda(), P)
    s = dn.stats()
    r = orc.denoise(xyz, oracle_params(P), debug=True)
    n1 = r["leaf_n1"].astype(np.int64)
    assert s["knn_pairs"] == int((n1 * (n1 - 1))[n1 > 1].sum())
    assert s["n_leaves"] == r["n_leaves"]
    assert s["n_p1"] == int(n1[n1 > 1].sum())
