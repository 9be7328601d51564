"""Pins of the FP64 oracle against facts that do not come from the oracle itself.

Each test checks one part of the method (arXiv 2512.10386, Sec. 3) against a
hand-worked value, a closed form, a library routine, an invariant or a brute
force written independently, so that a dropped term, a wrong sign, index or
exponent in oracle.c fails at least one of them.
"""

import os

import numpy as np
import pytest

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _params(orc, **kw):
    return orc.Params(**kw)


# --------------------------------------------------------------------------
# Morton keys (Sec. 3 octree; reading R1)
# --------------------------------------------------------------------------
def _golden_rows(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append(line.split())
    return rows


def test_interleave_hand_worked(orc):
    for qx, qy, qz, key in _golden_rows("morton_hand.txt"):
        assert orc.interleave(int(qx), int(qy), int(qz)) == int(key)


def _spread3(v):
    """Textbook magic-number bit spread (a different algorithm from the oracle's loop)."""
    v &= 0x1FFFFF
    v = (v | (v << 32)) & 0x1F00000000FFFF
    v = (v | (v << 16)) & 0x1F0000FF0000FF
    v = (v | (v << 8)) & 0x100F00F00F00F00F
    v = (v | (v << 4)) & 0x10C30C30C30C30C3
    v = (v | (v << 2)) & 0x1249249249249249
    return v


def test_interleave_matches_magic_bits(orc):
    rng = np.random.default_rng(3)
    for _ in range(300):
        qx, qy, qz = (int(v) for v in rng.integers(0, 2 ** 21, 3))
        want = (_spread3(qx) << 2) | (_spread3(qy) << 1) | _spread3(qz)
        assert orc.interleave(qx, qy, qz) == want


def test_root_cube_quantisation_hand_worked(orc):
    xyz = np.array([[0, 0, 0], [1.0, 0.5, 0.25]], np.float32)
    r = orc.denoise(xyz, _params(orc, k=1, min_vox_count=1), debug=True)
    assert r["root"].tolist() == [0.0, 0.0, 0.0, 1.0]
    # side 1 -> s = 2^21; q = (2^21 clamped to 2^21-1, 2^20, 2^19)
    assert int(r["key"][0]) == 0
    assert int(r["key"][1]) == 7720456504063707428


# --------------------------------------------------------------------------
# octree (Sec. 3; reading R2)
# --------------------------------------------------------------------------
def _leaf_partition_by_counting(keys, cap, max_depth):
    """Leaf of each point = shallowest ancestor holding <= cap points (or max depth).

    Counts are taken with numpy.unique on key prefixes, independently of the
    oracle's recursive split."""
    n = len(keys)
    level = np.full(n, -1, np.int64)
    for L in range(0, max_depth + 1):
        pref = keys >> np.uint64(63 - 3 * L) if L > 0 else np.zeros(n, np.uint64)
        _, inv, cnt = np.unique(pref, return_inverse=True, return_counts=True)
        c = cnt[inv]
        newly = (level < 0) & ((c <= cap) | (L == max_depth))
        level[newly] = L
    return level


@pytest.mark.parametrize("seed,cap,depth", [(0, 8, 21), (1, 32, 21), (2, 5, 4), (3, 64, 21)])
def test_octree_matches_prefix_counting(orc, seed, cap, depth):
    rng = np.random.default_rng(seed)
    a = rng.normal(size=(600, 3)) * 0.05
    b = rng.uniform(-1, 1, size=(400, 3))
    c = np.repeat(rng.uniform(-1, 1, size=(1, 3)), 40, axis=0)   # 40 exact duplicates
    xyz = np.concatenate([a, b, c]).astype(np.float32)
    p = _params(orc, k=4, leaf_capacity=cap, max_depth=depth, min_vox_count=1)
    r = orc.denoise(xyz, p, debug=True)
    keys = r["key"]
    lvl = _leaf_partition_by_counting(keys, cap, depth)
    order = np.lexsort((np.arange(len(keys)), keys))
    # leaves partition the sorted order into contiguous runs
    starts, counts, levels = r["leaf_start"], r["leaf_count"], r["leaf_level"]
    assert starts[0] == 0 and int(counts.sum()) == len(xyz)
    assert np.all(starts[1:] == starts[:-1] + counts[:-1])
    for s, cnt, L in zip(starts, counts, levels):
        pts = order[s:s + cnt]
        assert np.all(lvl[pts] == L)
        if L > 0:
            pref = keys[pts] >> np.uint64(63 - 3 * int(L))
            assert np.all(pref == pref[0])
        assert cnt <= cap or L == depth
    # every point's leaf id points at the leaf holding it
    pos = np.empty(len(xyz), np.int64)
    pos[order] = np.arange(len(xyz))
    lid = r["leaf_of"]
    assert np.all(pos >= starts[lid]) and np.all(pos < starts[lid] + counts[lid])


# --------------------------------------------------------------------------
# Eq. 11 cube root (reading R4)
# --------------------------------------------------------------------------
def test_cbrt_spec_against_numpy(orc):
    rng = np.random.default_rng(4)
    us = np.concatenate([10.0 ** rng.uniform(-30, 30, 2000), [1e-300, 1e300, 3.0, 0.5]])
    for u in us:
        got, want = orc.cbrt_spec(u), np.cbrt(u)
        assert abs(got - want) <= 2 * np.spacing(want)


@pytest.mark.parametrize("u,root", [(8.0, 2.0), (27.0, 3.0), (0.125, 0.5), (1.0, 1.0),
                                    (27.0 / 64.0, 0.75), (2.0 ** -30, 2.0 ** -10)])
def test_cbrt_spec_perfect_cubes(orc, u, root):
    assert abs(orc.cbrt_spec(u) - root) <= np.spacing(root)


# --------------------------------------------------------------------------
# voxel gate (Eq. 10-12; reading R5)
# --------------------------------------------------------------------------
def _lattice4():
    g = np.arange(4, dtype=np.float32)
    return np.stack(np.meshgrid(g, g, g, indexing="ij"), -1).reshape(-1, 3)


def test_voxel_gate_hand_worked_lattice(orc):
    xyz = _lattice4()
    for beta, m0, m1, m2, m3, p1 in _golden_rows("voxel_lattice.txt"):
        m = np.array([int(m0), int(m1), int(m2), int(m3)])
        p = _params(orc, k=4, beta=float(beta), min_vox_count=4, leaf_capacity=512)
        r = orc.denoise(xyz, p, debug=True)
        assert r["n_leaves"] == 1
        assert abs(float(r["leaf_h"][0]) - 0.75 * float(beta)) <= 1e-6
        xi = xyz.astype(int)
        want = m[xi[:, 0]] * m[xi[:, 1]] * m[xi[:, 2]]
        assert np.array_equal(r["vox_count"], want)
        assert int((r["stage"] != 1).sum()) == int(p1)


def test_voxel_counts_bruteforce_random(orc):
    rng = np.random.default_rng(5)
    xyz = (rng.normal(size=(700, 3)) * np.array([1.0, 1.0, 0.05])).astype(np.float32)
    p = _params(orc, k=4, beta=1.5, leaf_capacity=1000, min_vox_count=3)
    r = orc.denoise(xyz, p, debug=True)
    assert r["n_leaves"] == 1
    lo, h = r["leaf_lo"][0], r["leaf_h"][0]
    v = np.floor((xyz - lo) / h).astype(np.int64)     # FP32 ops, as Eq. 12's grid
    eq = (v[:, None, :] == v[None, :, :]).all(-1)       # O(N^2) pairwise equality
    assert np.array_equal(r["vox_count"], eq.sum(1))
    assert np.array_equal(r["stage"] == 1, eq.sum(1) < 3)


# --------------------------------------------------------------------------
# kNN (Sec. 3 "k nearest neighbours"; readings R6, R7)
# --------------------------------------------------------------------------
def test_knn_bruteforce_full_sort(orc):
    rng = np.random.default_rng(6)
    xyz = rng.uniform(-1, 1, size=(300, 3)).astype(np.float32)
    K = 10
    p = _params(orc, k=K, leaf_capacity=1000, min_vox_count=1)
    r = orc.denoise(xyz, p, debug=True)
    x64 = xyz.astype(np.float64)
    d2 = ((x64[:, None, :] - x64[None, :, :]) ** 2).sum(-1)
    np.fill_diagonal(d2, np.inf)
    srt = np.sort(d2, axis=1)
    checked = 0
    for i in range(len(xyz)):
        # skip queries with a near-tie at the K-th place (FP32 vs FP64 order)
        if srt[i, K] - srt[i, K - 1] < 1e-6 * srt[i, K]:
            continue
        want = set(np.argsort(d2[i], kind="stable")[:K].tolist())
        assert set(r["nbr"][i].tolist()) == want
        # listed in ascending distance
        assert np.all(np.diff(d2[i, r["nbr"][i]]) >= -1e-7)
        assert abs(float(r["r2"][i]) - srt[i, K - 1]) <= 1e-6 * srt[i, K - 1]
        checked += 1
    assert checked > 280


def test_knn_lattice_tie_break_by_index(orc):
    g = np.arange(5, dtype=np.float32)
    xyz = np.stack(np.meshgrid(g, g, g, indexing="ij"), -1).reshape(-1, 3)
    perm = np.random.default_rng(7).permutation(len(xyz))
    xyz = xyz[perm]
    p = _params(orc, k=8, leaf_capacity=1000, min_vox_count=1)
    r = orc.denoise(xyz, p, debug=True)
    c = int(np.where((xyz == 2).all(1))[0][0])
    d2 = ((xyz - xyz[c]) ** 2).sum(1)
    six = np.where(d2 == 1)[0]
    twelve = np.sort(np.where(d2 == 2)[0])
    assert len(six) == 6 and len(twelve) == 12
    got = r["nbr"][c].tolist()
    # six unit neighbours first, in index order; then the two lowest-index diagonals
    assert got[:6] == sorted(six.tolist())
    assert got[6:] == twelve[:2].tolist()
    assert float(r["r2"][c]) == 2.0
    # Eq. 13 closed form: rho = k / (4/3 pi r^3) with r = sqrt(2)
    assert abs(r["rho"][c] - 8 / (4 / 3 * np.pi * 2 ** 1.5)) < 1e-12


def test_small_leaf_keff_and_lone_removal(orc):
    # three points: k_eff = 2 although K = 16; a single point cannot be scored
    xyz = np.array([[0, 0, 0], [1, 0, 0], [0, 2, 0]], np.float32)
    p = _params(orc, k=16, min_vox_count=1)
    r = orc.denoise(xyz, p, debug=True)
    assert r["nbr"][0, :2].tolist() == [1, 2] and r["nbr"][0, 2] == 0xFFFFFFFF
    assert float(r["r2"][0]) == 4.0
    # Eq. 13 with k_eff = 2 for K: rho = 2 / (4/3 pi 2^3)
    assert abs(r["rho"][0] - 2 / (4 / 3 * np.pi * 8)) < 1e-15
    r1 = orc.denoise(xyz[:1], p, debug=True)
    assert r1["stage"].tolist() == [2] and r1["mask"].tolist() == [0]


# --------------------------------------------------------------------------
# density gate (Eq. 13-14; reading R8) and median (Eq. 16; R9)
# --------------------------------------------------------------------------
@pytest.mark.parametrize("q", [0.2, 5.0, 12.5, 33.0, 50.0, 99.0])
def test_percentile_gate_matches_numpy_hazen(orc, q):
    rng = np.random.default_rng(8)
    xyz = np.concatenate([rng.normal(size=(400, 3)) * 0.3,
                          rng.uniform(-3, 3, size=(100, 3))]).astype(np.float32)
    p = _params(orc, k=8, leaf_capacity=1000, min_vox_count=1, rho_percentile=q)
    r = orc.denoise(xyz, p, debug=True)
    rho = r["rho"]
    thr = np.percentile(rho, q, method="hazen")    # MATLAB prctile's definition
    assert np.array_equal(r["stage"] == 2, rho < thr)


def test_median_matches_numpy(orc):
    rng = np.random.default_rng(9)
    for n in (301, 302):
        xyz = rng.normal(size=(n, 3)).astype(np.float32)
        p = _params(orc, k=6, leaf_capacity=1000, min_vox_count=1, rho_percentile=20.0)
        r = orc.denoise(xyz, p, debug=True)
        p2 = r["stage"] != 2
        assert abs(r["leaf_rho_med"][0] - np.median(r["rho"][p2])) <= 1e-12 * r["leaf_rho_med"][0]
        assert r["leaf_n2"][0] == p2.sum()


# --------------------------------------------------------------------------
# score (Eq. 15-21; reading R10), closed forms
# --------------------------------------------------------------------------
SEPS = [0.5, 0.75, 1.0, 1.25]


def _pairs_cloud(loner=False):
    pts = []
    for i, s in enumerate(SEPS):
        pts += [[10.0 * i, 0, 0], [10.0 * i + s, 0, 0]]
    if loner:
        pts.append([0.0, 40.0, 0.0])
    return np.array(pts, np.float32)


def _f32(v):
    """The library's parameters are FP32: closed forms use the same rounded values."""
    return float(np.float32(v))


def _pair_score(s, rho_med, alpha, sigma, gamma, eps_k, eps_rho=0.0):
    # K = 1: the partner is the only neighbour; r_K = s, rho_i = rho_j = 3/(4 pi s^3)
    alpha, sigma, gamma, eps_k, eps_rho = map(_f32, (alpha, sigma, gamma, eps_k, eps_rho))
    rho = 3.0 / (4.0 * np.pi * s ** 3)
    w = (rho * rho / (rho_med ** 2 + eps_rho)) ** (alpha / 2)
    return w * np.exp(-1.0 / (2 * sigma ** 2)) / (s ** gamma + eps_k)


@pytest.mark.parametrize("alpha,sigma,gamma,eps_k", [
    (1.0, 1.0, 2.0, 0.0), (2.5, 0.5, 2.0, 0.0), (0.0, 2.0, 3.0, 0.0),
    (1.0, 1.0, 1.0, 0.1), (-1.0, 0.7, 2.0, 0.25)])
def test_score_closed_form_pairs_even(orc, alpha, sigma, gamma, eps_k):
    xyz = _pairs_cloud()
    p = _params(orc, k=1, min_vox_count=1, rho_percentile=0.0, alpha=alpha, sigma=sigma,
                gamma=gamma, eps_k=eps_k, eps_rho=0.0)
    r = orc.denoise(xyz, p, debug=True)
    rho = lambda s: 3.0 / (4.0 * np.pi * s ** 3)
    # 8 densities ascending: d,d,c,c,b,b,a,a -> median = mean of rho_c and rho_b
    rho_med = 0.5 * (rho(SEPS[1]) + rho(SEPS[2]))
    assert abs(r["leaf_rho_med"][0] - rho_med) <= 1e-12 * rho_med
    for i, s in enumerate(SEPS):
        want = _pair_score(s, rho_med, alpha, sigma, gamma, eps_k)
        for j in (2 * i, 2 * i + 1):
            assert abs(r["score"][j] - want) <= 1e-12 * want


def test_score_closed_form_pairs_odd_with_eps_rho(orc):
    xyz = _pairs_cloud(loner=True)
    rho = lambda s: 3.0 / (4.0 * np.pi * s ** 3)
    rho_med = rho(SEPS[2])       # 9 values: loner, d,d,c,c,b,b,a,a -> 5th = rho_c
    alpha, sigma = 1.5, 0.8
    p = _params(orc, k=1, min_vox_count=1, rho_percentile=0.0, alpha=alpha, sigma=sigma,
                gamma=2.0, eps_k=0.0, eps_rho=float(np.float32(rho_med ** 2)))
    r = orc.denoise(xyz, p, debug=True)
    assert abs(r["leaf_rho_med"][0] - rho_med) <= 1e-12 * rho_med
    eps_rho = float(np.float32(rho_med ** 2))
    for i, s in enumerate(SEPS):
        want = _pair_score(s, rho_med, alpha, sigma, 2.0, 0.0, eps_rho)
        assert abs(r["score"][2 * i] - want) <= 1e-12 * want
    # eps_rho = rho_med^2 halves W: the score scales by 2^(-alpha/2) vs eps_rho = 0
    p0 = _params(orc, k=1, min_vox_count=1, rho_percentile=0.0, alpha=alpha, sigma=sigma,
                 gamma=2.0, eps_k=0.0, eps_rho=0.0)
    r0 = orc.denoise(xyz, p0)
    ratio = r["score"][:8] / r0["score"][:8]
    assert np.allclose(ratio, (rho_med ** 2 / (rho_med ** 2 + eps_rho)) ** (_f32(alpha) / 2), rtol=1e-9)
    assert np.allclose(ratio, 2.0 ** (-alpha / 2), rtol=1e-6)


def test_score_closed_form_chain_unequal_densities(orc):
    # K = 1 on x = 0, 1, 3: NN(A)=B, NN(B)=A (d=1), NN(C)=B (d=2).  r = 1, 1, 2;
    # rho_A = rho_B = 3/(4 pi), rho_C = rho_A/8; ascending (C, A, B) -> rho_med = rho_A.
    # F_C = (rho_C rho_B / rho_med^2)^(alpha/2) exp(-4/(2 sigma^2 4)) / 2^gamma
    #     = (1/8)^(alpha/2) exp(-1/(2 sigma^2)) / 2^gamma
    xyz = np.array([[0, 0, 0], [1, 0, 0], [3, 0, 0]], np.float32)
    for alpha, sigma, gamma in ((1.0, 1.0, 2.0), (2.0, 0.5, 3.0)):
        p = _params(orc, k=1, min_vox_count=1, rho_percentile=0.0, alpha=alpha, sigma=sigma,
                    gamma=gamma, eps_k=0.0, eps_rho=0.0)
        r = orc.denoise(xyz, p, debug=True)
        assert abs(r["leaf_rho_med"][0] - 3 / (4 * np.pi)) < 1e-15
        want_c = 0.125 ** (alpha / 2) * np.exp(-1 / (2 * sigma ** 2)) / 2 ** gamma
        want_a = np.exp(-1 / (2 * sigma ** 2))
        assert abs(r["score"][2] - want_c) <= 1e-12 * want_c
        assert abs(r["score"][0] - want_a) <= 1e-12 * want_a


def test_flat_leaf_extent_floor(orc):
    # Eq. 10 on an exactly planar leaf (z = 0) would give V_t = 0; reading R3 floors
    # H_z at delta = side * 2^-21, so h = beta (H_x H_y delta / N_t)^(1/3).
    g = np.arange(4, dtype=np.float32)
    X, Y = np.meshgrid(g, g, indexing="ij")
    xyz = np.stack([X.ravel(), Y.ravel(), np.zeros(16, np.float32)], 1).astype(np.float32)
    beta = 2.0
    r = orc.denoise(xyz, _params(orc, k=4, beta=beta, min_vox_count=1), debug=True)
    delta = 3.0 * 2.0 ** -21
    want = beta * (3.0 * 3.0 * delta / 16.0) ** (1 / 3)
    assert abs(float(r["leaf_h"][0]) - want) <= 1e-6 * want


def test_score_closed_form_lattice_interior(orc):
    # interior point of a cubic lattice, spacing a, K = 6: r_K = a, all densities
    # equal near the centre, F = 6 exp(-1/(2 sigma^2)) / (a^gamma + eps_k) when W = 1
    a = 0.5
    g = np.arange(7, dtype=np.float32) * a
    xyz = np.stack(np.meshgrid(g, g, g, indexing="ij"), -1).reshape(-1, 3)
    sigma, gamma = 0.9, 2.0
    p = _params(orc, k=6, min_vox_count=1, rho_percentile=0.0, alpha=0.0, sigma=sigma,
                gamma=gamma, eps_k=0.0, leaf_capacity=1000)
    r = orc.denoise(xyz, p, debug=True)
    c = int(np.where((xyz == 3 * a).all(1))[0][0])
    assert float(r["r2"][c]) == a * a
    want = 6 * np.exp(-1 / (2 * _f32(sigma) ** 2)) / a ** gamma
    assert abs(r["score"][c] - want) <= 1e-12 * want


def test_scaling_law(orc):
    # F(sP) = s^(-gamma) F(P) for eps = 0; s a power of two keeps every FP32 step exact
    from synth import object_cloud
    xyz, _ = object_cloud(seed=11, n_surface=3000)
    for gamma in (2.0, 3.0):
        p = _params(orc, k=12, alpha=1.3, sigma=0.8, gamma=gamma, eps_k=0.0, eps_rho=0.0,
                    beta=3.0, leaf_capacity=256)
        r1 = orc.denoise(xyz, p)
        r2 = orc.denoise(xyz * np.float32(4.0), p)
        assert np.array_equal(r1["stage"], r2["stage"])
        sc = r1["score"] > 0
        assert np.allclose(r2["score"][sc], 4.0 ** -gamma * r1["score"][sc], rtol=1e-12)


# --------------------------------------------------------------------------
# THRESHOLD selection (ln F >= tau) and the soft removal of the differentiable form
# --------------------------------------------------------------------------
def _unit_weight_pairs(orc, tau, **kw):
    """Pairs cloud with K = 1, alpha = 0 (w_den = 1 exactly), sigma = 1e19 (the
    distance weight exp(-1/(2 sigma^2)) rounds to 1 exactly in FP64), gamma = 2,
    eps_k = 0: each pair's score is F = 1/s^2 exactly, so ln F = -2 ln s, and the
    pair at s = 1 scores F = 1, ln F = 0 exactly."""
    xyz = _pairs_cloud()
    p = _params(orc, k=1, min_vox_count=1, rho_percentile=0.0, alpha=0.0, sigma=1e19, gamma=2.0,
                eps_k=0.0, eps_rho=0.0, select_mode=1, tau=tau, **kw)
    return xyz, p


def test_threshold_selection_closed_form(orc):
    # F = 4, 16/9, 1, 0.64 for s = 0.5, 0.75, 1, 1.25 -> ln F = 1.386, 0.575, 0, -0.446
    want_F = [1.0 / s ** 2 for s in SEPS]
    for tau, kept in ((0.0, [True, True, True, False]),    # ln F >= 0 keeps F = 1 (>= not >)
                      (1.0, [True, False, False, False]),  # log10 F = 0.60 < 1 would drop s = 0.5
                      (0.5, [True, True, False, False]),   # F >= 0.5 would keep every pair
                      (-0.45, [True, True, True, True]),
                      (2.0, [False, False, False, False])):
        xyz, p = _unit_weight_pairs(orc, tau)
        r = orc.denoise(xyz, p)
        for i, s in enumerate(SEPS):
            for j in (2 * i, 2 * i + 1):
                assert r["score"][j] == want_F[i]
                assert bool(r["mask"][j]) == kept[i], (tau, s)
                assert r["stage"][j] == (0 if kept[i] else 3)
    # tau just above / below each pair's ln F flips exactly that pair
    for i, s in enumerate(SEPS):
        lnF = float(np.log(want_F[i]))
        for d, keep in ((1e-3, False), (-1e-3, True)):
            xyz, p = _unit_weight_pairs(orc, lnF + d)
            r = orc.denoise(xyz, p)
            assert bool(r["mask"][2 * i]) == keep and bool(r["mask"][2 * i + 1]) == keep


def test_soft_removal_closed_form(orc):
    # r_i = 1 - sigmoid((ln F_i - tau)/T) on P_2: with ln F = -2 ln s this is
    # 1/(1 + exp((-2 ln s - tau)/T)); the s = 1 pair at tau = 0 sits at exactly 0.5
    T = 0.5
    for tau in (0.0, 0.3):
        xyz, p = _unit_weight_pairs(orc, tau, temperature=T)
        noise = np.zeros(len(xyz), np.uint8)
        noise[-2:] = 1
        loss, grad, rem = orc.softf1(xyz, p, noise)
        for i, s in enumerate(SEPS):
            z = (-2.0 * np.log(s) - _f32(tau)) / T
            want = 1.0 / (1.0 + np.exp(z))
            assert abs(rem[2 * i] - want) <= 1e-12 and abs(rem[2 * i + 1] - want) <= 1e-12
        if tau == 0.0:
            assert rem[4] == 0.5 and rem[5] == 0.5
        # soft F1 of Eq. 26-28 with soft removal counts
        want_loss = 1 - 2 * (rem * noise).sum() / (rem.sum() + noise.sum())
        assert abs(loss - want_loss) <= 1e-12
    # points removed by a gate count as removed with probability 1
    xyz, p = _unit_weight_pairs(orc, 0.0, temperature=T)
    xyz = np.concatenate([xyz, np.array([[0.0, 60.0, 0.0]], np.float32)])
    p.min_vox_count = 2
    p.beta = 0.5
    r = orc.denoise(xyz, p)
    assert r["stage"][-1] == 1
    noise = np.zeros(len(xyz), np.uint8)
    _, _, rem = orc.softf1(xyz, p, noise)
    assert rem[-1] == 1.0


# --------------------------------------------------------------------------
# invariants and special cases of the whole pipeline
# --------------------------------------------------------------------------
def test_permutation_invariance(orc):
    from synth import object_cloud
    xyz, _ = object_cloud(seed=12, n_surface=4000)
    p = _params(orc, k=16, beta=3.0, leaf_capacity=256)
    r = orc.denoise(xyz, p)
    perm = np.random.default_rng(13).permutation(len(xyz))
    rp = orc.denoise(xyz[perm], p)
    assert np.array_equal(rp["mask"], r["mask"][perm])
    assert np.array_equal(rp["stage"], r["stage"][perm])
    assert np.array_equal(rp["score"], r["score"][perm])


def test_rigid_motion_invariance_of_scores(orc):
    # one leaf, voxel gate off (n_v = 1), density gate off (q = 0): rotation and
    # translation leave the kNN + score stages unchanged up to FP32 rounding of d^2
    rng = np.random.default_rng(14)
    xyz = np.concatenate([rng.normal(size=(500, 3)) * np.array([1, 0.5, 0.1]),
                          rng.uniform(-3, 3, size=(50, 3))]).astype(np.float32)
    p = _params(orc, k=10, min_vox_count=1, rho_percentile=0.0, leaf_capacity=1000,
                select_mode=1, tau=-1e30)
    r = orc.denoise(xyz, p, debug=True)
    q, _ = np.linalg.qr(rng.normal(size=(3, 3)))
    moved = (xyz.astype(np.float64) @ q.T + np.array([0.3, -2.0, 1.1])).astype(np.float32)
    rm = orc.denoise(moved, p, debug=True)
    same = np.array([set(a) == set(b) for a, b in zip(r["nbr"], rm["nbr"])])
    assert same.mean() > 0.97
    assert np.allclose(rm["score"][same], r["score"][same], rtol=1e-4)


def test_lone_far_point_removed(orc):
    from synth import object_cloud
    xyz, _ = object_cloud(seed=15, n_surface=3000)
    far = np.concatenate([xyz, np.array([[6.0, 6.0, 6.0]], np.float32)])
    for nv in (2, 4):
        p = _params(orc, k=16, beta=3.0, min_vox_count=nv)
        r = orc.denoise(far, p)
        assert r["stage"][-1] == 1 and r["mask"][-1] == 0


def test_dense_uniform_patch_kept(orc):
    # A 16^3 lattice (spacing a, tiny jitter) splits into eight 8^3 leaves at cap 512.
    # Per leaf H = 7a, V/N = 343a^3/512, (V/N)^(1/3) = 0.875a; beta = 2.2 gives
    # h = 1.925a, so x/h = 0, .52, 1.04, 1.56, 2.08, 2.60, 3.12, 3.64 (in a units):
    # every voxel holds 2 x 2 x 2 = 8 >= n_v points.  q = 0 keeps every density and
    # tau far below the scores keeps every point: the whole patch survives.
    rng = np.random.default_rng(16)
    a = 0.01
    g = np.arange(16) * a
    xyz = np.stack(np.meshgrid(g, g, g, indexing="ij"), -1).reshape(-1, 3)
    xyz = (xyz + rng.normal(scale=1e-5, size=xyz.shape)).astype(np.float32)
    p = _params(orc, k=12, beta=2.2, min_vox_count=4, rho_percentile=0.0,
                select_mode=1, tau=-50.0, leaf_capacity=512)
    r = orc.denoise(xyz, p, debug=True)
    assert r["n_leaves"] == 8 and np.all(r["leaf_count"] == 512)
    assert np.all(r["vox_count"] == 8)
    assert r["mask"].all()


def test_topratio_keeps_ceil_lambda_best_per_leaf(orc):
    from synth import object_cloud
    xyz, _ = object_cloud(seed=17, n_surface=5000)
    lam = 0.8
    p = _params(orc, k=12, beta=3.0, leaf_capacity=300, lam=lam)
    r = orc.denoise(xyz, p, debug=True)
    for L in range(r["n_leaves"]):
        inleaf = r["leaf_of"] == L
        scored = inleaf & ((r["stage"] == 0) | (r["stage"] == 3))
        m = int(scored.sum())
        assert m == r["leaf_n2"][L]
        kept = inleaf & (r["stage"] == 0)
        assert kept.sum() == int(np.ceil(np.float64(np.float32(lam)) * m))
        if kept.any() and (scored & ~kept).any():
            assert r["score"][kept].min() >= r["score"][scored & ~kept].max()


def test_empty_and_degenerate_inputs(orc):
    p = _params(orc, k=8)
    r = orc.denoise(np.zeros((0, 3), np.float32), p, debug=True)
    assert r["mask"].size == 0 and r["n_leaves"] == 0
    same = np.ones((700, 3), np.float32)           # all points identical
    r = orc.denoise(same, _params(orc, k=8, leaf_capacity=64), debug=True)
    assert r["root"][3] == 1.0 and r["n_leaves"] == 1 and r["leaf_level"][0] == 21
    assert np.all(r["vox_count"] == 700)
    # r_K = 0 for duplicates: reading R7 floors r_K^2 at delta^2 = (1 * 2^-21)^2
    assert np.all(r["r2"] == np.float32(2.0 ** -42))
    assert np.allclose(r["rho"], 8 / (4 / 3 * np.pi * 2.0 ** -63), rtol=1e-12)
    assert r["mask"].sum() == int(np.ceil(np.float64(np.float32(0.95)) * 700))


def test_invalid_inputs_rejected(orc):
    bad = np.array([[0, 0, 0], [np.nan, 0, 0]], np.float32)
    with pytest.raises(orc.OracleError) as e:
        orc.denoise(bad, _params(orc))
    assert e.value.status == orc.ENONFINITE
    for kw in (dict(k=0), dict(k=65), dict(beta=0.0), dict(lam=0.0), dict(lam=1.5),
               dict(rho_percentile=101.0), dict(gamma=0.0), dict(sigma=-1.0)):
        with pytest.raises(orc.OracleError) as e:
            orc.denoise(np.zeros((4, 3), np.float32), _params(orc, **kw))
        assert e.value.status == orc.EINVAL


# --------------------------------------------------------------------------
# differentiable form (reading R12): gradient vs FP64 central differences
# --------------------------------------------------------------------------
def _loss_at(orc, xyz, base, noise, subset, field, value):
    kw = dict(base.__dict__)
    kw[field] = value
    p = orc.Params(**kw)
    return orc.softf1(xyz, p, noise, subset)[0]


def test_softf1_gradient_matches_central_differences(orc):
    from synth import object_cloud
    xyz, lab = object_cloud(seed=18, n_surface=3000)
    noise = (lab != 0).astype(np.uint8)
    base = orc.Params(k=12, beta=3.0, select_mode=1, tau=7.5, alpha=1.0, sigma=1.0,
                      gamma=2.0, temperature=0.5)
    subset = (np.random.default_rng(19).uniform(size=len(xyz)) < 0.7).astype(np.uint8)
    loss, grad, rem = orc.softf1(xyz, base, noise, subset)
    # loss is 1 - soft-F1 of the removal probabilities (Eq. 26-28 with soft counts)
    sel = subset.astype(bool)
    want = 1 - 2 * (rem[sel] * noise[sel]).sum() / (rem[sel].sum() + noise[sel].sum())
    assert abs(loss - want) < 1e-12
    h = 1e-4
    for k_, field in enumerate(("alpha", "sigma", "gamma", "tau")):
        v = getattr(base, field)
        # parameters are FP32: divide by the step that was actually taken
        step = float(np.float32(v + h)) - float(np.float32(v - h))
        fd = (_loss_at(orc, xyz, base, noise, subset, field, v + h)
              - _loss_at(orc, xyz, base, noise, subset, field, v - h)) / step
        assert abs(grad[k_] - fd) <= 1e-4 * max(abs(fd), 1e-8), (field, grad[k_], fd)


def test_f1_metric_definitions_bruteforce():
    # Eq. 26-28 on a hand-countable example: 10 points, 4 noise, 5 removed of
    # which 3 noise -> P = 3/5, R = 3/4, F1 = 2PR/(P+R) = 2*3/(5+4) = 2/3
    from paper_2512_10386_gb300.metrics import precision_recall_f1
    noise = np.array([1, 1, 1, 1, 0, 0, 0, 0, 0, 0], bool)
    keep = np.array([0, 0, 0, 1, 0, 0, 1, 1, 1, 1], bool)
    P, R, F1 = precision_recall_f1(keep, noise)
    assert (P, R) == (3 / 5, 3 / 4) and abs(F1 - 2 / 3) < 1e-15


# --------------------------------------------------------------------------
# evaluation metrics (Sec. 4.1, Eq. 29-30)
# --------------------------------------------------------------------------
def test_nn_distances_match_kdtree(orc):
    spatial = pytest.importorskip("scipy.spatial")
    rng = np.random.default_rng(31)
    a = rng.normal(size=(700, 3)).astype(np.float32)
    b = (rng.normal(size=(500, 3)) * 1.3 + 0.2).astype(np.float32)
    got = orc.nn_d2(a, b)
    d, _ = spatial.cKDTree(b.astype(np.float64)).query(a.astype(np.float64), k=1)
    assert np.allclose(got, d ** 2, rtol=1e-12, atol=0)


def test_metrics_hand_worked(orc):
    # A = {(0,0,0), (1,0,0)}, B = {(0,0,0)}: A->B squared distances 0 and 1 (mean 0.5),
    # B->A 0; CD = 0.5; M = bbox diagonal of A = 1, PSNR = 10 log10(1 / 0.5)
    a = np.array([[0, 0, 0], [1, 0, 0]], np.float32)
    b = np.array([[0, 0, 0]], np.float32)
    m = orc.metrics(a, b)
    assert m["mse"] == 0.5 and m["chamfer"] == 0.5
    assert abs(m["psnr"] - 10 * np.log10(2.0)) < 1e-12
    # the Chamfer distance is symmetric; the MSE is not (it averages over the clean cloud)
    m2 = orc.metrics(b, a)
    assert m2["chamfer"] == 0.5 and m2["mse"] == 0.0


def test_metrics_translated_lattice_closed_form(orc):
    # a lattice of spacing 1 and a copy shifted by t (|t| < 1/2): each point's nearest
    # neighbour is its own shifted copy, so MSE = |t|^2, CD = 2|t|^2 and
    # PSNR = 10 log10(diag^2 / |t|^2) with diag^2 = 3 * 9^2 for a 10 x 10 x 10 lattice
    g = np.arange(10, dtype=np.float32)
    a = np.stack(np.meshgrid(g, g, g, indexing="ij"), -1).reshape(-1, 3)
    t = np.array([0.125, -0.25, 0.0625], np.float32)     # exact in FP32
    b = a + t
    t2 = float((t.astype(np.float64) ** 2).sum())
    m = orc.metrics(a, b)
    assert abs(m["mse"] - t2) < 1e-15 and abs(m["chamfer"] - 2 * t2) < 1e-15
    assert abs(m["psnr"] - 10 * np.log10(3 * 81 / t2)) < 1e-9
    same = orc.metrics(a, a)
    assert same["chamfer"] == 0.0 and np.isinf(same["psnr"])


# --------------------------------------------------------------------------
# the gravitational-function baseline (Sec. 2.2, Eq. 1-9)
# --------------------------------------------------------------------------
def test_baseline_hand_worked_lattice(orc):
    # 3 x 3 x 3 lattice, spacing 1: centroid = centre point, H = (2, 2, 2),
    # R = 6 (4 + 4 + 4) / 27 = 8/3 (Eq. 3), T = 600 G 6 / 27 (Eq. 7).  Keep iff
    # G n / d^2 >= T / d, i.e. n >= (600 * 6 / 27) d = 133.3 d: only the centre
    # (d = 0, F infinite) survives, since n <= 27.
    g = np.arange(3, dtype=np.float32)
    xyz = np.stack(np.meshgrid(g, g, g, indexing="ij"), -1).reshape(-1, 3)
    r = orc.baseline(xyz)
    assert abs(r["R"] - 8.0 / 3.0) < 1e-15
    assert abs(r["T"] - 600 * 6.67e-11 * 6 / 27) < 1e-24
    centre = int(np.where((xyz == 1).all(1))[0][0])
    assert r["keep"][centre] == 1 and r["keep"].sum() == 1
    # n_i: lattice points within 8/3 of each point (the point itself included), counted by hand
    # per offset class: |dx|,|dy|,|dz| in {0,1,2} with dx^2+dy^2+dz^2 <= 64/9 (7.1): all but
    # offsets with two or more 2s (8, 12) -> the centre sees all 27, a corner sees 27 - 7 = 20
    corner = int(np.where((xyz == 0).all(1))[0][0])
    assert r["n_i"][centre] == 27 and r["n_i"][corner] == 20
    assert r["d_i"][corner] == np.sqrt(3.0)


def test_baseline_counts_match_kdtree_and_threshold_rule(orc):
    spatial = pytest.importorskip("scipy.spatial")
    # a dense Gaussian cluster in sparse uniform noise, at a scale where Eq. 3's
    # radius (not scale-free: an area over a count) separates the two
    rng = np.random.default_rng(21)
    xyz = np.concatenate([rng.normal(size=(3000, 3)) * 2.0, rng.uniform(-8, 8, size=(300, 3))]).astype(np.float32)
    r = orc.baseline(xyz)
    tree = spatial.cKDTree(xyz.astype(np.float64))
    want = np.array([len(v) for v in tree.query_ball_point(xyz.astype(np.float64), r=r["R"])])
    assert np.array_equal(r["n_i"], want)
    theta = xyz.astype(np.float64).mean(0)
    assert np.allclose(r["d_i"], np.linalg.norm(xyz - theta, axis=1), rtol=1e-12)
    H = xyz.max(0).astype(np.float64) - xyz.min(0).astype(np.float64)
    assert abs(r["R"] - 6 * (H[0] * H[1] + H[0] * H[2] + H[1] * H[2]) / len(xyz)) <= 1e-12 * r["R"]
    # Eq. 8 with G cancelled: keep iff n_i >= alpha (Hx + Hy + Hz) d_i / N
    rhs = 600.0 * H.sum() * r["d_i"] / len(xyz)
    clear = np.abs(r["n_i"] - rhs) > 1e-6 * rhs
    assert np.array_equal(r["keep"][clear].astype(bool), (r["n_i"] >= rhs)[clear])
    assert r["keep"][:3000].mean() > 0.5 and r["keep"][3000:].mean() < 0.1   # cluster kept, noise removed


def test_baseline_translation_and_permutation_invariance(orc):
    from synth import object_cloud
    xyz, _ = object_cloud(seed=22, n_surface=2000)
    xyz = np.round(xyz * 64).astype(np.float32)                 # integer coordinates: translations stay exact
    r = orc.baseline(xyz)
    moved = orc.baseline(xyz + np.float32(1024.0))
    assert np.array_equal(r["keep"], moved["keep"]) and np.array_equal(r["n_i"], moved["n_i"])
    perm = np.random.default_rng(23).permutation(len(xyz))
    rp = orc.baseline(xyz[perm])
    assert np.array_equal(rp["keep"], r["keep"][perm]) and np.array_equal(rp["n_i"], r["n_i"][perm])


# --------------------------------------------------------------------------
# structural variants (Sec. 4.3.2, Tables 8-9; reading R13), each against an
# equivalent configuration of the full method
# --------------------------------------------------------------------------
def _variant_cloud():
    from synth import object_cloud
    xyz, _ = object_cloud(seed=24, n_surface=4000)
    return xyz


def test_without_voxel_gate_equals_occupancy_one(orc):
    xyz = _variant_cloud()
    off = orc.denoise(xyz, _params(orc, k=12, beta=3.0, stage_off=1))
    nv1 = orc.denoise(xyz, _params(orc, k=12, beta=3.0, min_vox_count=1))   # every voxel holds >= 1 point
    assert not (off["stage"] == 1).any()
    assert np.array_equal(off["stage"], nv1["stage"]) and np.array_equal(off["score"], nv1["score"])


def test_without_density_gate_equals_percentile_zero(orc):
    xyz = _variant_cloud()
    p = dict(k=12, beta=3.0, leaf_capacity=256)
    off = orc.denoise(xyz, _params(orc, stage_off=2, **p), debug=True)
    q0 = orc.denoise(xyz, _params(orc, rho_percentile=0.0, **p), debug=True)
    assert not (off["leaf_n1"] == 1).any()              # no leaf with a single point of P_1
    assert np.array_equal(off["stage"], q0["stage"]) and np.array_equal(off["score"], q0["score"])
    full = orc.denoise(xyz, _params(orc, rho_percentile=10.0, **p))
    assert (full["stage"] == 2).any() and not (off["stage"] == 2).any()


def test_without_score_keeps_p2(orc):
    xyz = _variant_cloud()
    p = dict(k=12, beta=3.0)
    off = orc.denoise(xyz, _params(orc, stage_off=4, **p))
    lam1 = orc.denoise(xyz, _params(orc, lam=1.0, **p))                   # Top-lambda with lambda = 1 keeps P_2
    assert np.array_equal(off["mask"], lam1["mask"]) and not off["score"].any()
    only_a1 = orc.denoise(xyz, _params(orc, stage_off=6, **p))             # A1 alone (Table 9 "OnlyA1")
    assert np.array_equal(only_a1["mask"], lam1["stage"] != 1) and not (only_a1["stage"] == 2).any()
    none = orc.denoise(xyz, _params(orc, stage_off=7, **p))
    assert none["mask"].all()


def test_rescore_on_p2_equals_scoring_p2_alone(orc):
    # one leaf, voxel gate passing every point: the kNN recomputed within P_2 for
    # the score is the kNN of the cloud made of P_2 alone, scored without a gate
    rng = np.random.default_rng(25)
    xyz = np.concatenate([rng.normal(size=(600, 3)), rng.uniform(-4, 4, size=(40, 3))]).astype(np.float32)
    base = dict(k=10, min_vox_count=1, leaf_capacity=4096, rho_percentile=8.0)
    r = orc.denoise(xyz, _params(orc, rescore_p2=1, **base))
    p2 = r["stage"] != 2
    assert 0 < (~p2).sum() < len(xyz)
    alone = orc.denoise(np.ascontiguousarray(xyz[p2]), _params(orc, stage_off=2, **base))
    assert np.array_equal(r["stage"][p2], alone["stage"])
    assert np.allclose(r["score"][p2], alone["score"], rtol=1e-12, atol=0)
    # with nothing removed by the gate, rescoring changes nothing
    same = dict(base, rho_percentile=0.0)
    assert np.array_equal(orc.denoise(xyz, _params(orc, rescore_p2=1, **same))["score"],
                          orc.denoise(xyz, _params(orc, **same))["score"])


def test_without_octree_is_one_leaf(orc):
    xyz = _variant_cloud()
    p = dict(k=12, beta=3.0)
    flat = orc.denoise(xyz, _params(orc, leaf_capacity=0xFFFFFFFF, **p), debug=True)
    d0 = orc.denoise(xyz, _params(orc, max_depth=0, **p), debug=True)
    assert flat["n_leaves"] == 1 and flat["leaf_count"][0] == len(xyz)
    assert np.array_equal(flat["stage"], d0["stage"]) and np.array_equal(flat["score"], d0["score"])


# --------------------------------------------------------------------------
# cross-leaf kNN (reading R14): candidates from the 27 same-level cells around a leaf
# --------------------------------------------------------------------------
def test_cross_leaf_equals_global_knn_when_cells_hold_the_neighbourhood(orc):
    # a jittered 16^3 lattice cut into 4^3-point leaves: every point's 8 nearest lie
    # within one lattice spacing and a half, inside the 27 cells around its leaf, so
    # the cross-leaf kNN is the global kNN (full sort over the whole cloud) -- which
    # the leaf-local kNN is not, for the points on a leaf's border
    rng = np.random.default_rng(26)
    g = np.arange(16, dtype=np.float64)
    xyz = np.stack(np.meshgrid(g, g, g, indexing="ij"), -1).reshape(-1, 3)
    xyz = (xyz + rng.uniform(-0.2, 0.2, size=xyz.shape)).astype(np.float32)
    p = dict(k=8, min_vox_count=1, leaf_capacity=64, rho_percentile=0.0)
    r = orc.denoise(xyz, _params(orc, cross_leaf=1, **p), debug=True)
    assert r["n_leaves"] == 64
    d2 = ((xyz[:, None, :].astype(np.float64) - xyz[None, :, :]) ** 2).sum(-1)
    np.fill_diagonal(d2, np.inf)
    want = np.argsort(d2, axis=1, kind="stable")[:, :8]
    assert all(set(a) == set(b) for a, b in zip(r["nbr"], want))
    local = orc.denoise(xyz, _params(orc, **p), debug=True)
    assert sum(set(a) != set(b) for a, b in zip(local["nbr"], want)) > 500


def test_cross_leaf_equals_leaf_local_for_a_single_leaf(orc):
    # with the root as the only leaf the 27-cell block is the root cell: nothing changes
    from synth import object_cloud
    xyz, _ = object_cloud(seed=27, n_surface=2500)
    for kw in (dict(max_depth=0), dict(leaf_capacity=0xFFFFFFFF)):
        p = dict(k=12, beta=3.0, rho_percentile=5.0, **kw)
        a = orc.denoise(xyz, _params(orc, **p))
        b = orc.denoise(xyz, _params(orc, cross_leaf=1, **p))
        assert np.array_equal(a["stage"], b["stage"]) and np.array_equal(a["score"], b["score"])
        for mode in (dict(select_mode=1, tau=4.0),):
            a = orc.denoise(xyz, _params(orc, **p, **mode))
            b = orc.denoise(xyz, _params(orc, cross_leaf=1, **p, **mode))
            assert np.array_equal(a["stage"], b["stage"])
