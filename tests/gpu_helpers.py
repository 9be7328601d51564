"""Shared comparison logic of the GPU parity tests (CUDA path vs FP64 oracle)."""

import numpy as np

SCORE_RTOL = 1e-5   # tolerance for scores (FP32 GPU vs FP64 oracle), relative


def oracle_params(P):
    import oracle
    return oracle.Params(k=P.k, leaf_capacity=P.leaf_capacity, max_depth=P.max_depth, beta=P.beta,
                         min_vox_count=P.min_vox_count, rho_percentile=P.rho_percentile, alpha=P.alpha,
                         sigma=P.sigma, gamma=P.gamma, eps_rho=P.eps_rho, eps_k=P.eps_k,
                         select_mode=P.select_mode, lam=P.lam, tau=P.tau, temperature=P.temperature,
                         stage_off=P.stage_off, rescore_p2=P.rescore_p2, cross_leaf=P.cross_leaf)


def to_np(d):
    return {k: (v.cpu().numpy() if hasattr(v, "cpu") else v) for k, v in d.items()}


def canonical_rows(nbr, d2):
    """Neighbour lists in the method's order, (d^2, input index) ascending, padding
    last.  The kernel emits a fixed but different order (its scan order)."""
    nbr = np.asarray(nbr, np.uint32)
    bits = np.asarray(d2, np.float32).view(np.uint32).astype(np.uint64)
    key = (bits << np.uint64(32)) | nbr.astype(np.uint64)
    key[nbr == 0xFFFFFFFF] = np.iinfo(np.uint64).max
    key = np.sort(key, axis=1)
    return (key & np.uint64(0xFFFFFFFF)).astype(np.uint32), (key >> np.uint64(32)).astype(np.uint32)


def ambiguous_points(ref, P, tol=SCORE_RTOL):
    """Points whose selection may legitimately differ between FP32 and FP64 scores:
    within `tol` of the leaf's Top-lambda cut, or with ln F within `tol` of tau."""
    F = ref["score"]
    st = ref["stage"]
    amb = np.zeros(len(F), bool)
    scored = (st == 0) | (st == 3)
    if P.select_mode == 1:
        with np.errstate(divide="ignore"):
            lf = np.log(np.where(F > 0, F, 1e-300))
        amb = scored & (np.abs(lf - np.float32(P.tau)) <= tol * max(1.0, abs(P.tau)) + 1e-6)
        return amb
    leaf = ref["leaf_of"]
    for L in np.unique(leaf[scored & (st == 3)]):
        inl = (leaf == L) & scored
        kept = inl & (st == 0)
        rem = inl & (st == 3)
        if not kept.any():
            continue
        c_keep = F[kept].min()
        c_rem = F[rem].max()
        band = inl & (F >= c_rem * (1 - 2 * tol)) & (F <= c_keep * (1 + 2 * tol))
        if c_keep <= c_rem * (1 + 2 * tol):
            amb |= band
    return amb


def compare_with_oracle(gpu, ref, P, check_debug=True):
    """Assert parity; return a dict of counts (mask mismatches, ambiguous points)."""
    n = len(ref["mask"])
    K = P.k
    if check_debug:
        assert np.array_equal(gpu["key"].astype(np.uint64), ref["key"]), "Morton keys differ"
        lid = ref["leaf_of"]
        assert np.array_equal(gpu["leaf_start"].astype(np.uint32), ref["leaf_start"][lid]), "leaf partition differs"
        assert np.array_equal(gpu["leaf_count"].astype(np.uint32), ref["leaf_count"][lid]), "leaf sizes differ"
        assert np.array_equal(gpu["leaf_h"].view(np.uint32), ref["leaf_h"][lid].view(np.uint32)), "voxel size h differs"
        assert np.array_equal(gpu["vox_count"].astype(np.uint32), ref["vox_count"]), "voxel counts differ"
    st_g, st_r = gpu["stage"], ref["stage"]
    assert np.array_equal(st_g == 1, st_r == 1), "voxel gate differs"
    assert np.array_equal(st_g == 2, st_r == 2), "density gate differs"
    if check_debug:
        p1 = st_r != 1
        inP1 = p1 & (ref["r2"] > 0)
        assert np.array_equal(gpu["r2"][inP1].view(np.uint32), ref["r2"][inP1].view(np.uint32)), "r_K^2 differs"
        gn, gd = canonical_rows(gpu["nbr"][inP1].astype(np.uint32), gpu["nbr_d2"][inP1])
        rn, rd = canonical_rows(ref["nbr"][inP1], ref["nbr_d2"][inP1])
        assert np.array_equal(gn, rn), "neighbour sets differ"
        assert np.array_equal(gd, rd), "neighbour distances differ"
        scored = (st_r == 0) | (st_r == 3)
        rm_r = ref["leaf_rho_med"][ref["leaf_of"]]
        assert np.allclose(gpu["leaf_rho_med"][scored], rm_r[scored], rtol=1e-14, atol=0), "rho_med differs"
    scored = (st_r == 0) | (st_r == 3)
    Fg = gpu["score"].astype(np.float64)
    Fr = ref["score"]
    assert np.all(Fg[~scored] == 0) and np.all(Fr[~scored] == 0)
    if scored.any():
        # a scored point with no neighbour to score with (a variant without the density
        # gate, or a one-point P_2) has F = 0 exactly on both sides
        zero = Fr[scored] == 0
        assert np.all(Fg[scored][zero] == 0), "score of a point without neighbours is not 0"
        rel = np.abs(Fg[scored][~zero] - Fr[scored][~zero]) / np.abs(Fr[scored][~zero])
        max_rel = float(rel.max()) if rel.size else 0.0
        assert max_rel <= SCORE_RTOL, f"score rel err {max_rel:.3e}"
    else:
        max_rel = 0.0
    amb = ambiguous_points(ref, P)
    mism = gpu["mask"] != ref["mask"]
    bad = mism & ~amb
    assert not bad.any(), f"{int(bad.sum())} mask mismatches outside the tolerance band"
    return {"n": n, "mismatch": int(mism.sum()), "ambiguous": int(amb.sum()), "max_score_rel": max_rel}
