"""The serving and differentiation workloads at their stated sizes.

- Serving stream (Poisson 20 Hz, seed 7): one dense 128-beam frame (~1.1 M
  points with 10 % uniform outliers) and one sparse 32-beam frame (~118 k with
  15 % snow), K = 24, compared with the FP64 oracle element by element like
  the other parity tests (bit-exact keys, leaves, h, voxel counts, gates,
  neighbour sets and r_K^2; scores within 1e-5; masks identical outside the
  tolerance band).
- Differentiation: the 16 labelled frames of the dense-scan generator (seeds
  100-115, 560,000 points each), THRESHOLD form with T = 0.05 and a soft-F1
  loss over a seeded 2,000-point subset of each frame's scored points: the
  GPU gradient with respect to (alpha, sigma, gamma, tau) against the oracle's
  analytic gradient and against FP64 central differences (h = 1e-4) of the
  oracle's loss, within 1e-4 relative.  The oracle runs in a spawned process
  pool (one frame per worker).
"""

import multiprocessing as mp
import os

import numpy as np
import pytest

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

torch = pytest.importorskip("torch")

from gpu_helpers import compare_with_oracle, oracle_params, to_np  # noqa: E402

FIELDS = ("alpha", "sigma", "gamma", "tau")


@pytest.fixture(scope="module")
def env():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__
    __graft_entry__.build()
    import oracle
    oracle.build()
    return oracle


def _first(stream, kind):
    return next(r for r in stream.requests if r.kind == kind)


@pytest.mark.parametrize("kind", ["dense", "sparse"])
def test_serving_stream_frame_parity(env, kind):
    orc = env
    import synth
    from paper_2512_10386_gb300 import Denoiser, Params
    stream = synth.serving_stream(seed=7)
    xyz, _ = stream.frame(_first(stream, kind))
    assert (len(xyz) > 1_000_000) if kind == "dense" else (100_000 < len(xyz) < 140_000)
    P = Params(k=24)
    d = Denoiser(max_points=len(xyz))
    try:
        g = to_np(d.run_debug(torch.from_numpy(xyz).cuda(), P))
    finally:
        d.close()
    r = orc.denoise(xyz, oracle_params(P), debug=True)
    stats = compare_with_oracle(g, r, P)
    print(f"serving {kind} frame ({len(xyz)} points):", stats)


def _c4_frame(seed):
    import synth
    xyz, lab = synth.superquadric_scan(seed=seed)
    return xyz, (lab != 0).astype(np.uint8)


def _c4_params():
    from paper_2512_10386_gb300 import Params
    return Params(k=32, select_mode=1, tau=9.0, temperature=0.05, alpha=1.0, sigma=1.0, gamma=2.0)


def _c4_oracle(seed):
    """Worker: the oracle's loss, analytic gradient and central differences for one frame."""
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    if root not in sys.path:
        sys.path.insert(0, root)
    import oracle
    from gpu_helpers import oracle_params as op
    xyz, noise = _c4_frame(seed)
    base = op(_c4_params())
    ref = oracle.denoise(xyz, base)
    scored = np.where((ref["stage"] == 0) | (ref["stage"] == 3))[0]
    pick = np.random.default_rng(seed).choice(scored, size=2000, replace=False)
    subset = np.zeros(len(xyz), np.uint8)
    subset[pick] = 1
    loss, grad, _ = oracle.softf1(xyz, base, noise, subset)
    h = 1e-4
    fd = []
    for f in FIELDS:
        v = getattr(base, f)
        step = float(np.float32(v + h)) - float(np.float32(v - h))
        vals = []
        for x in (v + h, v - h):
            kw = dict(base.__dict__)
            kw[f] = x
            vals.append(oracle.softf1(xyz, oracle.Params(**kw), noise, subset)[0])
        fd.append((vals[0] - vals[1]) / step)
    return seed, subset, loss, np.asarray(grad), np.asarray(fd)


def test_gradients_on_the_sixteen_labelled_frames(env):
    from paper_2512_10386_gb300 import Denoiser, SoftRemoval, soft_f1_loss
    seeds = list(range(100, 116))
    workers = max(1, min(len(seeds), os.cpu_count() or 1))
    ctx = mp.get_context("spawn")
    with ctx.Pool(workers) as pool:
        pending = pool.map_async(_c4_oracle, seeds)
        P = _c4_params()
        d = Denoiser(max_points=560_000)
        gpu = {}
        try:
            for s in seeds:
                xyz, noise = _c4_frame(s)
                gpu[s] = (xyz, noise)
            results = pending.get(timeout=3000)
            worst = [0.0] * 4
            for seed, subset, loss_o, g_o, fd in results:
                xyz, noise = gpu[seed]
                theta = torch.tensor([P.alpha, P.sigma, P.gamma, P.tau], dtype=torch.float64, requires_grad=True)
                r = SoftRemoval.apply(torch.from_numpy(xyz).cuda(), theta, d, P)
                sel = torch.from_numpy(subset.astype(bool)).cuda()
                loss = soft_f1_loss(r, torch.from_numpy(noise).cuda(), sel)
                loss.backward()
                g = theta.grad.numpy()
                assert abs(float(loss.detach()) - loss_o) <= 1e-6 * max(1.0, abs(loss_o)), seed
                for k in range(4):
                    assert abs(g_o[k] - fd[k]) <= 1e-4 * abs(fd[k]), (seed, FIELDS[k], g_o[k], fd[k])
                    assert abs(g[k] - fd[k]) <= 1e-4 * abs(fd[k]), (seed, FIELDS[k], g[k], fd[k])
                    worst[k] = max(worst[k], abs(g[k] - fd[k]) / abs(fd[k]))
            print("16 frames: worst GPU-vs-FD relative error per parameter", dict(zip(FIELDS, worst)))
        finally:
            d.close()
