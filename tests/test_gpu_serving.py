"""Serving on the GPU: every result is the same alone and in the mix.

A compressed Poisson stream of mixed-size frames is played through the
continuous-batching server (several slots, multi-frame batches, overlapping
work, frames large enough for the parallel staging copy); each completion must
equal the frame's solo denoise_run result bit for bit, and the test checks that
batches did overlap in time.
"""

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def test_results_identical_alone_and_in_the_mix():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__
    __graft_entry__.build()
    import synth
    from paper_2512_10386_gb300 import Denoiser, Params
    from paper_2512_10386_gb300.serving import Request, Server, latency_report

    rng = np.random.default_rng(7)
    reqs, t = [], 0.0
    for i in range(16):
        t += rng.exponential(1 / 400.0)           # 400 Hz: arrivals overlap with work in flight
        n_surface = int(rng.choice([2000, 6000, 15000, 40000]))
        xyz, _ = synth.object_cloud(seed=200 + i, n_surface=n_surface)
        reqs.append(Request(i, t, xyz, kind=str(n_surface)))
    # two frames above the staging copy's chunk size (their points and results move in row ranges on the copy threads)
    for i in (16, 17):
        t += rng.exponential(1 / 400.0)
        xyz, _ = synth.object_cloud(seed=200 + i, n_surface=90000)
        reqs.append(Request(i, t, xyz, kind="90000"))
    P = Params(k=16)
    srv = Server(P, capacities=[50_000, 50_000, 120_000], max_frames=4)
    try:
        import time
        t0 = time.perf_counter()
        comps = srv.serve(reqs, realtime=True)
        rep = latency_report(comps, time.perf_counter() - t0)
    finally:
        srv.close()
    assert [c.rid for c in comps] == list(range(18))
    d = Denoiser(max_points=120_000)
    try:
        for c, r in zip(comps, reqs):
            solo = d.run(torch.from_numpy(r.xyz).cuda(), P)
            assert np.array_equal(c.mask, solo.mask.cpu().numpy()), c.rid
            assert np.array_equal(c.score, solo.score.cpu().numpy()), c.rid
            assert np.array_equal(c.stage, solo.stage.cpu().numpy()), c.rid
    finally:
        d.close()
    # work overlapped: some batch was admitted before another one finished
    spans = sorted({(c.t_admit, c.t_done, c.slot) for c in comps})
    overlap = any(a2 < d1 and s1 != s2 for (a1, d1, s1) in spans for (a2, d2, s2) in spans if a2 > a1)
    assert overlap or rep["mean_batch_frames"] > 1.0
    print("serving:", rep)
