"""Host logic of the serving loop (no GPU): admission by slot fit, frame limit,
FIFO order and the in-flight point budget."""

import collections

import numpy as np
import pytest

from paper_2512_10386_gb300.serving import Request, Scheduler, latency_report, Completion


def _req(i, n):
    return Request(i, 0.0, np.zeros((n, 3), np.float32))


def test_admission_fills_slots_fifo_within_capacity_and_frames():
    s = Scheduler([1000, 5000], max_frames=3, budget_points=100_000)
    q = collections.deque([_req(0, 400), _req(1, 400), _req(2, 400), _req(3, 3000), _req(4, 100)])
    plan = s.admit(q, [0, 1])
    # smallest slot first: 0 takes 400+400 (a third 400 would exceed 1000)
    assert [r.rid for r in plan[0]] == [0, 1]
    # slot 1 continues in arrival order: 400 + 3000 + 100 (frame limit 3)
    assert [r.rid for r in plan[1]] == [2, 3, 4]
    assert not q and s.in_flight == 4300


def test_admission_respects_point_budget_and_release():
    s = Scheduler([1000, 1000], max_frames=8, budget_points=1200)
    q = collections.deque([_req(0, 800), _req(1, 800)])
    plan = s.admit(q, [0, 1])
    assert list(plan) == [0] and [r.rid for r in plan[0]] == [0]
    assert [r.rid for r in q] == [1]               # waits for memory, order kept
    s.release(800)
    plan = s.admit(q, [1])
    assert [r.rid for r in plan[1]] == [1]


def test_oversized_request_is_rejected():
    s = Scheduler([1000], max_frames=2, budget_points=10_000)
    with pytest.raises(ValueError):
        s.admit(collections.deque([_req(0, 5000)]), [0])


def test_latency_report_percentiles():
    comps = [Completion(i, "x", 10, 0.0, 0.0, (i + 1) / 1000.0, 0, 1, None, None, None) for i in range(100)]
    rep = latency_report(comps, wall_s=1.0)
    assert rep["frames"] == 100 and rep["points"] == 1000
    assert rep["latency_ms_p50"] == pytest.approx(51.0) or rep["latency_ms_p50"] == pytest.approx(50.0)
    assert rep["latency_ms_p99"] == pytest.approx(99.0, abs=1.0)


@pytest.mark.parametrize("threads", [1, 3, 8])
def test_parallel_staging_copy_places_every_row(threads):
    """The slots' staging copy: frames of a batch land back to back, large ones
    split into row ranges over the copy threads, small ones copied whole."""
    import concurrent.futures

    from paper_2512_10386_gb300.serving import _STAGE_CHUNK_ROWS, _stage_pieces
    rng = np.random.default_rng(3)
    sizes = [5, _STAGE_CHUNK_ROWS, _STAGE_CHUNK_ROWS + 1, 3 * _STAGE_CHUNK_ROWS + 17, 0]
    frames = [rng.standard_normal((n, 3)).astype(np.float32) for n in sizes]
    dst = np.full((sum(sizes) + 4, 3), np.nan, dtype=np.float32)
    offs = np.cumsum([0] + sizes)
    pool = concurrent.futures.ThreadPoolExecutor(threads) if threads > 1 else None
    try:
        _stage_pieces([(dst[offs[i]:offs[i + 1]], f) for i, f in enumerate(frames)], pool, threads)
    finally:
        if pool is not None:
            pool.shutdown()
    assert np.array_equal(dst[:offs[-1]], np.concatenate(frames))
    assert np.isnan(dst[offs[-1]:]).all()              # nothing written past the batch
