"""Autotuner of the batched (graph-captured) path.

It measures a workload under candidate settings and keeps the fastest:
  * leaf_capacity -- the octree's maximum points per leaf.  The paper leaves
    it unstated (Sec. 3), so it is a free method parameter; it changes which
    points share a leaf and therefore the result, so a tuned capacity must be
    used for every path that is compared (oracle, per-frame, batched).
  * leaf_ctas_per_sm -- persistent CTAs of the fused leaf kernel per SM
    (execution only; results do not depend on it).
  * leaf_smem_points -- largest leaf kept in shared memory; larger leaves take
    the kernel's global-memory path, and each CTA needs less shared memory, so
    more CTAs fit per SM (execution only).
  * leaf_threads -- 128 (0) or 64 threads per leaf CTA; 64 leaves fewer warps
    idle on small leaves (execution only).  With 64 the CTA count per SM is
    left at the occupancy limit.
The kNN tile is the whole leaf (it is staged in shared memory at once), so
there is no separate k-tile to tune; the block shape is fixed at compile time.
Results are cached as JSON keyed by (GPU name, K, frame count, size bucket).
"""

from __future__ import annotations

import dataclasses
import itertools
import json
import math
import os
from typing import Iterable, Optional, Sequence

import torch

from . import _native as N
from .api import Denoiser, Params

DEFAULT_CAPACITIES = (128, 192, 256, 384, 512)
DEFAULT_CTAS = (0, 2, 3)
DEFAULT_SMEM_POINTS = (0, 128, 256)
DEFAULT_THREADS = (0, 64)


def _cache_key(params: Params, offsets: Sequence[int]) -> str:
    name = torch.cuda.get_device_name()
    n = int(offsets[-1])
    frames = len(offsets) - 1
    bucket = 2 ** int(math.ceil(math.log2(max(n, 1))))
    return f"{name}|k={params.k}|frames={frames}|points<={bucket}|v3"


def tune_batch(xyz: torch.Tensor, offsets: Sequence[int], params: Params,
               capacities: Iterable[int] = DEFAULT_CAPACITIES, ctas: Iterable[int] = DEFAULT_CTAS,
               smem_points: Iterable[int] = DEFAULT_SMEM_POINTS, threads: Iterable[int] = DEFAULT_THREADS,
               reps: int = 5, cache_path: Optional[str] = None, denoiser: Optional[Denoiser] = None) -> dict:
    """Time ``denoise_run_batch`` (graph mode) for every candidate; return the best
    ``{"leaf_capacity", "leaf_ctas_per_sm", "leaf_smem_points", "leaf_threads", "ms", "table"}``
    (from the cache if present)."""
    key = _cache_key(params, offsets)
    if cache_path and os.path.exists(cache_path):
        with open(cache_path) as f:
            cache = json.load(f)
        if key in cache:
            return cache[key]
    offsets = [int(v) for v in offsets]
    own = denoiser is None
    d = denoiser or Denoiser(max_points=int(offsets[-1]), max_frames=len(offsets) - 1)
    stream = torch.cuda.Stream()
    n = int(offsets[-1])
    mask = torch.empty(n, dtype=torch.uint8, device="cuda")
    score = torch.empty(n, dtype=torch.float32, device="cuda")
    stage = torch.empty(n, dtype=torch.uint8, device="cuda")
    table = []
    try:
        d.set_graphs(True)
        d.set_sync(False)   # enqueue back to back: the events then bracket device work only
        for cap, nt, c, sp in itertools.product(capacities, threads, ctas, smem_points):
            if (nt and c) or (sp and sp >= cap):
                continue  # 64-thread CTAs run at the occupancy limit; sp >= cap is the same as 0
            p = dataclasses.replace(params, leaf_capacity=int(cap))
            d.set_tuning(int(c), int(sp), int(nt))
            d.run_batch(xyz, offsets, p, mask=mask, score=score, stage=stage, stream=stream)  # capture
            d.run_batch(xyz, offsets, p, mask=mask, score=score, stage=stage, stream=stream)
            ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
            ev[0].record(stream)
            for _ in range(reps):
                d.run_batch(xyz, offsets, p, mask=mask, score=score, stage=stage, stream=stream)
            ev[1].record(stream)
            torch.cuda.synchronize()
            N.check(d.status(stream), "denoise_run_batch")
            table.append({"leaf_capacity": int(cap), "leaf_ctas_per_sm": int(c), "leaf_smem_points": int(sp),
                          "leaf_threads": int(nt), "ms": ev[0].elapsed_time(ev[1]) / reps})
    finally:
        d.set_sync(True)
        d.set_graphs(False)
        d.set_tuning(0, 0, 0)
        if own:
            d.close()
    best = min(table, key=lambda r: r["ms"])
    result = dict(best, table=table, key=key)
    if cache_path:
        cache = {}
        if os.path.exists(cache_path):
            with open(cache_path) as f:
                cache = json.load(f)
        cache[key] = result
        os.makedirs(os.path.dirname(os.path.abspath(cache_path)), exist_ok=True)
        with open(cache_path, "w") as f:
            json.dump(cache, f, indent=1)
    return result
