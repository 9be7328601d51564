"""Serving loop: continuous batching of denoising requests on one GPU.

Requests (one point cloud each) arrive over time.  The server keeps a few
execution slots, each a device-resident native context (octree, sort and
neighbour scratch allocated once) with its own CUDA stream and pinned host
staging buffers.  Whenever a slot is free, the server admits waiting
requests in arrival order into it -- as many as fit the slot's point capacity,
the per-batch frame limit and the global in-flight point budget (memory-based
admission) -- and launches them as one asynchronous ``denoise_run_batch``
(host->device copy, kernels, device->host copy, all on the slot's stream).
Requests that arrive while others are on the GPU are admitted as slots and
budget free up, so batches on different slots overlap on the device.
Each frame of a batch is denoised exactly as it would be alone
(``denoise_run_batch`` is segmented per frame), so results do not depend on
the mix.  Latency is measured from a request's arrival to the moment its
result is in host memory.
"""

from __future__ import annotations

import collections
import concurrent.futures
import dataclasses
import os
import statistics
import time
from typing import Callable, Dict, Iterable, List, Optional, Sequence

import numpy as np


@dataclasses.dataclass
class Request:
    rid: int
    t_arrival: float            # seconds from stream start
    xyz: np.ndarray             # float32 [n, 3]
    kind: str = ""


@dataclasses.dataclass
class Completion:
    rid: int
    kind: str
    n: int
    t_arrival: float
    t_admit: float
    t_done: float
    slot: int
    batch_size: int
    mask: np.ndarray
    score: np.ndarray
    stage: np.ndarray

    @property
    def latency(self) -> float:
        return self.t_done - self.t_arrival


_STAGE_CHUNK_ROWS = 1 << 16   # rows (768 KB of xyz) per piece of a parallel staging copy


def _stage_pieces(pieces, pool, threads: int) -> None:
    """Copy (dst, src) array pairs; pieces above _STAGE_CHUNK_ROWS rows are split
    into at most `threads` row ranges spread over `pool` (numpy releases the GIL
    for a plain copy of one dtype, so the threads copy in parallel).  A dense
    frame of ~1 M points is ~13 MB: on one thread the copy alone takes about as
    long as the frame's device work, and it runs on the server's only control
    thread."""
    jobs = []
    for dst, src in pieces:
        n = len(src)
        if pool is None or n <= _STAGE_CHUNK_ROWS:
            np.copyto(dst, src)
            continue
        nch = min(threads, -(-n // _STAGE_CHUNK_ROWS))
        step = -(-n // nch)
        for a in range(0, n, step):
            b = min(n, a + step)
            jobs.append(pool.submit(np.copyto, dst[a:b], src[a:b]))
    for j in jobs:
        j.result()


class _Slot:
    """One execution slot: a native context, a stream, pinned staging."""

    def __init__(self, index: int, capacity: int, max_frames: int, params, device=None, pool=None, threads: int = 1):
        import torch

        from .api import Denoiser
        self.index = index
        self.capacity = capacity
        self.max_frames = max_frames
        self.params = params
        self.den = Denoiser(max_points=capacity, max_frames=max_frames, device=device)
        self.den.set_sync(False)
        self.stream = torch.cuda.Stream(device=self.den.device)
        self.xyz = torch.empty((capacity, 3), dtype=torch.float32).pin_memory()
        self.mask = torch.empty(capacity, dtype=torch.uint8).pin_memory()
        self.score = torch.empty(capacity, dtype=torch.float32).pin_memory()
        self.stage = torch.empty(capacity, dtype=torch.uint8).pin_memory()
        self.event = torch.cuda.Event()
        self.batch: Optional[List[Request]] = None
        self.offsets: List[int] = []
        self.t_admit = 0.0
        self.pool, self.threads = pool, threads

    def launch(self, batch: List[Request], t_admit: float):
        offs = [0]
        xv = self.xyz.numpy()
        pieces = []
        for r in batch:
            n = len(r.xyz)
            pieces.append((xv[offs[-1]:offs[-1] + n], np.asarray(r.xyz, dtype=np.float32).reshape(n, 3)))
            offs.append(offs[-1] + n)
        _stage_pieces(pieces, self.pool, self.threads)
        total = offs[-1]
        self.den.run_batch(self.xyz[:total], offs, self.params, mask=self.mask[:total], score=self.score[:total],
                           stage=self.stage[:total], stream=self.stream)
        self.event.record(self.stream)
        self.batch, self.offsets, self.t_admit = batch, offs, t_admit

    def done(self) -> bool:
        return self.batch is not None and self.event.query()

    def collect(self, t_done: float, keep_results: bool = True) -> List[Completion]:
        from . import _native as N
        st = self.den.status(self.stream)
        if st != N.DENOISE_OK:
            raise N.DenoiseError(st, "serving batch")
        out = []
        if keep_results:  # the batch's results out of the pinned buffers, in one parallel copy
            total = self.offsets[-1]
            m, sc, sg = np.empty(total, np.uint8), np.empty(total, np.float32), np.empty(total, np.uint8)
            _stage_pieces([(m, self.mask[:total].numpy()), (sc, self.score[:total].numpy()),
                           (sg, self.stage[:total].numpy())], self.pool, self.threads)
        for i, r in enumerate(self.batch):
            a, b = self.offsets[i], self.offsets[i + 1]
            res = (m[a:b], sc[a:b], sg[a:b]) if keep_results else (None, None, None)
            out.append(Completion(r.rid, r.kind, b - a, r.t_arrival, self.t_admit, t_done, self.index,
                                  len(self.batch), *res))
        self.batch = None
        return out

    def close(self):
        self.den.close()


class Scheduler:
    """Admission policy (host logic, no GPU): FIFO, memory budget, slot fit."""

    def __init__(self, capacities: Sequence[int], max_frames: int, budget_points: int):
        self.capacities = list(capacities)
        self.max_frames = max_frames
        self.budget = budget_points
        self.in_flight = 0

    def admit(self, queue: collections.deque, free_slots: Sequence[int]) -> Dict[int, list]:
        """Pop requests from the head of `queue` into free slots; returns {slot: [requests]}.
        A request larger than every slot's capacity is an error."""
        plan: Dict[int, list] = {}
        for s in sorted(free_slots, key=lambda i: self.capacities[i]):
            if not queue:
                break
            head = queue[0]
            n0 = len(head.xyz)
            if n0 > max(self.capacities):
                raise ValueError(f"request {head.rid} has {n0} points, above every slot's capacity")
            if n0 > self.capacities[s]:
                continue
            if self.in_flight + n0 > self.budget:
                break
            batch, pts = [], 0
            while queue and len(batch) < self.max_frames:
                n = len(queue[0].xyz)
                if pts + n > self.capacities[s] or self.in_flight + pts + n > self.budget:
                    break
                batch.append(queue.popleft())
                pts += n
            if batch:
                plan[s] = batch
                self.in_flight += pts
        return plan

    def release(self, points: int):
        self.in_flight -= points


class Server:
    """Continuous-batching denoising server on one GPU."""

    def __init__(self, params, capacities: Sequence[int], max_frames: int = 8,
                 budget_points: Optional[int] = None, device=None, copy_threads: Optional[int] = None):
        """copy_threads: host threads for staging request points into the slots'
        pinned buffers (default: half the host cores, at most 8; 0 or 1 = copy
        on the calling thread)."""
        self.params = params
        if copy_threads is None:
            copy_threads = max(1, min(8, (os.cpu_count() or 2) // 2))
        self.pool = concurrent.futures.ThreadPoolExecutor(copy_threads) if copy_threads > 1 else None
        self.slots = [_Slot(i, c, max_frames, params, device, self.pool, copy_threads)
                      for i, c in enumerate(capacities)]
        self.sched = Scheduler(capacities, max_frames, budget_points or sum(capacities))

    def close(self):
        for s in self.slots:
            s.close()
        if self.pool is not None:
            self.pool.shutdown()
            self.pool = None

    def serve(self, requests: Iterable[Request], realtime: bool = True, clock: Callable[[], float] = time.perf_counter,
              idle_sleep: float = 2e-4, keep_results: bool = True) -> List[Completion]:
        """Play `requests` (in arrival order) through the server.  With
        realtime=True a request becomes visible at its arrival time; otherwise
        all are visible at once (throughput mode, arrival = start).  `requests`
        may be a list or a lazy iterator (each request is drawn when its arrival
        time comes, so a long stream need not be held in memory); with
        keep_results=False the completions carry no per-point arrays."""
        if isinstance(requests, (list, tuple)):
            requests = sorted(requests, key=lambda r: r.t_arrival)
        source = iter(requests)
        nxt = next(source, None)
        queue: collections.deque = collections.deque()
        done: List[Completion] = []
        t0 = clock()
        while nxt is not None or queue or any(s.batch is not None for s in self.slots):
            now = clock() - t0
            while nxt is not None and (not realtime or nxt.t_arrival <= now):
                if not realtime:
                    nxt.t_arrival = 0.0
                queue.append(nxt)
                nxt = next(source, None)
                if not realtime and len(queue) >= 4 * len(self.slots) * self.sched.max_frames:
                    break                                    # throughput mode: a bounded look-ahead
            progressed = False
            for s in self.slots:
                if s.done():
                    comps = s.collect(clock() - t0, keep_results)
                    self.sched.release(sum(c.n for c in comps))
                    done.extend(comps)
                    progressed = True
            free = [s.index for s in self.slots if s.batch is None]
            if queue and free:
                for si, batch in self.sched.admit(queue, free).items():
                    self.slots[si].launch(batch, clock() - t0)
                    progressed = True
            if progressed:
                continue
            if any(s.batch is not None for s in self.slots):
                time.sleep(idle_sleep)                       # work in flight: poll again soon
            elif queue:
                raise RuntimeError(f"request {queue[0].rid} cannot be admitted (point budget too small)")
            elif nxt is not None:
                time.sleep(min(max(nxt.t_arrival - (clock() - t0), 0.0), 0.01))
        return sorted(done, key=lambda c: c.rid)


def latency_report(comps: Sequence[Completion], wall_s: float) -> dict:
    lat = sorted(c.latency * 1000.0 for c in comps)
    pts = sum(c.n for c in comps)

    def pct(p):
        return lat[min(len(lat) - 1, int(round(p / 100.0 * (len(lat) - 1))))]

    return {"frames": len(comps), "points": pts, "wall_s": wall_s, "points_per_s": pts / wall_s,
            "latency_ms_p50": pct(50), "latency_ms_p99": pct(99), "latency_ms_mean": statistics.mean(lat),
            "mean_batch_frames": statistics.mean(c.batch_size for c in comps)}
