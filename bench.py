"""Benchmark: points/s denoised on the dense-scan workload, one JSON line.

Workload (default): one 560,000-point cloud (8 random superquadrics, 0.5 %
surface jitter, 10 % uniform outliers, 2 % in 20 Gaussian blobs; seed 1),
K = 32, leaf capacity 512, the plain per-frame path (denoise_run with device
buffers).  A "step" denoises the whole cloud: bounding cube, Morton keys,
radix sort, octree leaves, voxel gate, kNN + density gate, score, selection.

Timing: W untimed warm-up steps, then K steps, each bracketed by CUDA events on
the library's stream; between timed steps L2 is flushed by writing a 256 MiB
buffer (outside the event pair).  Under torchrun each rank denoises its own
cloud (seed 1 + rank): weak scaling, no collective on the data path; the
reported time is the max over ranks.

Extra objects on the line:
  roofline      the fused leaf kernel (kNN + score), timed live with the
                library's per-stage CUDA events; FP32 work = 8 flop per
                candidate pair (3 sub + 1 mul + 2 fma of d^2)
  e2e           the same metric through the public call with pinned HOST
                buffers, host-device transfers included
  parity        the timed cloud's result against the FP64 oracle on the same
                cloud (gates identical, scores within 1e-5, masks identical
                outside the tolerance band; counts of each)
  roofline_score the score phase's SFU (XU) work, ex2 + rcp per neighbour term,
                against the SFU peak, over the score phase's time (the leaf
                stage with and without the score stage, interleaved medians)
  cpu_baseline  the FP64 oracle on the full cloud: single-threaded and with
                the leaves spread over all host cores
  batched       64 LiDAR frames (60k-130k points) as one graph-captured batch,
                against the same frames one call each
  serving       the 2,000-frame Poisson 20 Hz stream (seed 7) through the
                continuous-batching server in real time (latency p50/p99),
                the highest arrival rate whose p99 latency stays within one
                20 Hz period, and frames all at once (throughput)
  variants      the cross-leaf kNN, the ablation toggles (Table 9), the score on
                a kNN within P_2, one leaf without the octree (Table 8), and the
                evaluation calls (PSNR / Chamfer, Eq. 29-30; the Sec. 2.2
                baseline), each timed with its candidate pairs and FP32 fraction
``--impl reference`` times the FP64 oracle instead (the reference arm).
"""

from __future__ import annotations

import argparse
import collections
import hashlib
import json
import multiprocessing as mp
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "points/s denoised; ms/frame p50/p99 batched vs plain GPU path at oracle mask"
UNIT = "points/s"
WORKLOAD = "dense_scan_560k_k32"
FLOP_PER_PAIR = 8.0
XU_OPS_PER_TERM = 2.0      # ex2 and rcp on the SFU per neighbour term of the score (gamma = 2)
XU_PER_SM_CLK = 16.0       # SFU (MUFU) operations per clock per SM
NPROC = os.cpu_count() or 1
SCORE_RTOL = 1e-5
PROFILE = os.path.join(ROOT, "profiles", "leaf_kernel_dense_scan.txt")


def _dist():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", str(rank)))
    return rank, world, local


def rank_seed(rank: int) -> int:
    """Weak scaling: each rank denoises its own cloud (seed 1 + rank)."""
    return 1 + rank


def max_over_ranks(value: float, device: str) -> float:
    """The slowest rank's time, on every rank (the job's time)."""
    import torch
    import torch.distributed as dist
    if not dist.is_initialized() or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(value: float, device: str) -> float:
    """The units all ranks processed (each rank may hold a different cloud)."""
    import torch
    import torch.distributed as dist
    if not dist.is_initialized() or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def job_throughput(units: float, total_ms: float, device: str) -> float:
    """Whole-job throughput: the units of all ranks over the slowest rank's time."""
    return sum_over_ranks(units, device) / (max_over_ranks(total_ms, device) / 1000.0)


def _peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            return json.load(f), "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


class ClockSampler:
    """nvidia-smi clock / throttle samples during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax = float(parts[2])
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


def _kernel_source_hash():
    h = hashlib.sha256()
    for f in ("gd_leaf.cu", "gd_leaf_kernel.cuh", "gd_common.cuh", "gd_knn_select.cuh", "gd_f32x2.cuh"):
        with open(os.path.join(ROOT, "paper_2512_10386_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def _profile_traffic():
    """DRAM bytes per launch of the leaf kernel from the committed ncu summary, if it
    was taken on the current kernel source (else None)."""
    if not os.path.exists(PROFILE):
        return None
    vals = {}
    with open(PROFILE) as f:
        for line in f:
            if ":" in line:
                k, v = line.split(":", 1)
                vals[k.strip()] = v.strip()
    if vals.get("kernel_source_sha256_16") != _kernel_source_hash():
        return None
    try:
        return float(vals["dram_bytes_per_launch_full_workload"])
    except (KeyError, ValueError):
        return None


def _workload(rank: int):
    import synth
    return synth.superquadric_scan(seed=rank_seed(rank))


def _oracle_params(P=None):
    import oracle
    from paper_2512_10386_gb300 import Params
    p = P or Params(k=32)
    return oracle.Params(k=p.k, leaf_capacity=p.leaf_capacity, max_depth=p.max_depth, beta=p.beta,
                         min_vox_count=p.min_vox_count, rho_percentile=p.rho_percentile, alpha=p.alpha,
                         sigma=p.sigma, gamma=p.gamma, eps_rho=p.eps_rho, eps_k=p.eps_k,
                         select_mode=p.select_mode, lam=p.lam, tau=p.tau, temperature=p.temperature,
                         stage_off=p.stage_off, rescore_p2=p.rescore_p2, cross_leaf=p.cross_leaf)


def cpu_baseline_full(xyz):
    """The FP64 oracle on the full cloud: one single-threaded run, and the best of
    three with the (independent) leaves spread over all host cores."""
    import oracle
    op = _oracle_params()
    t0 = time.perf_counter()
    oracle.denoise(xyz, op)
    single = time.perf_counter() - t0
    times = []
    for _ in range(3):
        t0 = time.perf_counter()
        oracle.denoise(xyz, op, threads=NPROC)
        times.append(time.perf_counter() - t0)
    best = min(times)
    return {"value": len(xyz) / best, "unit": UNIT, "cores": NPROC, "kind": "oracle",
            "sample": f"the full {len(xyz)}-point dense-scan cloud (K = 32): best of 3 runs with the leaves on "
                      f"{NPROC} host threads ({best:.2f} s); single-threaded {single:.2f} s",
            "single_thread_value": len(xyz) / single, "single_thread_s": single, "all_cores_s": best}


def _ambiguous(ref, select_mode, tau, tol=SCORE_RTOL):
    """Points whose selection may differ between FP32 and FP64 scores: ln F within
    tol of tau, or a score within tol of its leaf's Top-lambda cut."""
    F, st = ref["score"], ref["stage"]
    scored = (st == 0) | (st == 3)
    amb = np.zeros(len(F), bool)
    if select_mode == 1:
        with np.errstate(divide="ignore"):
            lf = np.log(np.where(F > 0, F, 1e-300))
        return scored & (np.abs(lf - np.float32(tau)) <= tol * max(1.0, abs(tau)) + 1e-6)
    leaf = ref["leaf_of"]
    for L in np.unique(leaf[scored & (st == 3)]):
        inl = (leaf == L) & scored
        kept, rem = inl & (st == 0), inl & (st == 3)
        if kept.any():
            c_keep, c_rem = F[kept].min(), F[rem].max()
            if c_keep <= c_rem * (1 + 2 * tol):
                amb |= inl & (F >= c_rem * (1 - 2 * tol)) & (F <= c_keep * (1 + 2 * tol))
    return amb


def certify(xyz, out, P):
    """The timed step's result against the FP64 oracle on the same cloud."""
    import oracle
    t0 = time.perf_counter()
    ref = oracle.denoise(xyz, _oracle_params(P), debug=True, threads=NPROC)
    secs = time.perf_counter() - t0
    mask, score, stage = (t.cpu().numpy() for t in (out.mask, out.score, out.stage))
    st_r = ref["stage"]
    gates = bool(np.array_equal(stage == 1, st_r == 1) and np.array_equal(stage == 2, st_r == 2))
    scored = (st_r == 0) | (st_r == 3)
    Fr, Fg = ref["score"][scored], score[scored].astype(np.float64)
    nz = Fr != 0
    rel = np.abs(Fg[nz] - Fr[nz]) / Fr[nz]
    zero_ok = bool(np.all(Fg[~nz] == 0))
    amb = _ambiguous(ref, P.select_mode, P.tau)
    mism = mask != ref["mask"]
    outside = int((mism & ~amb).sum())
    max_rel = float(rel.max()) if rel.size else 0.0
    return {"against": "FP64 oracle on the same cloud", "gates_identical": gates, "mask_mismatch": int(mism.sum()),
            "ambiguous_band": int(amb.sum()), "mismatch_outside_band": outside, "max_score_rel": max_rel,
            "score_tol": SCORE_RTOL, "oracle_s": secs,
            "ok": bool(gates and zero_ok and max_rel <= SCORE_RTOL and outside == 0)}


def run_reference(args):
    """Reference arm: the FP64 oracle as it stands, the full dense-scan cloud per
    step, with its (independent) leaves spread over all host cores."""
    import oracle
    rank, world, _ = _dist()
    if rank != 0:
        return 0
    xyz, _ = _workload(0)
    op = _oracle_params()
    times = []
    for s in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        oracle.denoise(xyz, op, threads=NPROC)
        if s >= args.warmup:
            times.append(time.perf_counter() - t0)
    value = len(xyz) * len(times) / sum(times)
    sample = f"the full {len(xyz)}-point dense-scan cloud per step, leaves on {NPROC} host threads"
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * sum(times) / len(times),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": WORKLOAD, "sample": sample},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": NPROC, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def run_ours(args):
    import torch
    rank, world, local = _dist()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    import __graft_entry__
    if rank == 0 or world == 1:
        __graft_entry__.build()
    if dist:
        dist.barrier()
        __graft_entry__.build()
    from paper_2512_10386_gb300 import Denoiser, Params

    xyz_np, labels_np = _workload(rank)
    n = len(xyz_np)
    P = Params(k=32, leaf_capacity=512)
    d = Denoiser(max_points=n, device=local)
    stream = torch.cuda.Stream()
    xyz = torch.from_numpy(xyz_np).cuda()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    out = d.run(xyz, P, stream=stream)
    torch.cuda.synchronize()

    clocks = ClockSampler(local).__enter__()   # sampled from warm-up to the end of the GPU sections
    # Timed steps are enqueued asynchronously (denoise_set_sync(0)) so that the
    # events bracket device work only, not the host's wake-up after a sync.
    d.set_sync(False)
    for _ in range(args.warmup):
        d.run(xyz, P, mask=out.mask, score=out.score, stage=out.stage, stream=stream)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    torch.cuda.synchronize()
    for s in range(args.steps):
        with torch.cuda.stream(stream):
            flush.fill_(float(s))
            ev[s][0].record(stream)
        d.run(xyz, P, mask=out.mask, score=out.score, stage=out.stage, stream=stream)
        ev[s][1].record(stream)
    torch.cuda.synchronize()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    from paper_2512_10386_gb300 import _native as N
    N.check(d.status(stream), "denoise_run")
    d.set_sync(True)
    # per-kernel times of the same step (library events between its stages), outside the timed region,
    # interleaved with the same cloud with the score stage switched off (A3: P_2 kept, no score, no
    # selection): the difference of the two medians is the time of the score and selection phases
    d.set_profiling(True)
    P_noscore = Params(k=32, leaf_capacity=512, stage_off=4)
    out_ns = d.run(xyz, P_noscore, stream=stream)
    leaf_ms, leaf_ms_noscore = [], []
    for s in range(max(1, min(args.steps, 10))):
        with torch.cuda.stream(stream):
            flush.fill_(float(s))
        d.run(xyz, P, mask=out.mask, score=out.score, stage=out.stage, stream=stream)
        leaf_ms.append(d.stats()["stage_ms"][4])
        stats = d.stats()
        with torch.cuda.stream(stream):
            flush.fill_(float(s) + 0.5)
        d.run(xyz, P_noscore, mask=out_ns.mask, score=out_ns.score, stage=out_ns.stage, stream=stream)
        leaf_ms_noscore.append(d.stats()["stage_ms"][4])
    d.set_profiling(False)
    del out_ns
    launches = stats["launches"] * args.steps
    total_ms = max_over_ranks(sum(step_ms), "cuda")
    value = job_throughput(n * args.steps, sum(step_ms), "cuda")
    if dist:
        dist.barrier()

    # ---- roofline of the fused leaf kernel (kNN + score)
    peaks, peak_kind = _peaks()
    props = torch.cuda.get_device_properties(local)
    sm_mhz = float(peaks.get("sm_max_mhz", 2070.0))
    fp32_peak_tflops = props.multi_processor_count * 128 * 2 * sm_mhz * 1e6 / 1e12
    leaf_avg_ms = sum(leaf_ms) / len(leaf_ms)
    achieved = stats["knn_pairs"] * FLOP_PER_PAIR / (leaf_avg_ms / 1000.0) / 1e12
    roofline = {"bound": "alu", "achieved": achieved, "peak": fp32_peak_tflops, "unit": "TFLOP/s",
                "frac": achieved / fp32_peak_tflops, "traffic": _profile_traffic(),
                "kernel": "gd::k_leaf<32> (voxel gate + kNN + density gate + score + selection; leaves of more "
                          "and of at most 64 points in two concurrent launches, timed together)",
                "work": f"{stats['knn_pairs']} candidate pairs x {FLOP_PER_PAIR:g} FP32 flop per launch",
                "peak_basis": f"{props.multi_processor_count} SMs x 128 FP32 lanes x 2 flop x {sm_mhz:g} MHz "
                              f"(max SM clock, {peak_kind} peaks file)",
                "leaf_kernel_ms": leaf_avg_ms, "share_of_step": leaf_avg_ms / (total_ms / args.steps)}
    # the score's SFU work (ex2 + rcp per neighbour term) over the score phase's time, taken as
    # the leaf kernel's time minus its time with the score stage off (that difference also holds
    # the Top-lambda selection, so the fraction is a lower bound of the score phase's own); the
    # fraction over the whole kernel's time is reported beside it
    xu_peak = props.multi_processor_count * XU_PER_SM_CLK * sm_mhz * 1e6 / 1e12
    xu_ops = stats["score_terms"] * XU_OPS_PER_TERM
    noscore_ms = float(np.median(leaf_ms_noscore))
    score_phase_ms = float(np.median(leaf_ms)) - noscore_ms
    # (a difference lost in the timing noise -- as under a profiler -- gives no figure)
    xu_achieved = xu_ops / (score_phase_ms / 1000.0) / 1e12 if score_phase_ms > 0.02 * leaf_avg_ms else None
    roofline_score = {"bound": "xu", "achieved": xu_achieved, "peak": xu_peak, "unit": "Tops/s",
                      "frac": xu_achieved / xu_peak if xu_achieved is not None else None,
                      "work": f"{stats['score_terms']} neighbour terms x {XU_OPS_PER_TERM:g} SFU ops (ex2, rcp)",
                      "time_basis": "score + selection phases: leaf kernel with the score stage minus without it",
                      "score_phase_ms": score_phase_ms, "leaf_kernel_ms_score_off": noscore_ms,
                      "frac_over_whole_kernel": xu_ops / (leaf_avg_ms / 1000.0) / 1e12 / xu_peak,
                      "peak_basis": f"{props.multi_processor_count} SMs x {XU_PER_SM_CLK:g} SFU ops/clk x {sm_mhz:g} MHz"}

    # ---- the timed cloud's result against the FP64 oracle (outside every timed region)
    parity = certify(xyz_np, out, P) if not args.no_parity else None

    # ---- end to end through the public call with pinned host buffers
    d.set_profiling(False)
    xyz_h = torch.from_numpy(xyz_np).pin_memory()
    mh = torch.empty(n, dtype=torch.uint8).pin_memory()
    sh = torch.empty(n, dtype=torch.float32).pin_memory()
    gh = torch.empty(n, dtype=torch.uint8).pin_memory()
    for _ in range(2):
        d.run(xyz_h, P, mask=mh, score=sh, stage=gh, stream=stream)
    e2e_ms = []
    for s in range(args.steps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(stream):
            flush.fill_(float(s))
        a.record(stream)
        d.run(xyz_h, P, mask=mh, score=sh, stage=gh, stream=stream)
        b.record(stream)
        torch.cuda.synchronize()
        e2e_ms.append(a.elapsed_time(b))
    e2e_total = max_over_ranks(sum(e2e_ms), "cuda")
    e2e = {"value": n * world * args.steps / (e2e_total / 1000.0), "unit": UNIT,
           "h2d_bytes_per_step": 12 * n, "d2h_bytes_per_step": 6 * n,
           "ms_per_step": e2e_total / args.steps}

    # ---- graph-captured replay of the same frame, and the batched workload
    d.set_graphs(True)
    d.run(xyz, P, mask=out.mask, score=out.score, stage=out.stage, stream=stream)
    d.set_sync(False)
    gev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    for s in range(args.steps):
        with torch.cuda.stream(stream):
            flush.fill_(float(s))
        gev[s][0].record(stream)
        d.run(xyz, P, mask=out.mask, score=out.score, stage=out.stage, stream=stream)
        gev[s][1].record(stream)
    torch.cuda.synchronize()
    N.check(d.status(stream), "denoise_run")
    d.set_sync(True)
    g_ms = [a.elapsed_time(b) for a, b in gev]
    d.set_graphs(False)
    graph = {"value": n * args.steps / (sum(g_ms) / 1000.0), "unit": UNIT,
             "ms_per_step": sum(g_ms) / args.steps}
    # keep the GPU busy on the same step for ~1 s so the clock sampler sees load
    t_end = time.perf_counter() + 1.0
    while time.perf_counter() < t_end:
        d.run(xyz, P, mask=out.mask, score=out.score, stage=out.stage, stream=stream)
    torch.cuda.synchronize()
    clocks.__exit__(None, None, None)
    out_mask_np = out.mask.cpu().numpy()
    d.close()

    batched = None
    if not args.no_batch:
        batched = run_batched(args, stream, flush)
    serving = None
    if args.serving_frames > 0 and rank == 0:
        serving = run_serving(args)
    variants = None
    if not args.no_variants and rank == 0:
        try:
            variants = run_variants(xyz_np, labels_np, out_mask_np, fp32_peak_tflops, stream)
        except Exception as e:  # a failed variant call must not cost the headline line
            variants = {"error": f"{type(e).__name__}: {e}"[:300]}

    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return 0
    cpu = cpu_baseline_full(xyz_np) if (world == 1 and not args.no_cpu) else None
    srt = sorted(step_ms)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "points_per_frame": n, "k": P.k, "leaf_capacity": P.leaf_capacity,
                   "path": "plain per-frame denoise_run, device buffers, direct launches",
                   "l2": "flushed between timed steps (256 MiB write)", "parallelism": f"replicas x{world}"},
        "ms_per_frame": {"p50": srt[len(srt) // 2], "p99": srt[min(len(srt) - 1, int(0.99 * len(srt)))]},
        "roofline": roofline, "roofline_score": roofline_score, "parity": parity, "e2e": e2e, "cpu_baseline": cpu,
        "graph_replay": graph, "batched": batched,
        "serving": serving, "variants": variants,
        "clocks": clocks.summary(), "gpu_launches": launches,
        "stats": {k: stats[k] for k in ("n_leaves", "knn_pairs", "n_p1", "n_p2", "score_terms", "launches")},
    }
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()
    return 0


def run_variants(xyz_np, labels_np, mask_np, fp32_peak_tflops, stream):
    """The method's variants and the evaluation calls, each timed on its own
    (CUDA events on the call's stream, median of a few calls after one untimed
    call) with its candidate pairs and its FP32 fraction (8 flop a pair, as the
    leaf kernel's roofline):
      cross_leaf   kNN over the 27 same-level cells around each leaf, on the timed cloud
      A1/A2/A3     one gate or the score selection switched off (Table 9), on the timed cloud
      rescore_p2   the score on a kNN recomputed within P_2, on the timed cloud
      octree_off   one leaf for the whole cloud (Table 8), on the 36,750-point object cloud
                   (K = 16): the leaf is one CTA's work, so one SM of the GPU runs it
      metrics      PSNR / Chamfer distance (Eq. 29-30) between the timed cloud's clean points
                   and its denoised result (brute-force nearest neighbours both ways)
      baseline     the gravitational-function method of Sec. 2.2 on the timed cloud
                   (neighbour counts within R by brute force)"""
    import torch

    import synth
    from paper_2512_10386_gb300 import Denoiser, Params

    def timed(fn, reps):
        fn()
        torch.cuda.synchronize()
        ms = []
        for _ in range(reps):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            fn()
            b.record(stream)
            torch.cuda.synchronize()
            ms.append(a.elapsed_time(b))
        return float(np.median(ms))

    def entry(points, ms, pairs):
        return {"points": int(points), "ms": ms, "points_per_s": points / (ms / 1000.0), "pairs": int(pairs),
                "fp32_frac": pairs * FLOP_PER_PAIR / (ms / 1000.0) / 1e12 / fp32_peak_tflops}

    n = len(xyz_np)
    xyz = torch.from_numpy(xyz_np).cuda()
    out = {"workload": WORKLOAD + " (octree off: the 36,750-point object cloud, K = 16)",
           "timing": "CUDA events around each call (device buffers, one host synchronisation a call), median"}
    d = Denoiser(max_points=n)
    try:
        base = Params(k=32, leaf_capacity=512)
        for name, P in (("A1_voxel_gate_off", Params(k=32, leaf_capacity=512, stage_off=1)),
                        ("A2_density_gate_off", Params(k=32, leaf_capacity=512, stage_off=2)),
                        ("A3_score_selection_off", Params(k=32, leaf_capacity=512, stage_off=4)),
                        ("rescore_p2", Params(k=32, leaf_capacity=512, rescore_p2=1))):
            r = d.run(xyz, P, stream=stream)
            ms = timed(lambda: d.run(xyz, P, mask=r.mask, score=r.score, stage=r.stage, stream=stream), 7)
            out[name] = entry(n, ms, d.stats()["knn_pairs"])
        ref = d.run(xyz, base, stream=stream).mask.clone()
        d.set_cross_leaf(True)
        Px = Params(k=32, leaf_capacity=512, cross_leaf=1)
        r = d.run(xyz, Px, stream=stream)
        ms = timed(lambda: d.run(xyz, Px, mask=r.mask, score=r.score, stage=r.stage, stream=stream), 5)
        out["cross_leaf"] = entry(n, ms, d.stats()["knn_pairs"])
        out["cross_leaf"]["mask_differs_from_leaf_local"] = float((r.mask != ref).float().mean().item())
        d.set_cross_leaf(False)
        clean = torch.from_numpy(np.ascontiguousarray(xyz_np[labels_np == 0])).cuda()
        den = torch.from_numpy(np.ascontiguousarray(xyz_np[mask_np == 1])).cuda()
        m = {}

        def metrics():
            m.update(d.eval_metrics(clean, den, stream=stream))
        ms = timed(metrics, 3)
        out["metrics"] = entry(len(clean) + len(den), ms, 2 * len(clean) * len(den))
        out["metrics"].update(clean_points=len(clean), denoised_points=len(den), psnr=m["psnr"],
                              chamfer=m["chamfer"], mse=m["mse"])
        kept = {}

        def baseline():
            kept["n"] = d.run_baseline(xyz, stream=stream)["keep"]
        ms = timed(baseline, 3)
        out["baseline"] = entry(n, ms, n * n)
        out["baseline"]["kept"] = int(kept["n"].sum().item())
    finally:
        d.close()
    obj, _ = synth.object_cloud(seed=0)
    xo = torch.from_numpy(obj).cuda()
    d = Denoiser(max_points=len(obj))
    try:
        Po = Params(k=16, leaf_capacity=0xFFFFFFFF)
        r = d.run(xo, Po, stream=stream)
        ms = timed(lambda: d.run(xo, Po, mask=r.mask, score=r.score, stage=r.stage, stream=stream), 2)
        out["octree_off"] = entry(len(obj), ms, d.stats()["knn_pairs"])
    finally:
        d.close()
    return out


def run_batched(args, stream, flush):
    """64 LiDAR frames of 60k-130k points (K = 24): the autotuner picks the leaf
    capacity and the leaf kernel's CTAs per SM for the graph-captured batch; the
    batch is then timed against the same frames one call each, at the tuned
    capacity (identical masks required)."""
    import dataclasses

    import torch

    import synth
    from paper_2512_10386_gb300 import Denoiser, Params
    from paper_2512_10386_gb300.autotune import tune_batch
    frames = synth.lidar_batch(n_frames=args.frames)
    sizes = [len(f[0]) for f in frames]
    offs = np.cumsum([0] + sizes).tolist()
    xyz = torch.from_numpy(np.concatenate([f[0] for f in frames])).cuda()
    total = int(offs[-1])
    d = Denoiser(max_points=total, max_frames=len(frames))
    tuned = tune_batch(xyz, offs, Params(k=24), reps=3, denoiser=d)
    P = dataclasses.replace(Params(k=24), leaf_capacity=tuned["leaf_capacity"])
    d.set_tuning(tuned["leaf_ctas_per_sm"], tuned.get("leaf_smem_points", 0), tuned.get("leaf_threads", 0))
    mask = torch.empty(total, dtype=torch.uint8, device="cuda")
    score = torch.empty(total, dtype=torch.float32, device="cuda")
    stage = torch.empty(total, dtype=torch.uint8, device="cuda")
    # plain path: one call per frame, enqueued asynchronously like the batch
    from paper_2512_10386_gb300 import _native as N
    d.set_sync(False)
    per_frame = []
    for rep in range(args.warmup + max(1, args.steps // 4)):
        for f in range(len(frames)):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            s0, s1 = offs[f], offs[f + 1]
            a.record(stream)
            d.run(xyz[s0:s1], P, mask=mask[s0:s1], score=score[s0:s1], stage=stage[s0:s1], stream=stream)
            b.record(stream)
            if rep >= args.warmup:
                per_frame.append((a, b))
    torch.cuda.synchronize()
    N.check(d.status(stream), "denoise_run")
    plain_ms = [a.elapsed_time(b) for a, b in per_frame]
    plain_mask = mask.clone()
    # batched path: one graph per batch
    d.set_graphs(True)
    d.run_batch(xyz, offs, P, mask=mask, score=score, stage=stage, stream=stream)
    torch.cuda.synchronize()
    N.check(d.status(stream), "denoise_run_batch")
    identical = bool(torch.equal(mask, plain_mask))
    bev = []
    for s in range(args.warmup + args.steps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(stream):
            flush.fill_(float(s))
        a.record(stream)
        d.run_batch(xyz, offs, P, mask=mask, score=score, stage=stage, stream=stream)
        b.record(stream)
        if s >= args.warmup:
            bev.append((a, b))
    torch.cuda.synchronize()
    N.check(d.status(stream), "denoise_run_batch")
    batch_ms = [a.elapsed_time(b) for a, b in bev]
    d.set_sync(True)
    d.close()
    ps = sorted(plain_ms)
    per_frame_batched = [m / len(frames) for m in batch_ms]
    default = next((r for r in tuned["table"] if r["leaf_capacity"] == 512 and r["leaf_ctas_per_sm"] == 0
                    and r.get("leaf_smem_points", 0) == 0 and r.get("leaf_threads", 0) == 0), None)
    return {
        "workload": f"{len(frames)} LiDAR frames, {min(sizes)}-{max(sizes)} points, {total} total, K=24",
        "tuned": {"leaf_capacity": tuned["leaf_capacity"], "leaf_ctas_per_sm": tuned["leaf_ctas_per_sm"],
                  "leaf_smem_points": tuned.get("leaf_smem_points", 0),
                  "leaf_threads": tuned.get("leaf_threads", 0),
                  "batch_ms_at_default_capacity_512": default["ms"] if default else None},
        "batched_points_per_s": total * len(batch_ms) / (sum(batch_ms) / 1000.0),
        "plain_points_per_s": total * len(plain_ms) / len(frames) / (sum(plain_ms) / 1000.0),
        "batched_ms_per_batch": sum(batch_ms) / len(batch_ms),
        "batched_ms_per_frame": statistics.mean(per_frame_batched),
        "plain_ms_per_frame": {"p50": ps[len(ps) // 2], "p99": ps[min(len(ps) - 1, int(0.99 * len(ps)))]},
        "masks_identical": identical,
    }


_SERVE = None


def _serve_init(seed, n_frames, bases):
    global _SERVE
    import synth
    _SERVE = synth.serving_stream(seed=seed, n_frames=n_frames, bases=bases)


def _serve_frame(i):
    return i, _SERVE.frame(_SERVE.requests[i])[0]


def _lazy_requests(stream, pool, indices, window=64):
    """Requests of the stream in arrival order, their frames made by a process
    pool at most `window` ahead of the server (the stream is never all in memory)."""
    from paper_2512_10386_gb300.serving import Request
    indices = list(indices)
    pend = collections.deque()
    k = 0
    while k < len(indices) and len(pend) < window:
        pend.append(pool.apply_async(_serve_frame, (indices[k],)))
        k += 1
    while pend:
        i, xyz = pend.popleft().get()
        if k < len(indices):
            pend.append(pool.apply_async(_serve_frame, (indices[k],)))
            k += 1
        r = stream.requests[i]
        yield Request(i, r.t_arrival, xyz, r.kind)


def run_serving(args):
    """The serving workload: a Poisson 20 Hz stream of args.serving_frames frames
    (seed 7) mixing dense 128-beam frames (~1.0 M points, 10 % outliers) and
    32-beam frames (~100 k, 15 % snow), played in real time through the
    continuous-batching server, frames made ahead by a process pool; then the
    first 300 frames at higher arrival rates (the highest rate whose p99
    latency stays within one 20 Hz period is the sustained rate) and all at once."""
    import synth
    from paper_2512_10386_gb300 import Params
    from paper_2512_10386_gb300.serving import Request, Server, latency_report
    n = args.serving_frames
    stream = synth.serving_stream(seed=7, n_frames=n)
    bases = stream.bases()
    P = Params(k=24)
    dense = 1_200_000
    workers = max(2, min(16, NPROC))
    ctx = mp.get_context("spawn")
    with ctx.Pool(workers, initializer=_serve_init, initargs=(7, n, bases)) as pool:
        nhold = min(300, n)
        held = dict(pool.imap(_serve_frame, range(nhold), chunksize=4))
        reqs = [Request(i, stream.requests[i].t_arrival, held[i], stream.requests[i].kind) for i in range(nhold)]
        srv = Server(P, capacities=[dense, dense, 4 * 130_000, 4 * 130_000], max_frames=4)
        try:
            srv.serve(reqs[:4], realtime=False, keep_results=False)  # warm-up: first launches, module loading
            t0 = time.perf_counter()
            comps = srv.serve(_lazy_requests(stream, pool, range(n)), realtime=True, keep_results=False)
            live = latency_report(comps, time.perf_counter() - t0)
            sweep = []
            for scale in (10, 25, 50, 100, 200, 400):
                rs = [Request(r.rid, stream.requests[r.rid].t_arrival / scale, r.xyz, r.kind) for r in reqs]
                t0 = time.perf_counter()
                comps = srv.serve(rs, realtime=True, keep_results=False)
                rep = latency_report(comps, time.perf_counter() - t0)
                rep["rate_hz"] = 20.0 * scale
                sweep.append(rep)
            t0 = time.perf_counter()
            comps = srv.serve(reqs, realtime=False, keep_results=False)
            burst = latency_report(comps, time.perf_counter() - t0)
        finally:
            srv.close()
    ok = [r for r in sweep if r["latency_ms_p99"] <= 50.0]
    sustained = max(ok, key=lambda r: r["rate_hz"]) if ok else None
    return {"workload": f"{n} frames, Poisson 20 Hz, seed 7, dense ~1.0M / sparse ~100k mix, K=24",
            "realtime": live,
            "rate_sweep": [{k: r[k] for k in ("rate_hz", "latency_ms_p50", "latency_ms_p99", "points_per_s",
                                             "mean_batch_frames")} for r in sweep],
            "sustained_rate_hz_p99_within_50ms": sustained["rate_hz"] if sustained else None,
            "sustained_points_per_s": sustained["points_per_s"] if sustained else None,
            "all_at_once": burst, "all_at_once_frames": nhold}


def run_batch_profile(args):
    """The batched LiDAR workload alone (64 frames, K = 24, leaf capacity 128,
    64-thread leaf CTAs: the autotuner's usual pick), W + K graph-captured
    batches, for profiling the leaf kernel on it; prints one JSON line."""
    import dataclasses

    import torch

    import synth
    from paper_2512_10386_gb300 import Denoiser, Params
    from paper_2512_10386_gb300 import _native as N
    frames = synth.lidar_batch(n_frames=args.frames)
    offs = np.cumsum([0] + [len(f[0]) for f in frames]).tolist()
    xyz = torch.from_numpy(np.concatenate([f[0] for f in frames])).cuda()
    d = Denoiser(max_points=int(offs[-1]), max_frames=len(frames))
    d.set_tuning(0, 0, 64)
    d.set_graphs(True)
    P = dataclasses.replace(Params(k=24), leaf_capacity=128)
    stream = torch.cuda.Stream()
    ms = []
    for s in range(args.warmup + args.steps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        d.run_batch(xyz, offs, P, stream=stream)
        b.record(stream)
        b.synchronize()
        if s >= args.warmup:
            ms.append(a.elapsed_time(b))
    N.check(d.status(stream), "denoise_run_batch")
    d.close()
    print(json.dumps({"workload": f"{len(frames)} LiDAR frames, {offs[-1]} points, K=24, capacity 128",
                      "batch_ms": ms}), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--frames", type=int, default=64)
    ap.add_argument("--no-batch", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--serving-frames", type=int, default=2000)
    ap.add_argument("--no-parity", action="store_true")
    ap.add_argument("--no-variants", action="store_true", help="skip the variants and evaluation-call timings")
    ap.add_argument("--batch-profile", action="store_true",
                    help="run only the batched LiDAR workload at fixed knobs (for profiling)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    if args.batch_profile:
        return run_batch_profile(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
