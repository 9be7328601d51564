"""PyTorch-facing front end of the native denoiser.

PyTorch supplies device memory and streams; all computation happens in the
library's CUDA kernels through the C ABI (``_native``).  There is no CPU
fallback: without a CUDA device or without the built library every call
raises.
"""

from __future__ import annotations

import dataclasses
from typing import Optional, Sequence

import torch

from . import _native as N


@dataclasses.dataclass
class Params:
    """Method parameters (names follow the paper's notation, Sec. 3).

    Stated by the paper: K = 12, rho_percentile = 0.2 (percent),
    min_vox_count = 4 (Sec. 4.3.1).  The others are unstated there; the
    defaults here are this implementation's readings (beta 3 keeps surface
    leaves above n_v on the synthetic workloads)."""
    k: int = 12
    leaf_capacity: int = 512
    max_depth: int = 21
    beta: float = 3.0
    min_vox_count: int = 4
    rho_percentile: float = 0.2
    alpha: float = 1.0
    sigma: float = 1.0
    gamma: float = 2.0
    eps_rho: float = 1e-12
    eps_k: float = 1e-12
    select_mode: int = N.DENOISE_SELECT_TOPRATIO
    lam: float = 0.95
    tau: float = 0.0
    temperature: float = 0.05
    stage_off: int = 0      # ablations (Table 9): bit 0 no voxel gate, bit 1 no density gate, bit 2 no score
    rescore_p2: int = 0     # 1: the score uses a kNN recomputed within P_2
    cross_leaf: int = 0     # 1: kNN over the 27 same-level octree cells around the leaf (set_cross_leaf first)

    def to_c(self) -> N.denoise_params:
        return N.denoise_params(self.k, self.leaf_capacity, self.max_depth, self.beta, self.min_vox_count,
                                self.rho_percentile, self.alpha, self.sigma, self.gamma, self.eps_rho,
                                self.eps_k, self.select_mode, self.lam, self.tau, self.temperature,
                                self.stage_off, self.rescore_p2, self.cross_leaf)


@dataclasses.dataclass
class Result:
    mask: torch.Tensor    # uint8 [n], 1 = keep
    score: torch.Tensor   # float32 [n], F_i on P_2, 0 elsewhere
    stage: torch.Tensor   # uint8 [n], 0 kept / 1 voxel gate / 2 density gate / 3 score


def _stream_handle(device: torch.device, stream) -> int:
    if stream is None:
        stream = torch.cuda.current_stream(device)
    return stream.cuda_stream if isinstance(stream, torch.cuda.Stream) else int(stream)


def _ptr(t: Optional[torch.Tensor]):
    return None if t is None else t.data_ptr()


class Denoiser:
    """One native context: device scratch sized for ``max_points`` points in up
    to ``max_frames`` frames, allocated once."""

    def __init__(self, max_points: int, max_frames: int = 1, device=None):
        if not torch.cuda.is_available():
            raise RuntimeError("a CUDA device is required: the denoiser has no CPU path")
        self.device = torch.device("cuda", torch.cuda.current_device() if device is None else
                                   torch.device(device).index or 0)
        self.max_points = int(max_points)
        self.max_frames = int(max_frames)
        with torch.cuda.device(self.device):
            self.ctx = N.denoise_create(self.device.index, self.max_points, self.max_frames)
        self._sync = True

    # -- options ------------------------------------------------------------
    def set_sync(self, on: bool):
        self._sync = bool(on)
        N.check(N.denoise_set_sync(self.ctx, on), "denoise_set_sync")

    def set_graphs(self, on: bool):
        N.check(N.denoise_set_graphs(self.ctx, on), "denoise_set_graphs")

    def set_profiling(self, on: bool):
        N.check(N.denoise_set_profiling(self.ctx, on), "denoise_set_profiling")

    def set_tuning(self, leaf_ctas_per_sm: int = 0, leaf_smem_points: int = 0, leaf_threads: int = 0):
        """Execution tuning (``denoise_set_tuning``); results do not depend on it."""
        N.check(N.denoise_set_tuning(self.ctx, int(leaf_ctas_per_sm), int(leaf_smem_points), int(leaf_threads)),
                "denoise_set_tuning")

    def set_wait_limit(self, iterations: int):
        """Polls before a bounded device wait gives up (``denoise_set_wait_limit``; 0 = built-in)."""
        N.check(N.denoise_set_wait_limit(self.ctx, int(iterations)), "denoise_set_wait_limit")

    def test_hold_lookback(self, tile: int):
        """Test hook (``denoise_test_hold_lookback``): radix tile ``tile`` never publishes; -1 = off."""
        N.check(N.denoise_test_hold_lookback(self.ctx, int(tile)), "denoise_test_hold_lookback")

    def set_cross_leaf(self, on: bool):
        """Allocate the cross-leaf kNN tables (``denoise_set_cross_leaf``)."""
        N.check(N.denoise_set_cross_leaf(self.ctx, on), "denoise_set_cross_leaf")

    def set_training(self, on: bool):
        N.check(N.denoise_set_training(self.ctx, on), "denoise_set_training")

    # -- forward ------------------------------------------------------------
    def _outputs(self, n: int, like: torch.Tensor, mask, score, stage):
        dev = like.device
        pin = dev.type == "cpu"
        if mask is None:
            mask = torch.empty(n, dtype=torch.uint8, device=dev, pin_memory=pin)
        if score is None:
            score = torch.empty(n, dtype=torch.float32, device=dev, pin_memory=pin)
        if stage is None:
            stage = torch.empty(n, dtype=torch.uint8, device=dev, pin_memory=pin)
        return mask, score, stage

    @staticmethod
    def _check_xyz(xyz: torch.Tensor):
        if xyz.dtype != torch.float32 or xyz.dim() != 2 or xyz.shape[1] != 3 or not xyz.is_contiguous():
            raise ValueError("xyz must be a contiguous float32 tensor of shape [n, 3]")

    def run(self, xyz: torch.Tensor, params: Optional[Params] = None, *, mask=None, score=None, stage=None,
            stream=None) -> Result:
        """Denoise one cloud (``denoise_run``).  ``xyz`` on the GPU or on the
        host (pinned for asynchronous copies); results live beside it."""
        self._check_xyz(xyz)
        params = params or Params()
        n = xyz.shape[0]
        mask, score, stage = self._outputs(n, xyz, mask, score, stage)
        st = N.denoise_run(self.ctx, _ptr(xyz), n, params.to_c(), _ptr(mask), _ptr(score), _ptr(stage),
                           _stream_handle(self.device, stream))
        N.check(st, "denoise_run")
        return Result(mask, score, stage)

    def run_batch(self, xyz: torch.Tensor, offsets: Sequence[int], params: Optional[Params] = None, *,
                  mask=None, score=None, stage=None, stream=None) -> Result:
        """Denoise concatenated frames (``denoise_run_batch``); frame f owns
        rows offsets[f] .. offsets[f+1]-1."""
        self._check_xyz(xyz)
        params = params or Params()
        offsets = [int(v) for v in offsets]
        if offsets[-1] != xyz.shape[0]:
            raise ValueError("offsets[-1] must equal the number of points")
        n = xyz.shape[0]
        mask, score, stage = self._outputs(n, xyz, mask, score, stage)
        st = N.denoise_run_batch(self.ctx, _ptr(xyz), offsets, len(offsets) - 1, params.to_c(), _ptr(mask),
                                 _ptr(score), _ptr(stage), _stream_handle(self.device, stream))
        N.check(st, "denoise_run_batch")
        return Result(mask, score, stage)

    def run_debug(self, xyz: torch.Tensor, params: Optional[Params] = None, stream=None) -> dict:
        """``denoise_run_debug``: results plus per-stage intermediates (device tensors)."""
        self._check_xyz(xyz)
        if xyz.device.type != "cuda":
            raise ValueError("run_debug needs device input")
        params = params or Params()
        n, k = xyz.shape[0], params.k
        dev = xyz.device
        out = {
            "key": torch.zeros(n, dtype=torch.int64, device=dev),
            "leaf_start": torch.zeros(n, dtype=torch.int32, device=dev),
            "leaf_count": torch.zeros(n, dtype=torch.int32, device=dev),
            "leaf_h": torch.zeros(n, dtype=torch.float32, device=dev),
            "vox_count": torch.zeros(n, dtype=torch.int32, device=dev),
            "r2": torch.zeros(n, dtype=torch.float32, device=dev),
            "nbr": torch.full((n, k), -1, dtype=torch.int32, device=dev),
            "nbr_d2": torch.zeros((n, k), dtype=torch.float32, device=dev),
            "leaf_rho_med": torch.zeros(n, dtype=torch.float64, device=dev),
        }
        dbg = N.denoise_debug(**{name: out[name].data_ptr() for name, _ in N.denoise_debug._fields_})
        mask, score, stage = self._outputs(n, xyz, None, None, None)
        st = N.denoise_run_debug(self.ctx, _ptr(xyz), n, params.to_c(), _ptr(mask), _ptr(score), _ptr(stage),
                                 dbg, _stream_handle(self.device, stream))
        N.check(st, "denoise_run_debug")
        out.update(mask=mask, score=score, stage=stage)
        return out

    def eval_metrics(self, clean: torch.Tensor, denoised: torch.Tensor, per_point: bool = False, stream=None):
        """Evaluation metrics of Sec. 4.1 (``denoise_eval_metrics``): a dict with
        ``mse`` and ``psnr`` (Eq. 29) and ``chamfer`` (Eq. 30); with ``per_point``
        also the nearest squared distances of each clean / denoised point."""
        self._check_xyz(clean)
        self._check_xyz(denoised)
        na, nb = clean.shape[0], denoised.shape[0]
        nn_a = nn_b = None
        if per_point:
            nn_a = torch.empty(na, dtype=torch.float32, device=clean.device)
            nn_b = torch.empty(nb, dtype=torch.float32, device=denoised.device)
        st, m = N.denoise_eval_metrics(self.ctx, _ptr(clean), na, _ptr(denoised), nb, _ptr(nn_a), _ptr(nn_b),
                                       _stream_handle(self.device, stream))
        N.check(st, "denoise_eval_metrics")
        out = {"mse": m[0], "chamfer": m[1], "psnr": m[2]}
        if per_point:
            out.update(nn_clean=nn_a, nn_denoised=nn_b)
        return out

    def run_baseline(self, xyz: torch.Tensor, G: float = 6.67e-11, alpha: float = 600.0, counts: bool = False,
                     stream=None) -> dict:
        """The gravitational-function baseline of Sec. 2.2 (``denoise_run_baseline``):
        keep mask (Eq. 8-9), optionally the neighbour counts n_i (Eq. 5), and the
        centroid, R and T (Eq. 1, 3, 7)."""
        self._check_xyz(xyz)
        n = xyz.shape[0]
        mask = torch.empty(n, dtype=torch.uint8, device=xyz.device)
        n_i = torch.empty(n, dtype=torch.int32, device=xyz.device) if counts else None
        st, p = N.denoise_run_baseline(self.ctx, _ptr(xyz), n, G, alpha, _ptr(mask), _ptr(n_i),
                                       _stream_handle(self.device, stream))
        N.check(st, "denoise_run_baseline")
        out = {"keep": mask, "theta": p[0:3], "R": p[3], "T": p[4]}
        if counts:
            out["n_i"] = n_i
        return out

    def status(self, stream=None) -> int:
        return N.denoise_get_status(self.ctx, _stream_handle(self.device, stream))

    def stats(self) -> dict:
        s = N.denoise_get_stats(self.ctx)
        return {"n_points": s.n_points, "n_leaves": s.n_leaves, "knn_pairs": s.knn_pairs, "n_p1": s.n_p1,
                "n_p2": s.n_p2, "score_terms": s.score_terms, "launches": s.launches,
                "stage_ms": [s.stage_ms[i] for i in range(s.n_stages)]}

    # -- differentiable form ---------------------------------------------------
    def soft_removal(self, n: int, stream=None) -> torch.Tensor:
        out = torch.empty(n, dtype=torch.float32, device=self.device)
        N.check(N.denoise_soft_removal(self.ctx, out.data_ptr(), _stream_handle(self.device, stream)),
                "denoise_soft_removal")
        return out

    def backward(self, grad_removal: torch.Tensor, stream=None):
        g = grad_removal.detach().to(device=self.device, dtype=torch.float32).contiguous()
        st, grad = N.denoise_backward(self.ctx, g.data_ptr(), _stream_handle(self.device, stream))
        N.check(st, "denoise_backward")
        return grad

    def close(self):
        if getattr(self, "ctx", None):
            N.denoise_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class SoftRemoval(torch.autograd.Function):
    """Soft removal probabilities r_i as a differentiable function of
    theta = (alpha, sigma, gamma, tau); neighbour sets and gates stay fixed.
    The backward is the library's hand-written kernel (``denoise_backward``)."""

    @staticmethod
    def forward(ctx, xyz, theta, denoiser: Denoiser, params: Params):
        a, s, g, t = (float(v) for v in theta.detach().cpu().tolist())
        p = dataclasses.replace(params, alpha=a, sigma=s, gamma=g, tau=t, select_mode=N.DENOISE_SELECT_THRESHOLD)
        denoiser.set_training(True)
        denoiser.run(xyz, p)
        r = denoiser.soft_removal(xyz.shape[0])
        ctx.denoiser = denoiser
        ctx.theta_meta = (theta.dtype, theta.device)
        return r

    @staticmethod
    def backward(ctx, grad_r):
        grad = ctx.denoiser.backward(grad_r)
        dtype, device = ctx.theta_meta
        return None, torch.tensor(grad, dtype=dtype, device=device), None, None


def soft_f1_loss(removal: torch.Tensor, noise: torch.Tensor, select: Optional[torch.Tensor] = None) -> torch.Tensor:
    """1 - soft F1 of noise removal (Eq. 26-28 with soft counts):
    F1 = 2 sum(r y) / (sum r + sum y)."""
    r = removal.double()
    y = noise.double()
    if select is not None:
        r = r[select]
        y = y[select]
    return 1.0 - 2.0 * (r * y).sum() / (r.sum() + y.sum())
