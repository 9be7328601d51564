"""Calibration of the weighting parameters on labelled frames (differentiable form).

theta = (alpha, sigma, gamma, tau) is fitted by gradient descent on the mean
soft-F1 loss over labelled frames.  Each step runs the GPU forward with
training enabled and the library's hand-written backward (SoftRemoval);
neighbour sets, gates and densities do not depend on theta, so only the score
and the soft selection are differentiated.
"""

from __future__ import annotations

import dataclasses
from typing import Iterable, List, Optional, Tuple

import torch

from .api import Denoiser, Params, SoftRemoval, soft_f1_loss


@dataclasses.dataclass
class CalibrationResult:
    params: Params
    losses: List[float]


def calibrate(frames: Iterable[Tuple[torch.Tensor, torch.Tensor]], params: Params, steps: int = 20,
              lr: float = 0.05, denoiser: Optional[Denoiser] = None) -> CalibrationResult:
    """frames: (xyz float32 [n,3] on the GPU, noise labels [n] 0/1); returns the fitted params
    and the loss of every step (mean over frames, before the step's update)."""
    frames = list(frames)
    own = denoiser is None
    if own:
        denoiser = Denoiser(max_points=max(int(f[0].shape[0]) for f in frames))
    theta = torch.tensor([params.alpha, params.sigma, params.gamma, params.tau], dtype=torch.float64,
                         requires_grad=True)
    opt = torch.optim.Adam([theta], lr=lr)
    losses = []
    try:
        for _ in range(steps):
            opt.zero_grad()
            total = 0.0
            for xyz, noise in frames:
                r = SoftRemoval.apply(xyz, theta, denoiser, params)
                loss = soft_f1_loss(r, noise) / len(frames)
                loss.backward()
                total += float(loss.detach())
            losses.append(total)
            opt.step()
            with torch.no_grad():   # keep sigma and gamma in their valid ranges
                theta[1].clamp_(min=1e-3)
                theta[2].clamp_(min=1e-3)
    finally:
        if own:
            denoiser.close()
    a, s, g, t = (float(v) for v in theta.detach())
    return CalibrationResult(dataclasses.replace(params, alpha=a, sigma=s, gamma=g, tau=t, select_mode=1), losses)
