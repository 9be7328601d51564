"""Denoising quality metrics of the paper's evaluation (Sec. 4.1, Eq. 26-28).

Host-side reporting only; not part of the denoising path.
"""

from __future__ import annotations

import numpy as np


def precision_recall_f1(keep, noise):
    """Eq. 26-28: P_d = N_q/N_s, R_d = N_q/N_y, F1 = 2 P R / (P + R).

    ``keep`` is the method's output mask (1 = kept), ``noise`` the ground-truth
    noise labels (1 = noise).  N_q = removed noise points, N_s = removed points,
    N_y = noise points.
    """
    keep = np.asarray(keep).astype(bool)
    noise = np.asarray(noise).astype(bool)
    removed = ~keep
    nq = float(np.count_nonzero(removed & noise))
    ns = float(np.count_nonzero(removed))
    ny = float(np.count_nonzero(noise))
    p = nq / ns if ns else 0.0
    r = nq / ny if ny else 0.0
    f1 = 2 * p * r / (p + r) if (p + r) else 0.0
    return p, r, f1
