"""Seeded synthetic point clouds shaped like the paper's workloads.

This package holds data generators only: it contains none of the denoiser's
arithmetic, so both the FP64 oracle and the GPU path can consume the same
inputs without sharing any method code.

Every generator returns ``(xyz, labels)`` with ``xyz`` a C-contiguous
``float32`` array of shape ``[N, 3]`` and ``labels`` a ``uint8`` array of shape
``[N]``: 0 = surface (signal), 1 = uniform outlier, 2 = clustered noise
(Gaussian blob or snow).  Points are shuffled with the same seed so that the
input order carries no label information.

The paper evaluates on Stanford Bunny, CADC and in-house FMCW LiDAR frames
(Sec. 4.1, Tables 1, 6, 7); none of those datasets is available here, so these
seeded generators stand in for them.
"""

from .clouds import object_cloud, superquadric_scan, noise_labels_to_binary
from .lidar import lidar_frame, lidar_batch, serving_stream

__all__ = [
    "object_cloud",
    "superquadric_scan",
    "noise_labels_to_binary",
    "lidar_frame",
    "lidar_batch",
    "serving_stream",
]
