"""GB300-native adaptive dual-weight gravitational point-cloud denoiser (arXiv 2512.10386).

Layout:
  csrc/        CUDA kernels (sm_103a) and the C ABI of include/gravdenoise.h
  build.py     in-tree nvcc build of libgravdenoise.so
  _native.py   ctypes binding, same names as the C ABI
  api.py       PyTorch front end (Denoiser, Params, SoftRemoval, soft_f1_loss)
  metrics.py   precision / recall / F1 of the paper's evaluation (Eq. 26-28)
"""

from .metrics import precision_recall_f1


def __getattr__(name):
    # the PyTorch front end is imported on first use so that importing the
    # package (e.g. for metrics) does not require a GPU or a built library
    if name in ("Denoiser", "Params", "Result", "SoftRemoval", "soft_f1_loss"):
        from . import api
        return getattr(api, name)
    raise AttributeError(name)


__all__ = ["Denoiser", "Params", "Result", "SoftRemoval", "soft_f1_loss", "precision_recall_f1"]
