"""ctypes binding of libgravdenoise.so: the C ABI of include/gravdenoise.h under the same names.

Argument marshalling only.  Every step of the denoising path runs in the
library's CUDA kernels; there is no CPU fallback.  Importing this module does
not touch the GPU; ``lib()`` loads the shared library and raises if it is
missing (build it with ``paper_2512_10386_gb300.build.build()``).
"""

from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libgravdenoise.so")

DENOISE_OK = 0
DENOISE_E_INVAL = -1
DENOISE_E_NONFINITE = -2
DENOISE_E_CAPACITY = -3
DENOISE_E_NOMEM = -4
DENOISE_E_TIMEOUT = -5
DENOISE_E_CUDA = -6
DENOISE_E_STATE = -7

DENOISE_SELECT_TOPRATIO = 0
DENOISE_SELECT_THRESHOLD = 1

# every symbol include/gravdenoise.h declares
EXPORTED = [
    "denoise_create", "denoise_destroy", "denoise_strerror", "denoise_run", "denoise_run_batch",
    "denoise_set_sync", "denoise_set_graphs", "denoise_set_profiling", "denoise_get_status",
    "denoise_get_stats", "denoise_run_debug", "denoise_set_training", "denoise_soft_removal",
    "denoise_backward", "denoise_run_noalloc", "denoise_set_tuning", "denoise_noalloc_scratch_bytes",
    "denoise_set_wait_limit", "denoise_test_hold_lookback", "denoise_eval_metrics", "denoise_run_baseline",
    "denoise_set_cross_leaf",
]
DENOISE_NOALLOC_MAX_POINTS = 16384


class denoise_params(ctypes.Structure):
    _fields_ = [
        ("k", ctypes.c_uint32),
        ("leaf_capacity", ctypes.c_uint32),
        ("max_depth", ctypes.c_uint32),
        ("beta", ctypes.c_float),
        ("min_vox_count", ctypes.c_uint32),
        ("rho_percentile", ctypes.c_float),
        ("alpha", ctypes.c_float),
        ("sigma", ctypes.c_float),
        ("gamma", ctypes.c_float),
        ("eps_rho", ctypes.c_float),
        ("eps_k", ctypes.c_float),
        ("select_mode", ctypes.c_uint32),
        ("lambda_", ctypes.c_float),
        ("tau", ctypes.c_float),
        ("temperature", ctypes.c_float),
        ("stage_off", ctypes.c_uint32),
        ("rescore_p2", ctypes.c_uint32),
        ("cross_leaf", ctypes.c_uint32),
    ]


class denoise_stats(ctypes.Structure):
    _fields_ = [
        ("n_points", ctypes.c_uint64),
        ("n_leaves", ctypes.c_uint64),
        ("knn_pairs", ctypes.c_uint64),
        ("n_p1", ctypes.c_uint64),
        ("n_p2", ctypes.c_uint64),
        ("score_terms", ctypes.c_uint64),
        ("launches", ctypes.c_uint32),
        ("n_stages", ctypes.c_uint32),
        ("stage_ms", ctypes.c_float * 8),
    ]


class denoise_tuning(ctypes.Structure):
    _fields_ = [("leaf_ctas_per_sm", ctypes.c_uint32), ("leaf_smem_points", ctypes.c_uint32),
                ("leaf_threads", ctypes.c_uint32)]


class denoise_debug(ctypes.Structure):
    _fields_ = [(name, ctypes.c_void_p) for name in (
        "key", "leaf_start", "leaf_count", "leaf_h", "vox_count", "r2", "nbr", "nbr_d2", "leaf_rho_med")]


_V = ctypes.c_void_p
_P = ctypes.POINTER(denoise_params)
_lib = None


class DenoiseError(RuntimeError):
    def __init__(self, status: int, where: str = ""):
        self.status = status
        super().__init__(f"{where}: {strerror(status)} ({status})" if where else f"{strerror(status)} ({status})")


def lib():
    """Load the native library (once).  Raises if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"native library missing: {LIB_PATH}; build it with paper_2512_10386_gb300.build.build()")
    L = ctypes.CDLL(LIB_PATH)
    L.denoise_create.argtypes = [ctypes.POINTER(_V), ctypes.c_int, ctypes.c_size_t, ctypes.c_uint32]
    L.denoise_destroy.argtypes = [_V]
    L.denoise_strerror.argtypes = [ctypes.c_int]
    L.denoise_strerror.restype = ctypes.c_char_p
    L.denoise_run.argtypes = [_V, _V, ctypes.c_size_t, _P, _V, _V, _V, _V]
    L.denoise_run_batch.argtypes = [_V, _V, ctypes.POINTER(ctypes.c_uint64), ctypes.c_uint32, _P, _V, _V, _V, _V]
    L.denoise_run_debug.argtypes = [_V, _V, ctypes.c_size_t, _P, _V, _V, _V, ctypes.POINTER(denoise_debug), _V]
    for name in ("denoise_set_sync", "denoise_set_graphs", "denoise_set_profiling", "denoise_set_training",
                 "denoise_set_cross_leaf"):
        getattr(L, name).argtypes = [_V, ctypes.c_int]
    L.denoise_get_status.argtypes = [_V, _V]
    L.denoise_get_stats.argtypes = [_V, ctypes.POINTER(denoise_stats)]
    L.denoise_soft_removal.argtypes = [_V, _V, _V]
    L.denoise_backward.argtypes = [_V, _V, ctypes.POINTER(ctypes.c_double), _V]
    L.denoise_run_noalloc.argtypes = [_V, ctypes.c_size_t, _P, _V, _V, _V, _V]
    L.denoise_set_tuning.argtypes = [_V, ctypes.POINTER(denoise_tuning)]
    L.denoise_set_wait_limit.argtypes = [_V, ctypes.c_uint32]
    L.denoise_test_hold_lookback.argtypes = [_V, ctypes.c_int32]
    L.denoise_eval_metrics.argtypes = [_V, _V, ctypes.c_size_t, _V, ctypes.c_size_t, ctypes.POINTER(ctypes.c_double),
                                       _V, _V, _V]
    L.denoise_run_baseline.argtypes = [_V, _V, ctypes.c_size_t, ctypes.c_double, ctypes.c_double, _V, _V,
                                       ctypes.POINTER(ctypes.c_double), _V]
    for name in EXPORTED:
        if name != "denoise_strerror":
            getattr(L, name).restype = ctypes.c_int
    L.denoise_noalloc_scratch_bytes.argtypes = []
    L.denoise_noalloc_scratch_bytes.restype = ctypes.c_size_t
    _lib = L
    return L


def strerror(status: int) -> str:
    try:
        return lib().denoise_strerror(int(status)).decode()
    except ImportError:
        return f"status {status}"


def check(status: int, where: str = ""):
    if status != DENOISE_OK:
        raise DenoiseError(status, where)
    return status


# --- same names as the C ABI -------------------------------------------------
def denoise_create(device: int, max_points: int, max_frames: int = 1) -> int:
    h = _V()
    check(lib().denoise_create(ctypes.byref(h), device, max_points, max_frames), "denoise_create")
    return h.value


def denoise_destroy(ctx: int) -> int:
    return lib().denoise_destroy(ctx)


def denoise_strerror(status: int) -> str:
    return strerror(status)


def denoise_run(ctx, xyz_ptr, n, params: denoise_params, mask_ptr, score_ptr, stage_ptr, stream) -> int:
    return lib().denoise_run(ctx, xyz_ptr, n, ctypes.byref(params), mask_ptr, score_ptr, stage_ptr, stream)


def denoise_run_batch(ctx, xyz_ptr, offsets, nframes, params: denoise_params, mask_ptr, score_ptr, stage_ptr,
                      stream) -> int:
    arr = (ctypes.c_uint64 * (nframes + 1))(*[int(v) for v in offsets])
    return lib().denoise_run_batch(ctx, xyz_ptr, arr, nframes, ctypes.byref(params), mask_ptr, score_ptr,
                                   stage_ptr, stream)


def denoise_run_debug(ctx, xyz_ptr, n, params, mask_ptr, score_ptr, stage_ptr, dbg: denoise_debug, stream) -> int:
    return lib().denoise_run_debug(ctx, xyz_ptr, n, ctypes.byref(params), mask_ptr, score_ptr, stage_ptr,
                                   ctypes.byref(dbg), stream)


def denoise_set_sync(ctx, on: int) -> int:
    return lib().denoise_set_sync(ctx, int(on))


def denoise_set_graphs(ctx, on: int) -> int:
    return lib().denoise_set_graphs(ctx, int(on))


def denoise_set_profiling(ctx, on: int) -> int:
    return lib().denoise_set_profiling(ctx, int(on))


def denoise_set_cross_leaf(ctx, on: int) -> int:
    return lib().denoise_set_cross_leaf(ctx, int(on))


def denoise_set_training(ctx, on: int) -> int:
    return lib().denoise_set_training(ctx, int(on))


def denoise_set_tuning(ctx, leaf_ctas_per_sm: int = 0, leaf_smem_points: int = 0, leaf_threads: int = 0) -> int:
    return lib().denoise_set_tuning(ctx, ctypes.byref(denoise_tuning(leaf_ctas_per_sm, leaf_smem_points,
                                                                     leaf_threads)))


def denoise_set_wait_limit(ctx, iterations: int) -> int:
    return lib().denoise_set_wait_limit(ctx, int(iterations))


def denoise_test_hold_lookback(ctx, tile: int) -> int:
    return lib().denoise_test_hold_lookback(ctx, int(tile))


def denoise_eval_metrics(ctx, clean_ptr, n_clean, den_ptr, n_den, nn_clean_ptr, nn_den_ptr, stream):
    m = (ctypes.c_double * 3)()
    st = lib().denoise_eval_metrics(ctx, clean_ptr, n_clean, den_ptr, n_den, m, nn_clean_ptr, nn_den_ptr, stream)
    return st, [m[0], m[1], m[2]]


def denoise_run_baseline(ctx, xyz_ptr, n, G, alpha, mask_ptr, n_i_ptr, stream):
    p = (ctypes.c_double * 5)()
    st = lib().denoise_run_baseline(ctx, xyz_ptr, n, float(G), float(alpha), mask_ptr, n_i_ptr, p, stream)
    return st, [p[i] for i in range(5)]


def denoise_get_status(ctx, stream) -> int:
    return lib().denoise_get_status(ctx, stream)


def denoise_get_stats(ctx) -> denoise_stats:
    s = denoise_stats()
    check(lib().denoise_get_stats(ctx, ctypes.byref(s)), "denoise_get_stats")
    return s


def denoise_soft_removal(ctx, removal_ptr, stream) -> int:
    return lib().denoise_soft_removal(ctx, removal_ptr, stream)


def denoise_noalloc_scratch_bytes() -> int:
    return int(lib().denoise_noalloc_scratch_bytes())


def denoise_run_noalloc(xyz_ptr, n, params: denoise_params, mask_ptr, score_ptr, stage_ptr, stream) -> int:
    return lib().denoise_run_noalloc(xyz_ptr, n, ctypes.byref(params), mask_ptr, score_ptr, stage_ptr, stream)


def denoise_backward(ctx, grad_ptr, stream):
    g = (ctypes.c_double * 4)()
    st = lib().denoise_backward(ctx, grad_ptr, g, stream)
    return st, [g[i] for i in range(4)]
