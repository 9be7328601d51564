"""ctypes front end of the FP64 CPU oracle (oracle.c).

TEST INFRASTRUCTURE ONLY: the plain, slow reference the GPU library is checked
against.  Only the test-suite, ``__graft_entry__.smoke()`` and the benchmark's
CPU-baseline leg may import this module; the library never does.

``build()`` compiles ``oracle.c`` with gcc into ``liboracle.so`` beside it
(``-ffp-contract=off``, no fast-math, so every FP32 step is the IEEE
operation the source spells out).
"""

from __future__ import annotations

import ctypes
import dataclasses
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_HDR = os.path.join(_HERE, "oracle.h")
_LIB = os.path.join(_HERE, "liboracle.so")

CFLAGS = ["-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared", "-fopenmp"]

OK, EINVAL, ENONFINITE, ENOMEM = 0, -1, -2, -3


def build(force: bool = False) -> str:
    """Compile liboracle.so if missing or older than its sources."""
    newest = max(os.path.getmtime(_SRC), os.path.getmtime(_HDR))
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < newest:
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", *CFLAGS, "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


class _Params(ctypes.Structure):
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


_P = ctypes.c_void_p


class _Out(ctypes.Structure):
    _fields_ = [(name, _P) for name in (
        "mask", "stage", "score", "key", "leaf_of", "vox_count", "r2", "rho", "nbr", "nbr_d2",
        "n_leaves", "leaf_start", "leaf_count", "leaf_level", "leaf_lo", "leaf_h",
        "leaf_rho_med", "leaf_n1", "leaf_n2", "root")]


@dataclasses.dataclass
class Params:
    """Method parameters; defaults follow the paper where it states them
    (K = 12, rho_percentile = 0.2, min_vox_count = 4; Sec. 4.3.1) and the
    documented readings elsewhere."""
    k: int = 12
    leaf_capacity: int = 512
    max_depth: int = 21
    beta: float = 1.0
    min_vox_count: int = 4
    rho_percentile: float = 0.2
    alpha: float = 1.0
    sigma: float = 1.0
    gamma: float = 2.0
    eps_rho: float = 1e-12
    eps_k: float = 1e-12
    select_mode: int = 0
    lam: float = 0.95
    tau: float = 0.0
    temperature: float = 0.05
    stage_off: int = 0      # ablations: bit 0 no voxel gate (A1), bit 1 no density gate (A2), bit 2 no score (A3)
    rescore_p2: int = 0     # 1: the score uses a kNN recomputed within P_2
    cross_leaf: int = 0     # 1: kNN candidates from the 27 same-level octree cells around the leaf

    def _c(self) -> _Params:
        return _Params(self.k, self.leaf_capacity, self.max_depth, self.beta, self.min_vox_count,
                       self.rho_percentile, self.alpha, self.sigma, self.gamma, self.eps_rho,
                       self.eps_k, self.select_mode, self.lam, self.tau, self.temperature,
                       self.stage_off, self.rescore_p2, self.cross_leaf)


_lib = None


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        lib.orc_denoise.argtypes = [_P, ctypes.c_int64, ctypes.POINTER(_Params), ctypes.POINTER(_Out)]
        lib.orc_denoise.restype = ctypes.c_int
        lib.orc_denoise_threads.argtypes = [_P, ctypes.c_int64, ctypes.POINTER(_Params), ctypes.POINTER(_Out),
                                            ctypes.c_int]
        lib.orc_denoise_threads.restype = ctypes.c_int
        lib.orc_softf1.argtypes = [_P, ctypes.c_int64, ctypes.POINTER(_Params), _P, _P, _P, _P, _P]
        lib.orc_softf1.restype = ctypes.c_int
        lib.orc_cbrt_spec.argtypes = [ctypes.c_double]
        lib.orc_cbrt_spec.restype = ctypes.c_double
        lib.orc_interleave.argtypes = [ctypes.c_uint32] * 3
        lib.orc_interleave.restype = ctypes.c_uint64
        lib.orc_nn_d2.argtypes = [_P, ctypes.c_int64, _P, ctypes.c_int64, _P]
        lib.orc_nn_d2.restype = ctypes.c_int
        lib.orc_metrics.argtypes = [_P, ctypes.c_int64, _P, ctypes.c_int64, _P, _P, _P]
        lib.orc_metrics.restype = ctypes.c_int
        lib.orc_baseline.argtypes = [_P, ctypes.c_int64, ctypes.c_double, ctypes.c_double, _P, _P, _P, _P, _P, _P]
        lib.orc_baseline.restype = ctypes.c_int
        _lib = lib
    return _lib


class OracleError(RuntimeError):
    def __init__(self, status):
        super().__init__(f"oracle status {status}")
        self.status = status


def _ptr(a):
    return None if a is None else a.ctypes.data


def denoise(xyz, params: Params | None = None, debug: bool = False, threads: int = 1) -> dict:
    """Run the whole method on one cloud.  Returns a dict of numpy arrays:
    mask, stage, score (input order); with ``debug`` also the per-stage
    intermediates (keys, leaves, voxel counts, neighbour lists, ...).
    ``threads`` > 1 spreads the leaves over host threads (same results)."""
    params = params or Params()
    xyz = np.ascontiguousarray(xyz, dtype=np.float32).reshape(-1, 3)
    n = xyz.shape[0]
    nn = max(n, 1)
    r = {"mask": np.zeros(nn, np.uint8), "stage": np.zeros(nn, np.uint8),
         "score": np.zeros(nn, np.float64)}
    if debug:
        k = params.k
        r.update(key=np.zeros(nn, np.uint64), leaf_of=np.zeros(nn, np.uint32),
                 vox_count=np.zeros(nn, np.uint32), r2=np.zeros(nn, np.float32),
                 rho=np.zeros(nn, np.float64), nbr=np.full((nn, k), 0xFFFFFFFF, np.uint32),
                 nbr_d2=np.zeros((nn, k), np.float32), n_leaves=np.zeros(1, np.int64),
                 leaf_start=np.zeros(nn, np.uint32), leaf_count=np.zeros(nn, np.uint32),
                 leaf_level=np.zeros(nn, np.uint32), leaf_lo=np.zeros((nn, 3), np.float32),
                 leaf_h=np.zeros(nn, np.float32), leaf_rho_med=np.zeros(nn, np.float64),
                 leaf_n1=np.zeros(nn, np.uint32), leaf_n2=np.zeros(nn, np.uint32),
                 root=np.zeros(4, np.float32))
    out = _Out(**{f: _ptr(r.get(f)) for f, _ in _Out._fields_})
    st = _load().orc_denoise_threads(_ptr(xyz), n, ctypes.byref(params._c()), ctypes.byref(out), int(threads))
    if st != OK:
        raise OracleError(st)
    res = {k_: v[:n] for k_, v in r.items() if k_ in ("mask", "stage", "score")}
    if debug:
        L = int(r["n_leaves"][0])
        for k_ in ("key", "leaf_of", "vox_count", "r2", "rho", "nbr", "nbr_d2"):
            res[k_] = r[k_][:n]
        for k_ in ("leaf_start", "leaf_count", "leaf_level", "leaf_lo", "leaf_h",
                   "leaf_rho_med", "leaf_n1", "leaf_n2"):
            res[k_] = r[k_][:L]
        res["n_leaves"] = L
        res["root"] = r["root"]
    return res


def softf1(xyz, params: Params, noise, in_loss=None):
    """Soft-F1 loss of the differentiable form and d loss / d(alpha, sigma, gamma, tau)."""
    xyz = np.ascontiguousarray(xyz, dtype=np.float32).reshape(-1, 3)
    n = xyz.shape[0]
    noise = np.ascontiguousarray(noise, dtype=np.uint8)
    inl = None if in_loss is None else np.ascontiguousarray(in_loss, dtype=np.uint8)
    loss = np.zeros(1, np.float64)
    grad = np.zeros(4, np.float64)
    rem = np.zeros(max(n, 1), np.float64)
    st = _load().orc_softf1(_ptr(xyz), n, ctypes.byref(params._c()), _ptr(noise), _ptr(inl),
                            _ptr(loss), _ptr(grad), _ptr(rem))
    if st != OK:
        raise OracleError(st)
    return float(loss[0]), grad, rem[:n]


def cbrt_spec(u: float) -> float:
    return _load().orc_cbrt_spec(float(u))


def interleave(qx: int, qy: int, qz: int) -> int:
    return int(_load().orc_interleave(qx, qy, qz))


def _xyz(a):
    return np.ascontiguousarray(a, dtype=np.float32).reshape(-1, 3)


def nn_d2(a, b) -> np.ndarray:
    """Squared distance from each point of ``a`` to its nearest point of ``b`` (FP64, brute force)."""
    a, b = _xyz(a), _xyz(b)
    out = np.zeros(max(len(a), 1), np.float64)
    st = _load().orc_nn_d2(_ptr(a), len(a), _ptr(b), len(b), _ptr(out))
    if st != OK:
        raise OracleError(st)
    return out[:len(a)]


def metrics(clean, denoised) -> dict:
    """MSE and PSNR of Eq. 29 (nearest-neighbour correspondence, M = the clean
    cloud's bounding-box diagonal) and the Chamfer distance of Eq. 30."""
    a, b = _xyz(clean), _xyz(denoised)
    v = np.zeros(3, np.float64)
    st = _load().orc_metrics(_ptr(a), len(a), _ptr(b), len(b), _ptr(v[0:]), v[1:].ctypes.data,
                             v[2:].ctypes.data)
    if st != OK:
        raise OracleError(st)
    return {"mse": float(v[0]), "chamfer": float(v[1]), "psnr": float(v[2])}


G_DEFAULT = 6.67e-11   # Eq. 6: the gravitational constant as the paper sets it
ALPHA_DEFAULT = 600.0  # Eq. 7: the paper's weighting parameter


def baseline(xyz, G: float = G_DEFAULT, alpha: float = ALPHA_DEFAULT) -> dict:
    """The gravitational-function baseline of Sec. 2.2 (Eq. 1-9)."""
    xyz = _xyz(xyz)
    n = len(xyz)
    nn = max(n, 1)
    r = {"keep": np.zeros(nn, np.uint8), "n_i": np.zeros(nn, np.uint32), "d_i": np.zeros(nn, np.float64),
         "F_i": np.zeros(nn, np.float64)}
    RT = np.zeros(2, np.float64)
    st = _load().orc_baseline(_ptr(xyz), n, G, alpha, _ptr(r["keep"]), _ptr(r["n_i"]), _ptr(r["d_i"]),
                              _ptr(r["F_i"]), RT[0:].ctypes.data, RT[1:].ctypes.data)
    if st != OK:
        raise OracleError(st)
    out = {k: v[:n] for k, v in r.items()}
    out["R"], out["T"] = float(RT[0]), float(RT[1])
    return out
