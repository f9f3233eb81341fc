"""ctypes front end of the plain FP64 CPU oracle (``ctqr_oracle.c``).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this module.  It shares no code
with the CUDA library and never imports it.

Every function takes and returns numpy arrays; matrices are column-major
(Fortran order) FP64, matching the layout of the method's system ``A X = B``
(paper Eq. (sistema)).  ``build()`` compiles the C source with
``-ffp-contract=off`` so no multiply-add is fused and the arithmetic is the
plain sequence written in the C file.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ctqr_oracle.c")
_LIB = os.path.join(_HERE, "_build", "libctqr_oracle.so")
_lock = threading.Lock()
_lib = None

# Status code the back-substitution returns for a numerically rank-deficient R.
ORACLE_RANK = 4


class Geometry(ctypes.Structure):
    """Scanner geometry (same meaning as the C struct ``og_geometry``).

    beam 0: parallel beam, det_span = detector width (image units).
    beam 1: equiangular fan beam, det_span = total fan angle (radians),
            src_iso = source-to-isocentre distance.
    Views: angle0 + v * angle_span / n_views, with angle_rule 1 shifted per
    quarter of the views as Eq. (angulos) reads (0, +0.5, -0.25, -0.5
    degrees).  Rays: ray = view*n_bins + bin.
    """

    _fields_ = [
        ("beam", ctypes.c_int), ("nx", ctypes.c_int), ("ny", ctypes.c_int),
        ("pixel", ctypes.c_double), ("n_views", ctypes.c_int), ("n_bins", ctypes.c_int),
        ("angle0", ctypes.c_double), ("angle_span", ctypes.c_double),
        ("src_iso", ctypes.c_double), ("det_span", ctypes.c_double),
        ("angle_rule", ctypes.c_int),
    ]

    @property
    def m(self) -> int:
        return self.n_views * self.n_bins

    @property
    def n(self) -> int:
        return self.nx * self.ny


def build(force: bool = False) -> str:
    """Compile the oracle into ``oracle/_build/libctqr_oracle.so``."""
    with _lock:
        if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
            return _LIB
        os.makedirs(os.path.dirname(_LIB), exist_ok=True)
        tmp = _LIB + f".{os.getpid()}.tmp"
        cmd = ["gcc", "-O2", "-fopenmp", "-ffp-contract=off", "-fPIC", "-shared",
               "-std=c11", _SRC, "-o", tmp, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
        return _LIB


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        D = ctypes.POINTER(ctypes.c_double)
        I64 = ctypes.c_int64
        lib.oracle_ray.argtypes = [ctypes.POINTER(Geometry), I64, D, D, D, D]
        lib.oracle_view_angle.argtypes = [ctypes.POINTER(Geometry), ctypes.c_int]
        lib.oracle_joseph.argtypes = [ctypes.POINTER(Geometry), D, I64, I64, D, I64]
        lib.oracle_quality.argtypes = [D, D, ctypes.c_int, ctypes.c_int, D]
        lib.oracle_view_angle.restype = ctypes.c_double
        lib.oracle_system_matrix.argtypes = [ctypes.POINTER(Geometry), D, I64]
        lib.oracle_qr.argtypes = [D, I64, I64, I64, D]
        lib.oracle_apply_qt.argtypes = [D, I64, I64, I64, D, D, I64, I64]
        lib.oracle_apply_q.argtypes = [D, I64, I64, I64, D, D, I64, I64]
        lib.oracle_backsolve.argtypes = [D, I64, I64, I64, D, I64, I64]
        lib.oracle_backsolve.restype = ctypes.c_int
        ci = ctypes.c_int
        lib.oracle_conv3x3_fwd.argtypes = [D, D, D, D, ci, ci, ci, ci, ci]
        lib.oracle_conv3x3_bwd.argtypes = [D, D, D, D, D, D, ci, ci, ci, ci, ci]
        _lib = lib
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _f64f(a) -> np.ndarray:
    return np.array(a, dtype=np.float64, order="F", copy=True)


def set_threads(n: int) -> None:
    """Number of OpenMP threads the oracle uses (applies to later calls)."""
    os.environ["OMP_NUM_THREADS"] = str(int(n))


def ray(g: Geometry, i: int):
    """(px, py, dx, dy): a point on ray i and its unit direction."""
    out = [ctypes.c_double() for _ in range(4)]
    _load().oracle_ray(ctypes.byref(g), i, *[ctypes.byref(o) for o in out])
    return tuple(o.value for o in out)


def view_angle(g: Geometry, v: int) -> float:
    """Angle (radians) of view v (0-based)."""
    return _load().oracle_view_angle(ctypes.byref(g), v)


def system_matrix(g: Geometry) -> np.ndarray:
    """Dense m x n FP64 A, a_ij = length of ray i inside pixel j."""
    A = np.zeros((g.m, g.n), dtype=np.float64, order="F")
    _load().oracle_system_matrix(ctypes.byref(g), _p(A), g.m)
    return A


def qr(A) -> tuple[np.ndarray, np.ndarray]:
    """Householder QR.  Returns (F, tau): R on/above the diagonal of F, the
    reflectors' v[1:] below it (v_0 = 1 implicit), H_j = I - tau_j v v^T."""
    F = _f64f(A)
    m, n = F.shape
    tau = np.zeros(min(m, n), dtype=np.float64)
    _load().oracle_qr(_p(F), m, n, m, _p(tau))
    return F, tau


def apply_qt(F, tau, B) -> np.ndarray:
    """Q^T B from the reflectors of ``qr``."""
    F = np.asfortranarray(F, dtype=np.float64)
    Bo = _f64f(B if np.ndim(B) == 2 else np.reshape(B, (-1, 1)))
    m, n = F.shape
    _load().oracle_apply_qt(_p(F), m, n, m, _p(np.ascontiguousarray(tau)), _p(Bo), Bo.shape[0], Bo.shape[1])
    return Bo if np.ndim(B) == 2 else Bo[:, 0]


def apply_q(F, tau, B) -> np.ndarray:
    """Q B from the reflectors of ``qr``."""
    F = np.asfortranarray(F, dtype=np.float64)
    Bo = _f64f(B if np.ndim(B) == 2 else np.reshape(B, (-1, 1)))
    m, n = F.shape
    _load().oracle_apply_q(_p(F), m, n, m, _p(np.ascontiguousarray(tau)), _p(Bo), Bo.shape[0], Bo.shape[1])
    return Bo if np.ndim(B) == 2 else Bo[:, 0]


def backsolve(F, Y) -> np.ndarray:
    """Solve R X = Y[0:n] by backward substitution (R = upper part of F).
    Raises ``np.linalg.LinAlgError`` when R is numerically rank deficient."""
    F = np.asfortranarray(F, dtype=np.float64)
    m, n = F.shape
    Yo = _f64f(Y if np.ndim(Y) == 2 else np.reshape(Y, (-1, 1)))
    rc = _load().oracle_backsolve(_p(F), m, n, m, _p(Yo), Yo.shape[0], Yo.shape[1])
    if rc == ORACLE_RANK:
        raise np.linalg.LinAlgError("R is numerically rank deficient")
    X = Yo[:n]
    return X if np.ndim(Y) == 2 else X[:, 0]


def joseph_project(g: Geometry, X) -> np.ndarray:
    """Sinograms of the images X (n x k, or a length-n vector) by Joseph's
    projector: B (m x k)."""
    Xo = _f64f(X if np.ndim(X) == 2 else np.reshape(X, (-1, 1)))
    k = Xo.shape[1]
    B = np.zeros((g.m, k), dtype=np.float64, order="F")
    _load().oracle_joseph(ctypes.byref(g), _p(Xo), Xo.shape[0], k, _p(B), g.m)
    return B if np.ndim(X) == 2 else B[:, 0]


def quality(x, ref, nx: int, ny: int) -> tuple[float, float, float]:
    """(MSE, PSNR in dB, SSIM) of image x against the reference image."""
    xo = np.ascontiguousarray(x, dtype=np.float64).reshape(-1)
    ro = np.ascontiguousarray(ref, dtype=np.float64).reshape(-1)
    out = np.zeros(3)
    _load().oracle_quality(_p(xo), _p(ro), nx, ny, _p(out))
    return float(out[0]), float(out[1]), float(out[2])


def lstsq(A, B) -> np.ndarray:
    """X = R^{-1} (Q^T B)[0:n] (paper Eq. (qr1))."""
    F, tau = qr(A)
    return backsolve(F, apply_qt(F, tau, B))


def conv3x3_fwd(x, wt, bias=None) -> np.ndarray:
    """NCHW 3x3 convolution (cross-correlation), stride 1, zero padding 1."""
    x = np.ascontiguousarray(x, dtype=np.float64)
    wt = np.ascontiguousarray(wt, dtype=np.float64)
    B, C, H, W = x.shape
    O = wt.shape[0]
    y = np.zeros((B, O, H, W), dtype=np.float64)
    b = None if bias is None else np.ascontiguousarray(bias, dtype=np.float64)
    _load().oracle_conv3x3_fwd(_p(x), _p(wt), _p(b) if b is not None else None, _p(y), B, C, O, H, W)
    return y


def conv3x3_bwd(x, wt, gy):
    """Gradients (gx, gw, gb) of sum(gy * conv3x3_fwd(x, wt, bias))."""
    x = np.ascontiguousarray(x, dtype=np.float64)
    wt = np.ascontiguousarray(wt, dtype=np.float64)
    gy = np.ascontiguousarray(gy, dtype=np.float64)
    B, C, H, W = x.shape
    O = wt.shape[0]
    gx = np.zeros_like(x)
    gw = np.zeros_like(wt)
    gb = np.zeros(O, dtype=np.float64)
    _load().oracle_conv3x3_bwd(_p(x), _p(wt), _p(gy), _p(gx), _p(gw), _p(gb), B, C, O, H, W)
    return gx, gw, gb
