"""Thin ctypes binding of ``libctqr.so`` (the C ABI in ``include/ctqr.h``).

Argument marshalling only: every step of the computation runs in the CUDA
library.  Matrices are torch CUDA tensors in column-major layout (use
``colmajor()`` to make one); the current torch CUDA stream is passed to every
call.  There is no CPU fallback: if the library cannot be loaded, every call
raises.
"""
from __future__ import annotations

import ctypes
import enum
import os
from dataclasses import dataclass

import torch

from . import build as _build

CT_OK, CT_ERR_INVALID, CT_ERR_NOMEM, CT_ERR_CUDA, CT_ERR_RANK = 0, 1, 2, 3, 4
CT_ERR_NONFINITE, CT_ERR_NOCONVERGE, CT_ERR_TIMEOUT, CT_ERR_UNSUPPORTED = 5, 6, 7, 8
CT_F64, CT_F32 = 0, 1


class Prec(enum.IntEnum):
    F64 = 0
    F32 = 1
    TF32 = 2
    F16X3 = 3


class CtError(RuntimeError):
    def __init__(self, status: int, what: str):
        self.status = status
        super().__init__(f"{what}: {_status_name(status)}")


class Geometry(ctypes.Structure):
    _fields_ = [
        ("beam", ctypes.c_int), ("nx", ctypes.c_int), ("ny", ctypes.c_int),
        ("pixel", ctypes.c_double), ("n_views", ctypes.c_int), ("n_bins", ctypes.c_int),
        ("angle0", ctypes.c_double), ("angle_span", ctypes.c_double),
        ("src_iso", ctypes.c_double), ("det_span", ctypes.c_double), ("angle_rule", ctypes.c_int),
    ]


class QrOpts(ctypes.Structure):
    _fields_ = [("nb", ctypes.c_int), ("in_place", ctypes.c_int), ("tf32_passes", ctypes.c_int),
                ("outer_nb", ctypes.c_int)]


class OocOpts(ctypes.Structure):
    _fields_ = [("device_bytes", ctypes.c_size_t), ("nb", ctypes.c_int), ("no_overlap", ctypes.c_int)]


class RefineOpts(ctypes.Structure):
    _fields_ = [("max_iter", ctypes.c_int), ("lambda_", ctypes.c_double), ("tol", ctypes.c_double),
                ("method", ctypes.c_int)]


REFINE_AUTO, REFINE_CLASSICAL, REFINE_CGLS = 0, 1, 2


class Report(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int), ("last_update", ctypes.c_double),
                ("residual", ctypes.c_double), ("ms_total", ctypes.c_double),
                ("ms_build", ctypes.c_double), ("ms_factor", ctypes.c_double),
                ("ms_solve", ctypes.c_double)]


class KernelStats(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char_p), ("launches", ctypes.c_uint64), ("timed", ctypes.c_uint64),
                ("ms", ctypes.c_double), ("flops", ctypes.c_double), ("bytes", ctypes.c_double)]


CT_DEVICE_BUFFERS, CT_HOST_BUFFERS = 0, 1


class BatchSystem(ctypes.Structure):
    _fields_ = [("m", ctypes.c_int64), ("n", ctypes.c_int64), ("A", ctypes.c_void_p), ("lda", ctypes.c_int64),
                ("B", ctypes.c_void_p), ("ldb", ctypes.c_int64), ("k", ctypes.c_int64)]


class BatchOpts(ctypes.Structure):
    _fields_ = [("tile", ctypes.c_int), ("prec", ctypes.c_int), ("no_cache", ctypes.c_int)]


class BatchReport(ctypes.Structure):
    _fields_ = [("tile", ctypes.c_int), ("ms", ctypes.c_double), ("tasks", ctypes.c_int),
                ("iterations", ctypes.c_int)]


class SurrogateOpts(ctypes.Structure):
    _fields_ = [("in_scale", ctypes.c_double), ("out_scale", ctypes.c_double), ("seed", ctypes.c_uint64)]


class SurrogateReport(ctypes.Structure):
    _fields_ = [("slices", ctypes.c_int64), ("fallbacks", ctypes.c_int64), ("max_residual", ctypes.c_double),
                ("ms_total", ctypes.c_double), ("ms_network", ctypes.c_double), ("ms_gate", ctypes.c_double),
                ("ms_fallback", ctypes.c_double)]


_lib = None

# Every entry point of include/ctqr.h, with its ctypes signature.
_VP, _I64, _D, _I = ctypes.c_void_p, ctypes.c_int64, ctypes.c_double, ctypes.c_int
_P64 = ctypes.POINTER(ctypes.c_int64)
SIGNATURES = {
    "ct_status_str": ([_I], ctypes.c_char_p),
    "ct_version": ([], ctypes.c_char_p),
    "ct_system_size": ([ctypes.POINTER(Geometry), _D, _P64, _P64], _I),
    "ct_build_system": ([ctypes.POINTER(Geometry), _I, _D, _VP, _I64, _VP], _I),
    "ct_qr_factor": ([_VP, _I, _I64, _I64, _I64, _I, ctypes.POINTER(QrOpts),
                      ctypes.POINTER(_VP), _VP], _I),
    "ct_qr_factor_host": ([_VP, _I64, _I64, _I64, ctypes.POINTER(OocOpts), ctypes.POINTER(_VP), _VP], _I),
    "ct_project_joseph": ([ctypes.POINTER(Geometry), _VP, _I64, _I64, _VP, _I64, _VP], _I),
    "ct_image_quality": ([_VP, _I64, _VP, _I64, _I, _I, _I64, _VP, _VP], _I),
    "ct_factor_info": ([_VP, _P64, _P64, ctypes.POINTER(_I), ctypes.POINTER(_I)], _I),
    "ct_factor_data": ([_VP, ctypes.POINTER(_VP), ctypes.POINTER(_I), _P64, ctypes.POINTER(_VP)], _I),
    "ct_factor_status": ([_VP, _VP], _I),
    "ct_factor_copy": ([_VP, _VP, _I64, _VP, _VP], _I),
    "ct_apply_qt": ([_VP, _VP, _I64, _I64, _VP], _I),
    "ct_apply_qt_f32": ([_VP, _VP, _I64, _I64, _VP], _I),
    "ct_apply_qt_noalloc": ([_VP, _VP, _I64, _I64, _VP], _I),
    "ct_trsm_solve": ([_VP, _VP, _I64, _I64, _VP], _I),
    "ct_trsm_solve_f32": ([_VP, _VP, _I64, _I64, _I, _VP], _I),
    "ct_reconstruct_batch": ([_VP, _VP, _I, _I64, _VP, _I64, _VP, _I64, _I64,
                              ctypes.POINTER(RefineOpts), ctypes.POINTER(Report), _VP], _I),
    "ct_factor_destroy": ([_VP], None),
    "ct_factor_save": ([_VP, ctypes.c_char_p, ctypes.c_uint64, _VP], _I),
    "ct_factor_load": ([ctypes.c_char_p, ctypes.POINTER(_VP), ctypes.POINTER(ctypes.c_uint64), _VP], _I),
    "ct_factor_file_info": ([ctypes.c_char_p, _P64, _P64, ctypes.POINTER(_I), ctypes.POINTER(_I),
                             ctypes.POINTER(ctypes.c_uint64)], _I),
    "ct_geometry_hash": ([ctypes.POINTER(Geometry), _D], ctypes.c_uint64),
    "ct_reconstruct_scan": ([ctypes.POINTER(Geometry), _D, _I, _VP, _I64, _VP, _I64, _I64, _I,
                             ctypes.POINTER(RefineOpts), ctypes.POINTER(Report), _VP], _I),
    "ct_gemm_tf32_tn": ([_I64, _I64, _I64, _VP, _I64, _VP, _I64, _VP, _I64, _I, _I, _VP], _I),
    "ct_gemm_f16x3_tn": ([_I64, _I64, _I64, _VP, _I64, _VP, _I64, _VP, _I64, _I, _VP], _I),
    "ct_gemm_status": ([_VP], _I),
    "ct_qr_solve_batched": ([_I, ctypes.POINTER(BatchSystem), ctypes.POINTER(BatchOpts),
                             ctypes.POINTER(BatchReport), _VP], _I),
    "ct_qr_solve_batched_release": ([], None),
    "ct_batch_plan": ([_I, ctypes.POINTER(BatchSystem), _I, _VP, _I64, ctypes.POINTER(_I64),
                       ctypes.POINTER(_I)], _I),
    "ct_surrogate_init": ([ctypes.POINTER(Geometry), ctypes.POINTER(SurrogateOpts), ctypes.POINTER(_VP)], _I),
    "ct_surrogate_num_params": ([_VP], _I64),
    "ct_surrogate_params": ([_VP, _VP, _I], _I),
    "ct_surrogate_backproject": ([_VP, _VP, _I64, _I64, _VP, _VP], _I),
    "ct_surrogate_project": ([_VP, _VP, _I64, _VP, _I64, _VP], _I),
    "ct_surrogate_train_step": ([_VP, _VP, _VP, _I64, ctypes.c_float, ctypes.POINTER(_D), _VP], _I),
    "ct_surrogate_grad": ([_VP, _VP, _VP, _I64, ctypes.POINTER(_D), _VP, _VP], _I),
    "ct_surrogate_forward": ([_VP, _VP, _VP, _I64, _VP], _I),
    "ct_surrogate_infer": ([_VP, _VP, _I64, _VP, _I64, _I64, _D, _VP, ctypes.POINTER(RefineOpts), _VP,
                            ctypes.POINTER(SurrogateReport), _VP], _I),
    "ct_surrogate_destroy": ([_VP], None),
    "ct_profile_enable": ([_I], None),
    "ct_profile_reset": ([], None),
    "ct_profile_kernels": ([ctypes.POINTER(KernelStats), _I], _I),
    "ct_kernel_launches": ([], ctypes.c_uint64),
}


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load libctqr.so (building it first if needed) and bind every symbol."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.build() if build_if_missing else _build.LIB
    if not os.path.exists(path):
        raise RuntimeError(f"libctqr.so not found at {path}; run build() first")
    lib = ctypes.CDLL(path)
    for name, (args, res) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = res
    _lib = lib
    return lib


def _status_name(s: int) -> str:
    try:
        return load().ct_status_str(s).decode()
    except Exception:  # library not loadable: still give a readable message
        return f"status {s}"


def _check(st: int, what: str) -> None:
    if st != CT_OK:
        raise CtError(st, what)


def _stream() -> int:
    return torch.cuda.current_stream().cuda_stream


def _dt(t: torch.Tensor) -> int:
    if t.dtype == torch.float64:
        return CT_F64
    if t.dtype == torch.float32:
        return CT_F32
    raise TypeError(f"unsupported dtype {t.dtype}")


def _ld(t: torch.Tensor) -> int:
    """Leading dimension of a column-major 2-D CUDA tensor."""
    if not t.is_cuda:
        raise ValueError("expected a CUDA tensor")
    if t.dim() != 2:
        raise ValueError("expected a 2-D tensor")
    if t.stride(0) != 1 and t.shape[0] > 1:
        raise ValueError("expected a column-major tensor (stride(0) == 1); use colmajor()")
    return max(t.stride(1), t.shape[0], 1)


def colmajor(rows: int, cols: int, dtype=torch.float64, device="cuda", ld: int | None = None,
             fill=None) -> torch.Tensor:
    """A rows x cols column-major CUDA tensor (leading dimension ld >= rows)."""
    ld = rows if ld is None else ld
    storage = torch.empty((cols, ld), dtype=dtype, device=device)
    if fill is not None:
        storage.fill_(fill)  # padding rows included
    return storage.t()[:rows]


def to_colmajor(x, dtype=None, device="cuda") -> torch.Tensor:
    """Copy a 2-D array (numpy or torch) into a new column-major CUDA tensor."""
    x = torch.as_tensor(x)
    if x.dim() == 1:
        x = x[:, None]
    t = colmajor(x.shape[0], x.shape[1], dtype=dtype or x.dtype, device=device)
    t.copy_(x)
    return t


def geometry(g) -> Geometry:
    """Geometry from an ``inputs.ScanGeometry`` (or anything with the fields)."""
    return Geometry(g.beam, g.nx, g.ny, g.pixel, g.n_views, g.n_bins, g.angle0, g.angle_span,
                    g.src_iso, g.det_span, getattr(g, "angle_rule", 0))


def version() -> str:
    return load().ct_version().decode()


def system_size(geom, lam: float = 0.0) -> tuple[int, int]:
    m, n = ctypes.c_int64(), ctypes.c_int64()
    _check(load().ct_system_size(ctypes.byref(geometry(geom)), lam, ctypes.byref(m), ctypes.byref(n)),
           "ct_system_size")
    return m.value, n.value


def build_system(geom, dtype=torch.float64, lam: float = 0.0, out: torch.Tensor | None = None) -> torch.Tensor:
    """Dense system matrix A (m x n, column-major) built on the GPU."""
    m, n = system_size(geom, lam)
    A = colmajor(m, n, dtype=dtype) if out is None else out
    _check(load().ct_build_system(ctypes.byref(geometry(geom)), _dt(A), lam, A.data_ptr(), _ld(A),
                                  _stream()), "ct_build_system")
    return A


def project_joseph(geom, X: torch.Tensor, B: torch.Tensor | None = None) -> torch.Tensor:
    """Sinograms (m x k) of the images X (n x k, FP64 CUDA) by Joseph's projector."""
    m, n = system_size(geom)
    k = X.shape[1]
    if B is None:
        B = colmajor(m, k)
    _check(load().ct_project_joseph(ctypes.byref(geometry(geom)), X.data_ptr(), _ld(X), k, B.data_ptr(), _ld(B),
                                    _stream()), "ct_project_joseph")
    return B


def image_quality(X: torch.Tensor, R: torch.Tensor, nx: int, ny: int) -> torch.Tensor:
    """k x 3 tensor of (MSE, PSNR dB, SSIM) per slice of X against R."""
    k = X.shape[1]
    out = torch.empty(3 * max(k, 1), dtype=torch.float64, device=X.device)
    _check(load().ct_image_quality(X.data_ptr(), _ld(X), R.data_ptr(), _ld(R), nx, ny, k, out.data_ptr(),
                                   _stream()), "ct_image_quality")
    return out[:3 * k].view(k, 3)


class Factor:
    """Owning handle of a ``ct_factor``."""

    def __init__(self, handle: int, keep=None):
        self._h = ctypes.c_void_p(handle)
        self._keep = keep  # borrowed matrix for in-place factors

    @property
    def handle(self) -> ctypes.c_void_p:
        if not self._h:
            raise RuntimeError("factor already destroyed")
        return self._h

    def info(self):
        m, n, nb, prec = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int(), ctypes.c_int()
        _check(load().ct_factor_info(self.handle, ctypes.byref(m), ctypes.byref(n), ctypes.byref(nb),
                                     ctypes.byref(prec)), "ct_factor_info")
        return dict(m=m.value, n=n.value, nb=nb.value, prec=Prec(prec.value))

    def data(self):
        """(F, tau) as torch views of the factor's device memory (copies)."""
        F, dt, ld, tau = ctypes.c_void_p(), ctypes.c_int(), ctypes.c_int64(), ctypes.c_void_p()
        _check(load().ct_factor_data(self.handle, ctypes.byref(F), ctypes.byref(dt), ctypes.byref(ld),
                                     ctypes.byref(tau)), "ct_factor_data")
        inf = self.info()
        return F.value, dt.value, ld.value, tau.value, inf

    def status(self) -> int:
        return load().ct_factor_status(self.handle, _stream())

    def destroy(self) -> None:
        if self._h:
            load().ct_factor_destroy(self._h)
            self._h = ctypes.c_void_p()
            self._keep = None

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass


def qr_factor(A: torch.Tensor, prec: Prec = Prec.F64, nb: int = 0, in_place: bool = False,
              tf32_passes: int = 0, outer_nb: int = 0) -> Factor:
    m, n = A.shape
    h = ctypes.c_void_p()
    opts = QrOpts(nb, 1 if in_place else 0, tf32_passes, outer_nb)
    _check(load().ct_qr_factor(A.data_ptr(), _dt(A), m, n, _ld(A), int(prec), ctypes.byref(opts),
                               ctypes.byref(h), _stream()), "ct_qr_factor")
    return Factor(h.value, keep=A if in_place else None)


def qr_factor_host(A: torch.Tensor, device_bytes: int = 0, nb: int = 0, overlap: bool = True) -> Factor:
    """Out-of-core QR of a host FP64 column-major tensor A (overwritten by the
    factor, which borrows it): block columns stream through HBM within
    device_bytes."""
    if A.is_cuda or A.dtype != torch.float64 or A.dim() != 2 or (A.stride(0) != 1 and A.shape[0] > 1):
        raise ValueError("expected a host FP64 column-major matrix")
    m, n = A.shape
    h = ctypes.c_void_p()
    opts = OocOpts(device_bytes, nb, 0 if overlap else 1)
    _check(load().ct_qr_factor_host(A.data_ptr(), m, n, max(A.stride(1), m), ctypes.byref(opts), ctypes.byref(h),
                                    _stream()), "ct_qr_factor_host")
    return Factor(h.value, keep=A)


def factor_save(f: Factor, path: str, tag: int = 0) -> None:
    """Write the factor to a file (ct_factor_save)."""
    _check(load().ct_factor_save(f.handle, os.fsencode(path), tag, _stream()), "ct_factor_save")


def factor_load(path: str) -> tuple[Factor, int]:
    """Read a factor file into a new factor on the current device; returns (factor, tag)."""
    h, tag = ctypes.c_void_p(), ctypes.c_uint64()
    _check(load().ct_factor_load(os.fsencode(path), ctypes.byref(h), ctypes.byref(tag), _stream()),
           "ct_factor_load")
    return Factor(h.value), tag.value


def factor_file_info(path: str) -> dict:
    """Header of a factor file (no GPU needed)."""
    m, n, nb, prec, tag = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int(), ctypes.c_int(), ctypes.c_uint64()
    _check(load().ct_factor_file_info(os.fsencode(path), ctypes.byref(m), ctypes.byref(n), ctypes.byref(nb),
                                      ctypes.byref(prec), ctypes.byref(tag)), "ct_factor_file_info")
    return dict(m=m.value, n=n.value, nb=nb.value, prec=Prec(prec.value), tag=tag.value)


def geometry_hash(geom, lam: float = 0.0) -> int:
    return int(load().ct_geometry_hash(ctypes.byref(geometry(geom)), lam))


def factor_matrix(f: Factor) -> tuple[torch.Tensor, torch.Tensor]:
    """Copies of the factored matrix (R on/above, reflectors below the
    diagonal; the factor's storage type) and of tau (FP64)."""
    inf = f.info()
    _, dt, _, _, _ = f.data()
    dtype = torch.float64 if dt == CT_F64 else torch.float32
    F = colmajor(inf["m"], inf["n"], dtype=dtype)
    tau = torch.empty(inf["n"], dtype=torch.float64, device="cuda")
    _check(load().ct_factor_copy(f.handle, F.data_ptr(), _ld(F), tau.data_ptr(), _stream()),
           "ct_factor_copy")
    return F, tau


def apply_qt(f: Factor, B: torch.Tensor) -> torch.Tensor:
    """B <- Q^T B in place (FP64, m x k column-major)."""
    _check(load().ct_apply_qt(f.handle, B.data_ptr(), _ld(B), B.shape[1], _stream()), "ct_apply_qt")
    return B


def apply_qt_noalloc(f: Factor, B: torch.Tensor) -> torch.Tensor:
    """B <- Q^T B in place without any device allocation (k <= 64 columns)."""
    _check(load().ct_apply_qt_noalloc(f.handle, B.data_ptr(), _ld(B), B.shape[1], _stream()),
           "ct_apply_qt_noalloc")
    return B


def apply_qt_f32(f: Factor, B: torch.Tensor) -> torch.Tensor:
    """B <- Q^T B in place in FP32 (m x k FP32 column-major) with a mixed-precision factor."""
    _check(load().ct_apply_qt_f32(f.handle, B.data_ptr(), _ld(B), B.shape[1], _stream()), "ct_apply_qt_f32")
    return B


def trsm_solve_f32(f: Factor, B: torch.Tensor, transpose: bool = False) -> torch.Tensor:
    """B <- R^{-1} B (or R^{-T} B) in FP32 with a mixed-precision factor's R."""
    _check(load().ct_trsm_solve_f32(f.handle, B.data_ptr(), _ld(B), B.shape[1], 1 if transpose else 0, _stream()),
           "ct_trsm_solve_f32")
    return B


def trsm_solve(f: Factor, B: torch.Tensor) -> torch.Tensor:
    """B[0:n] <- R^{-1} B[0:n] in place (FP64)."""
    _check(load().ct_trsm_solve(f.handle, B.data_ptr(), _ld(B), B.shape[1], _stream()), "ct_trsm_solve")
    return B


@dataclass
class ReconReport:
    status: int
    iterations: int
    last_update: float
    residual: float
    ms_total: float
    ms_build: float = 0.0
    ms_factor: float = 0.0
    ms_solve: float = 0.0


def reconstruct(f: Factor, B: torch.Tensor, A: torch.Tensor | None = None, X: torch.Tensor | None = None,
                max_iter: int = 0, tol: float = 0.0, method: int = REFINE_AUTO, lam: float = 0.0,
                check: bool = True):
    """X = R^{-1}(Q^T B)[0:n], refined with FP64 residuals against A when given.
    Returns (X, ReconReport)."""
    inf = f.info()
    k = B.shape[1]
    if X is None:
        X = colmajor(inf["n"], k, dtype=torch.float64)
    rep = Report()
    ro = RefineOpts(max_iter, lam, tol, method)
    st = load().ct_reconstruct_batch(
        f.handle, A.data_ptr() if A is not None else None, _dt(A) if A is not None else CT_F64,
        _ld(A) if A is not None else 0, B.data_ptr(), _ld(B), X.data_ptr(), _ld(X), k,
        ctypes.byref(ro), ctypes.byref(rep), _stream())
    if check:
        _check(st, "ct_reconstruct_batch")
    return X, ReconReport(st, rep.iterations, rep.last_update, rep.residual, rep.ms_total)


def reconstruct_scan(geom, B, X=None, prec: Prec = Prec.F64, lam: float = 0.0, max_iter: int = 0,
                     tol: float = 0.0, method: int = REFINE_AUTO, check: bool = True):
    """Whole method for one scan (build A, factor, reconstruct).  B and X are
    either CUDA tensors (device buffers) or numpy arrays / CPU tensors (host
    buffers, copied inside the call).  Returns (X, ReconReport)."""
    m, n = system_size(geom, lam)
    rep = Report()
    ro = RefineOpts(max_iter, 0.0, tol, method)
    on_device = isinstance(B, torch.Tensor) and B.is_cuda
    if on_device:
        k = B.shape[1]
        if X is None:
            X = colmajor(n, k)
        args = (B.data_ptr(), _ld(B), X.data_ptr(), _ld(X), k, CT_DEVICE_BUFFERS)
    else:
        Bt = torch.as_tensor(B)
        if Bt.dim() == 1:
            Bt = Bt[:, None]
        k = Bt.shape[1]
        if not (Bt.dtype == torch.float64 and Bt.stride(0) == 1):
            Bt = Bt.t().contiguous().t().to(torch.float64) if Bt.dtype != torch.float64 else Bt.t().contiguous().t()
        if X is None:
            X = torch.empty((k, n), dtype=torch.float64).t()
        ldb = Bt.stride(1) if k > 1 else m
        ldx = X.stride(1) if k > 1 else n
        args = (Bt.data_ptr(), ldb, X.data_ptr(), ldx, k, CT_HOST_BUFFERS)
        B = Bt
    st = load().ct_reconstruct_scan(ctypes.byref(geometry(geom)), lam, int(prec), *args,
                                    ctypes.byref(ro), ctypes.byref(rep), _stream())
    if check:
        _check(st, "ct_reconstruct_scan")
    return X, ReconReport(st, rep.iterations, rep.last_update, rep.residual, rep.ms_total,
                          rep.ms_build, rep.ms_factor, rep.ms_solve)


def gemm_tf32_tn(A: torch.Tensor, B: torch.Tensor, C: torch.Tensor | None = None, accumulate: bool = False,
                 split3: bool = True) -> torch.Tensor:
    """C = A^T B (or C -= A^T B) on the tensor cores; A is K x M, B is K x N,
    FP32 column-major."""
    K, M = A.shape
    N = B.shape[1]
    if C is None:
        C = colmajor(M, N, dtype=torch.float32)
    _check(load().ct_gemm_tf32_tn(M, N, K, A.data_ptr(), _ld(A), B.data_ptr(), _ld(B), C.data_ptr(), _ld(C),
                                  1 if accumulate else 0, 1 if split3 else 0, _stream()), "ct_gemm_tf32_tn")
    return C


def gemm_f16x3_tn(A: torch.Tensor, B: torch.Tensor, C: torch.Tensor | None = None,
                  accumulate: bool = False) -> torch.Tensor:
    """C = A^T B (or C -= A^T B) on the tensor cores with the operands split
    into two FP16 parts each; A is K x M, B is K x N, FP32 column-major."""
    K, M = A.shape
    N = B.shape[1]
    if C is None:
        C = colmajor(M, N, dtype=torch.float32)
    _check(load().ct_gemm_f16x3_tn(M, N, K, A.data_ptr(), _ld(A), B.data_ptr(), _ld(B), C.data_ptr(), _ld(C),
                                   1 if accumulate else 0, _stream()), "ct_gemm_f16x3_tn")
    return C


def batch_plan(shapes, tile: int):
    """The tile-task list of ct_qr_solve_batched for systems of the given
    (m, n, k) sizes (host only, no GPU): an int32 array of ntasks x 25
    records (ct_batch_plan) and the number of tile parts."""
    import numpy as np
    arr = (BatchSystem * len(shapes))()
    for q, (m, n, k) in enumerate(shapes):
        arr[q] = BatchSystem(m, n, None, m, None, m, k)
    nt, npart = ctypes.c_int64(0), ctypes.c_int(0)
    lib = load()
    _check(lib.ct_batch_plan(len(shapes), arr, tile, None, 0, ctypes.byref(nt), ctypes.byref(npart)), "ct_batch_plan")
    out = np.zeros((nt.value, 25), dtype=np.int32)
    _check(lib.ct_batch_plan(len(shapes), arr, tile, out.ctypes.data, nt.value, ctypes.byref(nt),
                             ctypes.byref(npart)), "ct_batch_plan")
    return out, npart.value


def qr_solve_batched_release() -> None:
    """Free what ct_qr_solve_batched keeps on the device for its last batch shape."""
    load().ct_qr_solve_batched_release()


def gemm_status() -> int:
    return load().ct_gemm_status(_stream())


def qr_solve_batched(As, Bs, tile: int = 0, check: bool = True, prec: Prec = Prec.F64, cache: bool = True):
    """Factor and solve a batch of systems in place (lists of column-major
    FP64 CUDA tensors; Bs entries may be None).  Rows [0, n) of every B hold X
    afterwards.  cache=False releases the batch's task list and graph before
    returning (ct_batch_opts.no_cache).  Returns (status, BatchReport)."""
    arr = (BatchSystem * len(As))()
    for q, (A, B) in enumerate(zip(As, Bs)):
        m, n = A.shape
        arr[q] = BatchSystem(m, n, A.data_ptr(), _ld(A), B.data_ptr() if B is not None else None,
                             _ld(B) if B is not None else m, B.shape[1] if B is not None else 0)
    rep = BatchReport()
    st = load().ct_qr_solve_batched(len(As), arr, ctypes.byref(BatchOpts(tile, int(prec), 0 if cache else 1)),
                                    ctypes.byref(rep),
                                    _stream())
    if check:
        _check(st, "ct_qr_solve_batched")
    return st, rep


class Surrogate:
    """The convolutional surrogate of ``include/ctqr.h`` (ct_surrogate_*):
    images are FP64 CUDA tensors of n x k, column-major with ld = n (one
    image per column, pixel iy * nx + ix)."""

    def __init__(self, geom, in_scale: float = 1.0, out_scale: float = 1.0, seed: int = 0):
        h = ctypes.c_void_p()
        opts = SurrogateOpts(in_scale, out_scale, seed)
        _check(load().ct_surrogate_init(ctypes.byref(geometry(geom)), ctypes.byref(opts), ctypes.byref(h)),
               "ct_surrogate_init")
        self.handle = h.value
        self.m, self.n = system_size(geom)

    def __del__(self):
        if getattr(self, "handle", None) and _lib is not None:
            _lib.ct_surrogate_destroy(self.handle)
            self.handle = None

    def num_params(self) -> int:
        return int(load().ct_surrogate_num_params(self.handle))

    def get_params(self):
        import numpy as np
        out = np.zeros(self.num_params(), dtype=np.float32)
        _check(load().ct_surrogate_params(self.handle, out.ctypes.data, 0), "ct_surrogate_params")
        return out

    def set_params(self, p) -> None:
        import numpy as np
        p = np.ascontiguousarray(p, dtype=np.float32)
        assert p.size == self.num_params()
        _check(load().ct_surrogate_params(self.handle, p.ctypes.data, 1), "ct_surrogate_params")

    def backproject(self, B: torch.Tensor, G: torch.Tensor | None = None) -> torch.Tensor:
        k = B.shape[1]
        if G is None:
            G = colmajor(self.n, k, ld=self.n)
        _check(load().ct_surrogate_backproject(self.handle, B.data_ptr(), _ld(B), k, G.data_ptr(), _stream()),
               "ct_surrogate_backproject")
        return G

    def project(self, X: torch.Tensor, B: torch.Tensor | None = None) -> torch.Tensor:
        k = X.shape[1]
        if B is None:
            B = colmajor(self.m, k, ld=self.m)
        _check(load().ct_surrogate_project(self.handle, X.data_ptr(), k, B.data_ptr(), _ld(B), _stream()),
               "ct_surrogate_project")
        return B

    def train_step(self, G: torch.Tensor, X: torch.Tensor, lr: float) -> float:
        loss = ctypes.c_double()
        _check(load().ct_surrogate_train_step(self.handle, G.data_ptr(), X.data_ptr(), G.shape[1], lr,
                                              ctypes.byref(loss), _stream()), "ct_surrogate_train_step")
        return loss.value

    def grad(self, G: torch.Tensor, X: torch.Tensor):
        import numpy as np
        loss = ctypes.c_double()
        g = np.zeros(self.num_params(), dtype=np.float32)
        _check(load().ct_surrogate_grad(self.handle, G.data_ptr(), X.data_ptr(), G.shape[1], ctypes.byref(loss),
                                        g.ctypes.data, _stream()), "ct_surrogate_grad")
        return loss.value, g

    def forward(self, G: torch.Tensor) -> torch.Tensor:
        k = G.shape[1]
        X = colmajor(self.n, k, ld=self.n)
        _check(load().ct_surrogate_forward(self.handle, G.data_ptr(), X.data_ptr(), k, _stream()),
               "ct_surrogate_forward")
        return X

    def infer(self, B: torch.Tensor, tol: float = 1e-3, factor: "Factor | None" = None, lam: float = 0.0,
              max_iter: int = 0, X: torch.Tensor | None = None, check: bool = True):
        """Gated reconstruction.  Returns (X, per-slice residuals, report dict)."""
        k = B.shape[1]
        if X is None:
            X = colmajor(self.n, k, ld=self.n)
        resid = torch.empty(max(k, 1), dtype=torch.float64, device=B.device)
        ro = RefineOpts(max_iter, lam, 0.0, REFINE_AUTO)
        rep = SurrogateReport()
        st = load().ct_surrogate_infer(self.handle, B.data_ptr(), _ld(B), X.data_ptr(), _ld(X), k, tol,
                                       factor.handle if factor is not None else None, ctypes.byref(ro),
                                       resid.data_ptr(), ctypes.byref(rep), _stream())
        if check:
            _check(st, "ct_surrogate_infer")
        return X, resid[:k], dict(status=st, slices=rep.slices, fallbacks=rep.fallbacks,
                                  max_residual=rep.max_residual, ms_total=rep.ms_total,
                                  ms_network=rep.ms_network, ms_gate=rep.ms_gate, ms_fallback=rep.ms_fallback)


def profile_enable(on: bool = True) -> None:
    load().ct_profile_enable(1 if on else 0)


def profile_reset() -> None:
    load().ct_profile_reset()


def profile_kernels() -> list[dict]:
    lib = load()
    n = lib.ct_profile_kernels(None, 0)
    arr = (KernelStats * n)()
    n = lib.ct_profile_kernels(arr, n)
    return [dict(name=a.name.decode(), launches=a.launches, timed=a.timed, ms=a.ms, flops=a.flops,
                 bytes=a.bytes) for a in arr[:n]]


def kernel_launches() -> int:
    return int(load().ct_kernel_launches())
