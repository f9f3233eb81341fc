"""Tensor-core (tcgen05 TF32) contraction C = A^T B used by the trailing
update, against an FP64 product of the same FP32 inputs.

Error bounds (elementwise, relative to (|A|^T |B|)_ij):
  TF32 (1 pass): each product loses at most ~2^-10 per operand to the TF32
  input format -> 4e-3 plus FP32 accumulation K * 2^-24;
  3xTF32: the dropped lo*lo term and the TF32 rounding of the lo parts are
  ~2^-20 each -> 1e-5 plus K * 2^-24.
  FP16 split (h + l, 22 significant bits per operand, three FP16 products):
  ~2^-21 per product -> the same 1e-5 plus K * 2^-24, with B's columns spread
  over twelve decades (the per-column scales keep each column's relative
  accuracy) and A up to 100 in magnitude.
"""
import numpy as np
import pytest
import torch

from paper_1907_01891_gb300 import ctqr
from paper_1907_01891_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def _cm(x):
    """Column-major FP32 CUDA copy with the leading dimension padded to a
    multiple of 4 floats (16-byte column strides, as TMA requires)."""
    rows, cols = x.shape
    t = ctqr.colmajor(rows, cols, dtype=torch.float32, ld=(rows + 3) // 4 * 4)
    t.copy_(torch.as_tensor(x))
    return t


def _case(M, N, K, seed):
    A = I.random_matrix(K, M, seed=seed, dtype=np.float32)
    B = I.random_matrix(K, N, seed=seed + 1, dtype=np.float32)
    ref = A.astype(np.float64).T @ B.astype(np.float64)
    bound = np.abs(A.astype(np.float64)).T @ np.abs(B.astype(np.float64))
    return A, B, ref, bound


@pytest.mark.parametrize("shape", [(128, 128, 32), (200, 300, 100), (64, 16, 1000), (257, 129, 4097),
                                   (1, 1, 1), (130, 5, 31)])
@pytest.mark.parametrize("split3", [False, True])
def test_tc_gemm_store_matches_fp64(shape, split3):
    M, N, K = shape
    A, B, ref, bound = _case(M, N, K, seed=M + N + K)
    C = ctqr.gemm_tf32_tn(_cm(A), _cm(B), split3=split3)
    assert ctqr.gemm_status() == ctqr.CT_OK
    got = C.cpu().numpy().astype(np.float64)
    tol = (1e-5 if split3 else 4e-3) + K * 2.0 ** -24 * 2
    err = np.abs(got - ref) / np.maximum(bound, 1e-30)
    assert err.max() <= tol, (err.max(), tol)


def test_tc_gemm_subtract_in_place_and_3x_is_more_accurate():
    M, N, K = 300, 200, 512
    A, B, ref, bound = _case(M, N, K, seed=5)
    C0 = I.random_matrix(M, N, seed=9, dtype=np.float32)
    Ct = ctqr.to_colmajor(C0)
    ctqr.gemm_tf32_tn(_cm(A), _cm(B), C=Ct, accumulate=True, split3=True)
    got = Ct.cpu().numpy().astype(np.float64)
    want = C0.astype(np.float64) - ref
    assert (np.abs(got - want) / (bound + np.abs(C0))).max() <= 1e-5 + K * 2.0 ** -23
    e1 = np.abs(ctqr.gemm_tf32_tn(_cm(A), _cm(B), split3=False).cpu().numpy() - ref).max()
    e3 = np.abs(ctqr.gemm_tf32_tn(_cm(A), _cm(B), split3=True).cpu().numpy() - ref).max()
    assert e3 < e1 / 50


def test_tc_gemm_respects_leading_dimensions():
    M, N, K = 150, 70, 96
    A, B, ref, bound = _case(M, N, K, seed=3)
    At = ctqr.colmajor(K, M, dtype=torch.float32, ld=K + 4, fill=1e30)
    At.copy_(torch.as_tensor(A))
    Bt = ctqr.colmajor(K, N, dtype=torch.float32, ld=K + 8, fill=1e30)
    Bt.copy_(torch.as_tensor(B))
    C = ctqr.colmajor(M, N, dtype=torch.float32, ld=M + 3, fill=-7.0)
    ctqr.gemm_tf32_tn(At, Bt, C=C, split3=True)
    assert (np.abs(C.cpu().numpy() - ref) / bound).max() <= 1e-5 + K * 2.0 ** -23
    pad = C.as_strided((M + 3, N), (1, M + 3)).cpu().numpy()[M:]
    assert (pad == -7.0).all()


def _case16(M, N, K, seed):
    """A within |A| < 100; B's columns scaled by 10^-9 ... 10^3."""
    A = (I.random_matrix(K, M, seed=seed) * 30.0).clip(-99, 99).astype(np.float32)
    B = I.random_matrix(K, N, seed=seed + 1) * (10.0 ** (np.arange(N) % 13 - 9))[None, :]
    B = B.astype(np.float32)
    ref = A.astype(np.float64).T @ B.astype(np.float64)
    bound = np.abs(A.astype(np.float64)).T @ np.abs(B.astype(np.float64))
    return A, B, ref, bound


@pytest.mark.parametrize("shape", [(128, 128, 32), (200, 300, 100), (64, 16, 1000), (257, 129, 4097),
                                   (1, 1, 1), (130, 5, 31), (256, 700, 20000), (300, 260, 3000)])
def test_f16x3_gemm_store_matches_fp64(shape):
    """The split-K product kernel (one or two 128-row M tiles per CTA, B split
    on chip with its column scales)."""
    M, N, K = shape
    A, B, ref, bound = _case16(M, N, K, seed=M + 2 * N + K)
    C = ctqr.gemm_f16x3_tn(_cm(A), _cm(B))
    assert ctqr.gemm_status() == ctqr.CT_OK
    got = C.cpu().numpy().astype(np.float64)
    tol = 1e-5 + K * 2.0 ** -24 * 2
    err = np.abs(got - ref) / np.maximum(bound, 1e-300)
    assert err.max() <= tol, (err.max(), tol)


@pytest.mark.parametrize("shape", [(300, 200, 256), (129, 130, 100), (1000, 77, 200), (5000, 300, 128), (7, 3, 9)])
def test_f16x3_update_subtracts_in_place(shape):
    """The persistent update kernel C -= A^T B on operands split beforehand."""
    M, N, K = shape
    A, B, ref, bound = _case16(M, N, K, seed=3 * M + N + K)
    C0 = (I.random_matrix(M, N, seed=11) * (10.0 ** (np.arange(N) % 13 - 9))[None, :]).astype(np.float32)
    Ct = ctqr.to_colmajor(C0)
    ctqr.gemm_f16x3_tn(_cm(A), _cm(B), C=Ct, accumulate=True)
    assert ctqr.gemm_status() == ctqr.CT_OK
    got = Ct.cpu().numpy().astype(np.float64)
    want = C0.astype(np.float64) - ref
    err = np.abs(got - want) / (bound + np.abs(C0.astype(np.float64)))
    assert err.max() <= 1e-5 + K * 2.0 ** -23, err.max()


def test_f16x3_is_as_accurate_as_three_pass_tf32():
    M, N, K = 300, 200, 512
    A, B, ref, bound = _case(M, N, K, seed=5)
    e16 = (np.abs(ctqr.gemm_f16x3_tn(_cm(A), _cm(B)).cpu().numpy() - ref) / bound).max()
    e3 = (np.abs(ctqr.gemm_tf32_tn(_cm(A), _cm(B), split3=True).cpu().numpy() - ref) / bound).max()
    assert e16 <= 2 * e3, (e16, e3)
