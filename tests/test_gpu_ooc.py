"""Out-of-core factorization and solve (ct_qr_factor_host): the matrix and its
factor live in host memory and stream through HBM by block columns (the
paper's out-of-core algorithm-by-blocks, Sec. II-B / II-C, with host memory in
place of the disk).  A small device budget forces several block columns (and
a ragged last one); the factor must equal the oracle's Householder QR (R, V,
tau within 1e-11 of the largest entry, the bound of the in-HBM factor tests)
and the reconstruction the oracle's solution (1e-10).  The copy-stream
(overlapped) and single-stream runs must agree bitwise."""
import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_1907_01891_gb300 import ctqr
from paper_1907_01891_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def _host(A):
    """Page-locked column-major FP64 host copy of A."""
    m, n = A.shape
    H = torch.empty((n, m), dtype=torch.float64).pin_memory().t()
    H.copy_(torch.as_tensor(A))
    return H


def _np(t):
    torch.cuda.synchronize()
    return t.detach().cpu().numpy()


def _budget(m, bw):
    return 3 * ((m + 3) // 4 * 4) * bw * 8 + 4096


@pytest.mark.parametrize("shape,bw", [((2700, 1024), 128), ((3000, 1100), 256), ((900, 700), 64)])
def test_host_factor_matches_oracle(shape, bw):
    m, n = shape
    A = I.random_matrix(m, n, seed=m + n)
    H = _host(A)
    f = ctqr.qr_factor_host(H, device_bytes=_budget(m, bw), nb=64)
    assert f.status() == ctqr.CT_OK
    Fo, tauo = O.qr(A)
    F = H.numpy()
    scale = np.abs(Fo).max()
    assert np.abs(np.triu(F[:n]) - np.triu(Fo[:n])).max() <= 1e-11 * scale
    assert np.abs(np.tril(F, -1) - np.tril(Fo, -1)).max() <= 1e-11 * max(1.0, np.abs(np.tril(Fo, -1)).max())
    Fd, tau = ctqr.factor_matrix(f)  # the host matrix copied to HBM, tau from HBM
    assert np.array_equal(_np(Fd), F)
    assert np.abs(_np(tau) - tauo).max() <= 1e-11


@pytest.mark.parametrize("overlap", [True, False])
def test_host_factor_reconstruction_matches_oracle(overlap):
    g = I.CONFIG1["geom"]
    Ao = O.system_matrix(O.Geometry(*g.as_tuple()))
    b = I.poisson_noise(Ao @ I.phantoms(g, list(range(1000, 1017))), g.fov, 1e4, seed=17)
    H = _host(Ao)
    f = ctqr.qr_factor_host(H, device_bytes=_budget(g.m, 128), overlap=overlap)
    assert f.status() == ctqr.CT_OK
    X, _ = ctqr.reconstruct(f, ctqr.to_colmajor(b))
    Xo = O.lstsq(Ao, b)
    assert np.linalg.norm(_np(X) - Xo) / np.linalg.norm(Xo) <= 1e-10
    assert np.abs(_np(X) - Xo).max() <= 1e-10 * np.abs(Xo).max()


def test_overlapped_and_serial_streaming_agree_bitwise():
    A = I.random_matrix(1500, 600, seed=9)
    B = I.random_matrix(1500, 5, seed=10)
    out = []
    for overlap in (True, False):
        H = _host(A)
        f = ctqr.qr_factor_host(H, device_bytes=_budget(1500, 128), overlap=overlap)
        Bg = ctqr.to_colmajor(B)
        ctqr.apply_qt(f, Bg)
        ctqr.trsm_solve(f, Bg)
        out.append((H.numpy().copy(), _np(Bg)))
    assert np.array_equal(out[0][0], out[1][0]) and np.array_equal(out[0][1], out[1][1])


def test_host_factor_budget_too_small_and_unsupported_uses():
    A = I.random_matrix(500, 200, seed=3)
    with pytest.raises(ctqr.CtError) as e:
        ctqr.qr_factor_host(_host(A), device_bytes=3 * 500 * 8 * 8)  # under one 64-column block
    assert e.value.status == ctqr.CT_ERR_NOMEM
    f = ctqr.qr_factor_host(_host(A), device_bytes=_budget(500, 64))
    with pytest.raises(ctqr.CtError) as e:
        ctqr.apply_qt_f32(f, ctqr.to_colmajor(I.random_matrix(500, 2, seed=4), dtype=torch.float32))
    assert e.value.status == ctqr.CT_ERR_UNSUPPORTED
    with pytest.raises(ctqr.CtError) as e:
        ctqr.apply_qt_noalloc(f, ctqr.to_colmajor(I.random_matrix(500, 2, seed=4)))
    assert e.value.status == ctqr.CT_ERR_UNSUPPORTED


def test_host_factor_reports_rank_deficiency():
    A = I.random_matrix(600, 300, seed=5)
    A[:, 200] = A[:, 17]
    f = ctqr.qr_factor_host(_host(A), device_bytes=_budget(600, 64))
    assert f.status() == ctqr.CT_ERR_RANK
