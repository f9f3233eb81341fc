"""The allocation-free Q^T entry point (ct_apply_qt_noalloc), called through the
C ABI, against the allocating ct_apply_qt on the same factor and inputs, two
calls in a row (the second call reuses the static workspace the first one
left behind).  Tolerance: the same 1e-11 relative bound as the Q^T parity tests
(both paths do identical arithmetic up to the row splitting of V^T B).  Each
result is also held against the oracle's reflector-by-reflector Q^T built from
the factor's own V and tau (Sec. II-C-4): 1e-11 for FP64 factors, 2e-5 for
FP32-stored ones (whose T was formed before V was rounded to FP32).
Callers that cannot allocate are modelled with the library's allocation-
failure injection: with it on, the allocating entry point fails and this one
still works.  A tall case (9000 rows, k = 64) fills the static workspace: 64
row splits of V^T B."""
import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_1907_01891_gb300 import ctqr
from paper_1907_01891_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("prec,m,n,ks", [(ctqr.Prec.F64, 1500, 330, (37, 64)), (ctqr.Prec.F32, 1500, 330, (37, 64)),
                                         (ctqr.Prec.F64, 9000, 330, (64, 64))])
def test_noalloc_apply_qt_matches_allocating_entry_point_twice(prec, m, n, ks, monkeypatch):
    lib = ctqr.load()
    A = ctqr.to_colmajor(I.random_matrix(m, n, seed=101))
    f = ctqr.qr_factor(A if prec == ctqr.Prec.F64 else A.to(torch.float32), prec=prec)
    refs = []
    for call, k in enumerate(ks):
        B = I.random_matrix(m, k, seed=200 + call)
        ref = ctqr.to_colmajor(B)
        ctqr.apply_qt(f, ref)
        refs.append((B, ref))
    F, tau = ctqr.factor_matrix(f)
    torch.cuda.synchronize()
    Fo, tauo = F.cpu().numpy().astype(np.float64), tau.cpu().numpy()
    qtol = 1e-11 if prec == ctqr.Prec.F64 else 2e-5
    monkeypatch.setenv("CTQR_FAULT_NOMEM", "1")  # every library allocation now fails
    s = torch.cuda.current_stream().cuda_stream
    for B, ref in refs:
        k = B.shape[1]
        got = ctqr.to_colmajor(B)
        assert lib.ct_apply_qt(f.handle, ctqr.to_colmajor(B).data_ptr(), m, k, s) == ctqr.CT_ERR_NOMEM
        st = lib.ct_apply_qt_noalloc(f.handle, got.data_ptr(), m, k, s)
        assert st == ctqr.CT_OK
        torch.cuda.synchronize()
        r, g = ref.cpu().numpy(), got.cpu().numpy()
        assert np.abs(g - r).max() <= 1e-11 * np.abs(r).max()
        Yo = O.apply_qt(Fo, tauo, B)
        assert np.abs(g - Yo).max() <= qtol * np.abs(Yo).max(), np.abs(g - Yo).max() / np.abs(Yo).max()


def test_noalloc_apply_qt_rejects_more_columns_than_its_workspace():
    lib = ctqr.load()
    A = ctqr.to_colmajor(I.random_matrix(200, 50, seed=5))
    f = ctqr.qr_factor(A)
    B = ctqr.colmajor(200, 65, fill=0.0)
    st = lib.ct_apply_qt_noalloc(f.handle, B.data_ptr(), 200, 65, torch.cuda.current_stream().cuda_stream)
    assert st == ctqr.CT_ERR_INVALID
