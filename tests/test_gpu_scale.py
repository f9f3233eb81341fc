"""Parity at scale: the paths the 256 x 256 and 128 x 128 workloads take,
against the oracle element by element (paper Eq. (QR), (qr1)).

The sizes are chosen so that one system crosses every size threshold of the
mixed-precision path the benchmark times -- more than 32 outer blocks of 128
columns and more than 32 block rows of the FP32 triangular solve, the
one-launch Q^T, the fused inner updates, the Cholesky-QR panel, and noisy data
(so the refinement goes to CGLS) -- and a tall system has the 135,232 rows of
the lambda-stacked 256 x 256 system (the per-column panel, Q^T block by block,
the inner update streamed through shared memory in chunks of rows).  Tolerance: the 1e-10 relative error of the
reconstruction target, on every element of X (max norm over the max of
|X_oracle|) and in the Frobenius norm.  The oracle's solution of each system
is computed once per module (it takes seconds on the host cores)."""
import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_1907_01891_gb300 import ctqr
from paper_1907_01891_gb300 import inputs as I

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


def _np(t):
    torch.cuda.synchronize()
    return t.detach().cpu().numpy()


def _close(X, Xo, tol=1e-10):
    X = np.asarray(X)
    fro = np.linalg.norm(X - Xo) / np.linalg.norm(Xo)
    elem = np.abs(X - Xo).max() / np.abs(Xo).max()
    return fro <= tol and elem <= tol, (fro, elem)


@pytest.fixture(scope="module")
def fan72():
    """72 x 72 fan beam, 72 views x 103 bins: 7416 x 5184 (40.5 outer blocks,
    41 FP32 block rows), Poisson-noisy sinograms of four phantoms."""
    g = I.fan_geometry(72, 72, 103)
    Ao = O.system_matrix(O.Geometry(*g.as_tuple()))
    b = I.poisson_noise(Ao @ I.phantoms(g, [300, 301, 302, 303]), g.fov, 1e5, seed=300)
    Xo = O.lstsq(Ao, b)
    return g, Ao, b, Xo


def test_fan72_fp64_path_matches_oracle(fan72):
    g, Ao, b, Xo = fan72
    A = ctqr.build_system(g, torch.float64)
    assert np.abs(_np(A) - Ao).max() <= 1e-12
    f = ctqr.qr_factor(A)
    assert f.status() == ctqr.CT_OK
    X, _ = ctqr.reconstruct(f, ctqr.to_colmajor(b))
    ok, e = _close(_np(X), Xo)
    assert ok, e


@pytest.mark.parametrize("prec", [ctqr.Prec.TF32, ctqr.Prec.F16X3], ids=["tf32x3", "f16x3"])
def test_fan72_tf32_path_crosses_every_threshold_and_matches_oracle(fan72, prec):
    g, Ao, b, Xo = fan72
    m, n = g.m, g.n
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    assert n // 128 > 32 and n // 128 > 32           # outer blocks, FP32 block rows
    assert -(-m // sms) <= 160                        # one-launch Q^T fits
    A32 = ctqr.build_system(g, torch.float32)
    A64 = ctqr.build_system(g, torch.float64)
    torch.cuda.synchronize()
    ctqr.profile_reset()
    ctqr.profile_enable(True)
    f = ctqr.qr_factor(A32, prec)
    X, rep = ctqr.reconstruct(f, ctqr.to_colmajor(b), A=A64)
    torch.cuda.synchronize()
    ctqr.profile_enable(False)
    launches = {p["name"]: p["launches"] for p in ctqr.profile_kernels()}
    assert launches.get("inner_update", 0) > 0, launches   # fused inner updates
    assert launches.get("qt_outer", 0) >= 1, launches      # one-launch Q^T of X_0
    assert launches.get("tc_update", 0) > 32, launches     # tensor-core outer updates
    assert rep.iterations >= 2, rep                         # noisy data: CGLS steps
    ok, e = _close(_np(X), Xo)
    assert ok, (e, rep)


@pytest.fixture(scope="module")
def tall():
    """The row count of the lambda-stacked 256 x 256 system (135,232) with
    1024 columns: a random matrix with column scales spread over three
    decades (condition ~1e3), two noisy right-hand sides."""
    m, n = 135232, 1024
    A = I.random_matrix(m, n, seed=501)
    A *= np.logspace(0, -3, n)[None, :]
    rng = np.random.default_rng(502)
    b = A @ rng.standard_normal((n, 2)) + 1e-3 * rng.standard_normal((m, 2))
    Xo = O.lstsq(A, b)
    return A, np.asfortranarray(b), Xo


@pytest.mark.parametrize("prec", [ctqr.Prec.F64, ctqr.Prec.TF32, ctqr.Prec.F16X3])
def test_tall_135232_rows_matches_oracle(tall, prec):
    A, b, Xo = tall
    At = ctqr.to_colmajor(A)
    if prec == ctqr.Prec.F64:
        f = ctqr.qr_factor(At)
        X, rep = ctqr.reconstruct(f, ctqr.to_colmajor(b))
    else:
        f = ctqr.qr_factor(At.to(torch.float32), prec)
        X, rep = ctqr.reconstruct(f, ctqr.to_colmajor(b), A=At)
    assert f.status() == ctqr.CT_OK
    ok, e = _close(_np(X), Xo)
    assert ok, (e, rep)


def test_config4a_512_right_hand_sides_in_one_call():
    """512 Poisson-noisy sinograms (I0 = 1e4) of the 32 x 32 parallel-beam
    system through one factor in one multi-RHS call, FP64 and the refined
    TF32 factor, against the oracle; one column alone gives the same result."""
    g = I.CONFIG4A["geom"]
    seeds = I.CONFIG4A["seeds"]
    assert len(seeds) == 512
    A = ctqr.build_system(g, torch.float64)
    Ao = _np(A)
    b = I.poisson_noise(Ao @ I.phantoms(g, seeds), g.fov, I.CONFIG4A["noise_i0"], seed=seeds[0])
    Xo = O.lstsq(Ao, b)
    f = ctqr.qr_factor(A)
    X, _ = ctqr.reconstruct(f, ctqr.to_colmajor(b))
    ok, e = _close(_np(X), Xo)
    assert ok, e
    x1, _ = ctqr.reconstruct(f, ctqr.to_colmajor(b[:, 311:312]))
    assert np.abs(_np(x1)[:, 0] - _np(X)[:, 311]).max() <= 1e-13 * np.abs(_np(X)[:, 311]).max()
    for prec in (ctqr.Prec.TF32, ctqr.Prec.F16X3):
        ft = ctqr.qr_factor(A.to(torch.float32), prec)
        Xt, rep = ctqr.reconstruct(ft, ctqr.to_colmajor(b), A=A)
        ok, e = _close(_np(Xt), Xo)
        assert ok, (prec, e, rep)
