"""GPU vs oracle parity through the C ABI (paper Eq. (sistema), (QR), (qr1)).

Sizes span several 64-column panels and 64-row tiles with ragged tails; the
oracle computes the same quantities from the same seeded inputs.
Tolerances: the reconstructions X must match the oracle to a relative error of
1e-10 (the accuracy target for the plain and refined paths); the factors
R, V, tau and Q^T B, which a backward-stable QR perturbs by O(kappa * eps),
are held to 1e-11 relative to the largest entry; the system matrix A, whose
entries both sides compute with the same FP64 expressions (up to the last bit
of sin/cos), to 1e-12 absolute.
"""
import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_1907_01891_gb300 import ctqr
from paper_1907_01891_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def _np(t: torch.Tensor) -> np.ndarray:
    torch.cuda.synchronize()
    return t.detach().cpu().numpy()


def _og(g):
    return O.Geometry(*g.as_tuple())


# ---------------------------------------------------------------- system matrix
@pytest.mark.parametrize("geom", [I.CONFIG1["geom"], I.fan_geometry(24, 30, 37),
                                  I.parallel_geometry(20, 13, 29, pixel=0.37),
                                  I.ScanGeometry(0, 8, 8, 1.0, 2, 9, 0.0, np.pi, 0.0, 8.1),
                                  I.scanner_geometry(20, 36, 31)],
                         ids=["config1", "fan24", "par20_pix037", "axis_aligned", "scanner20_eq_angulos"])
def test_system_matrix_matches_oracle(geom):
    A = ctqr.build_system(geom, torch.float64)
    ref = O.system_matrix(_og(geom))
    got = _np(A)
    assert got.shape == ref.shape
    assert np.abs(got - ref).max() <= 1e-12 * geom.pixel
    assert ((got != 0) == (ref != 0)).mean() > 0.9999


def test_system_matrix_fp32_and_lambda_rows():
    geom = I.fan_geometry(16, 20, 25)
    lam = 1e-3
    A32 = _np(ctqr.build_system(geom, torch.float32, lam=lam))
    ref = O.system_matrix(_og(geom))
    m = geom.m
    assert A32.dtype == np.float32
    assert np.abs(A32[:m] - ref.astype(np.float32)).max() <= 1e-6
    assert np.array_equal(A32[m:], (lam * np.eye(geom.n)).astype(np.float32))


def test_system_matrix_respects_leading_dimension():
    geom = I.parallel_geometry(8, 5, 11)
    A = ctqr.colmajor(geom.m, geom.n, torch.float64, ld=geom.m + 13, fill=7.0)
    ctqr.build_system(geom, torch.float64, out=A)
    assert np.abs(_np(A) - O.system_matrix(_og(geom))).max() <= 1e-12
    storage = A.as_strided((geom.m + 13, geom.n), (1, geom.m + 13))
    pad = _np(storage)[geom.m:]
    assert (pad == 7.0).all(), "rows beyond m must not be touched"


# ---------------------------------------------------------------- factorization
SHAPES = [(1, 1), (7, 3), (64, 64), (130, 65), (517, 203), (1000, 129), (2700, 1024)]


@pytest.mark.parametrize("shape", SHAPES)
def test_qr_factor_matches_oracle(shape):
    m, n = shape
    A = I.random_matrix(m, n, seed=m + 7 * n)
    f = ctqr.qr_factor(ctqr.to_colmajor(A))
    assert f.status() == ctqr.CT_OK
    F, tau = ctqr.factor_matrix(f)
    F, tau = _np(F), _np(tau)
    Fo, tauo = O.qr(A)
    scale = max(1.0, np.abs(Fo).max())
    assert np.abs(np.triu(F[:n]) - np.triu(Fo[:n])).max() <= 1e-11 * scale
    assert np.abs(np.tril(F, -1) - np.tril(Fo, -1)).max() <= 1e-11 * max(1.0, np.abs(np.tril(Fo, -1)).max())
    assert np.abs(tau - tauo).max() <= 1e-11


@pytest.mark.parametrize("nb", [8, 16, 33, 64])
def test_qr_panel_widths_agree(nb):
    A = I.random_matrix(300, 150, seed=5)
    f = ctqr.qr_factor(ctqr.to_colmajor(A), nb=nb)
    assert f.info()["nb"] == nb
    F, tau = ctqr.factor_matrix(f)
    Fo, tauo = O.qr(A)
    assert np.abs(np.triu(_np(F)[:150]) - np.triu(Fo[:150])).max() <= 1e-11 * np.abs(Fo).max()
    assert np.abs(_np(tau) - tauo).max() <= 1e-11


def test_qr_factor_ct_matrix_from_device_build():
    g = I.CONFIG1["geom"]
    A = ctqr.build_system(g, torch.float64)
    f = ctqr.qr_factor(A)
    F, tau = ctqr.factor_matrix(f)
    Fo, tauo = O.qr(_np(A))  # oracle on the GPU-built A isolates the QR error
    n = g.n
    assert np.abs(np.triu(_np(F)[:n]) - np.triu(Fo[:n])).max() <= 1e-11 * np.abs(Fo).max()
    assert np.abs(_np(tau) - tauo).max() <= 1e-11


def test_factorization_is_deterministic():
    A = ctqr.to_colmajor(I.random_matrix(700, 300, seed=2))
    F1, t1 = ctqr.factor_matrix(ctqr.qr_factor(A))
    F2, t2 = ctqr.factor_matrix(ctqr.qr_factor(A))
    assert torch.equal(F1, F2) and torch.equal(t1, t2)


# ---------------------------------------------------------------- apply / solve
@pytest.mark.parametrize("shape,k", [((517, 203), 1), ((517, 203), 5), ((1000, 129), 17), ((300, 300), 70)])
def test_apply_qt_and_trsm_match_oracle(shape, k):
    m, n = shape
    A = I.random_matrix(m, n, seed=11)
    B = I.random_matrix(m, k, seed=12)
    f = ctqr.qr_factor(ctqr.to_colmajor(A))
    Fo, tauo = O.qr(A)
    Bg = ctqr.to_colmajor(B)
    ctqr.apply_qt(f, Bg)
    QtB = O.apply_qt(Fo, tauo, B)
    assert np.abs(_np(Bg) - QtB).max() <= 1e-11 * np.abs(QtB).max()
    ctqr.trsm_solve(f, Bg)
    X = O.backsolve(Fo, QtB)
    got = _np(Bg)[:n]
    assert np.linalg.norm(got - X) / np.linalg.norm(X) <= 1e-10


def test_trsm_respects_leading_dimension_and_rows_below_n():
    m, n, k = 400, 150, 3
    A = I.random_matrix(m, n, seed=21)
    f = ctqr.qr_factor(ctqr.to_colmajor(A))
    B = ctqr.colmajor(m, k, ld=m + 5)
    B.copy_(torch.as_tensor(I.random_matrix(m, k, seed=22)))
    before = _np(B)[n:].copy()
    ctqr.trsm_solve(f, B)
    assert np.array_equal(_np(B)[n:], before)


# ---------------------------------------------------------------- reconstruction
def test_reconstruct_config1_matches_oracle():
    g = I.CONFIG1["geom"]
    A = ctqr.build_system(g, torch.float64)
    x_true = I.phantoms(g, I.CONFIG1["seeds"])
    Anp = _np(A)
    b = Anp @ x_true
    f = ctqr.qr_factor(A)
    X, rep = ctqr.reconstruct(f, ctqr.to_colmajor(b))
    Xo = O.lstsq(Anp, b)
    err = np.linalg.norm(_np(X) - Xo) / np.linalg.norm(Xo)
    assert err <= 1e-10
    assert np.linalg.norm(_np(X) - x_true) / np.linalg.norm(x_true) <= 1e-10


def test_reconstruct_multi_rhs_noisy_config4a_subset():
    g = I.CONFIG4A["geom"]
    A = ctqr.build_system(g, torch.float64)
    Anp = _np(A)
    seeds = I.CONFIG4A["seeds"][:40]
    b = I.poisson_noise(Anp @ I.phantoms(g, seeds), g.fov, I.CONFIG4A["noise_i0"], seed=1000)
    f = ctqr.qr_factor(A)
    X, _ = ctqr.reconstruct(f, ctqr.to_colmajor(b))
    Xo = O.lstsq(Anp, b)
    assert np.linalg.norm(_np(X) - Xo) / np.linalg.norm(Xo) <= 1e-10
    # one RHS at a time gives the same columns
    X1, _ = ctqr.reconstruct(f, ctqr.to_colmajor(b[:, 7:8]))
    assert np.linalg.norm(_np(X1)[:, 0] - _np(X)[:, 7]) <= 1e-13 * np.linalg.norm(_np(X)[:, 7])


def test_mixed_fp32_factor_refined_to_fp64_accuracy():
    g = I.CONFIG1["geom"]
    A = ctqr.build_system(g, torch.float64)
    Anp = _np(A)
    x_true = I.phantoms(g, [1, 2, 3])
    b = Anp @ x_true
    f = ctqr.qr_factor(A.to(torch.float32), prec=ctqr.Prec.F32)
    assert f.info()["prec"] == ctqr.Prec.F32
    X0, _ = ctqr.reconstruct(f, ctqr.to_colmajor(b))  # unrefined: FP32-level accuracy
    X, rep = ctqr.reconstruct(f, ctqr.to_colmajor(b), A=A)
    Xo = O.lstsq(Anp, b)
    e0 = np.linalg.norm(_np(X0) - Xo) / np.linalg.norm(Xo)
    e = np.linalg.norm(_np(X) - Xo) / np.linalg.norm(Xo)
    assert e <= 1e-10, (e, rep)
    assert e0 > 1e-9  # the refinement did the work
    assert 1 <= rep.iterations <= 10


# ---------------------------------------------------------------- edge cases
def test_rank_deficient_reported():
    A = I.random_matrix(50, 20, seed=3)
    A[:, 7] = 0.0
    f = ctqr.qr_factor(ctqr.to_colmajor(A))
    assert f.status() == ctqr.CT_ERR_RANK
    A = I.random_matrix(50, 20, seed=3)
    A[:, 9] = A[:, 2]
    f = ctqr.qr_factor(ctqr.to_colmajor(A))
    assert f.status() == ctqr.CT_ERR_RANK


def test_nonfinite_reported():
    A = I.random_matrix(80, 30, seed=4)
    A[10, 5] = np.nan
    f = ctqr.qr_factor(ctqr.to_colmajor(A))
    assert f.status() == ctqr.CT_ERR_NONFINITE


def test_invalid_arguments():
    A = ctqr.to_colmajor(I.random_matrix(10, 20, seed=1))  # m < n
    with pytest.raises(ctqr.CtError) as e:
        ctqr.qr_factor(A)
    assert e.value.status == ctqr.CT_ERR_INVALID
    f = ctqr.qr_factor(ctqr.to_colmajor(I.random_matrix(30, 10, seed=1)))
    short = ctqr.colmajor(20, 2)  # fewer rows than m
    with pytest.raises(ctqr.CtError):
        ctqr.apply_qt(f, short)
    empty = ctqr.colmajor(30, 0)
    assert ctqr.load().ct_apply_qt(f.handle, empty.data_ptr() or 16, 30, 0, None) == ctqr.CT_OK


def test_in_place_factor_borrows_the_matrix():
    A = I.random_matrix(200, 90, seed=8)
    At = ctqr.to_colmajor(A)
    f = ctqr.qr_factor(At, in_place=True)
    Fo, _ = O.qr(A)
    assert np.abs(np.triu(_np(At)[:90]) - np.triu(Fo[:90])).max() <= 1e-11 * np.abs(Fo).max()


def test_mixed_factor_cgls_reaches_least_squares_on_noisy_data():
    """Noisy sinograms make A x = b inconsistent; the FP64 CGLS phase (R from
    the FP32 factor as right preconditioner) must still land on the oracle's
    least-squares solution."""
    g = I.CONFIG4A["geom"]
    A = ctqr.build_system(g, torch.float64)
    Anp = _np(A)
    seeds = I.CONFIG4A["seeds"][:12]
    b = I.poisson_noise(Anp @ I.phantoms(g, seeds), g.fov, I.CONFIG4A["noise_i0"], seed=77)
    Xo = O.lstsq(Anp, b)
    f = ctqr.qr_factor(A.to(torch.float32), prec=ctqr.Prec.F32)
    for method in (ctqr.REFINE_AUTO, ctqr.REFINE_CGLS):
        X, rep = ctqr.reconstruct(f, ctqr.to_colmajor(b), A=A, method=method)
        err = np.linalg.norm(_np(X) - Xo) / np.linalg.norm(Xo)
        assert err <= 1e-10, (method, err, rep)
    # classical refinement alone stalls above the target on inconsistent data
    X, rep = ctqr.reconstruct(f, ctqr.to_colmajor(b), A=A, method=ctqr.REFINE_CLASSICAL, max_iter=8,
                              check=False)
    assert rep.status in (ctqr.CT_OK, ctqr.CT_ERR_NOCONVERGE)


def test_cgls_on_fp64_factor_and_fp32_system_matrix():
    g = I.parallel_geometry(24, 40, 35)
    A = ctqr.build_system(g, torch.float64)
    Anp = _np(A)
    b = I.poisson_noise(Anp @ I.phantoms(g, [4, 5]), g.fov, 1e4, seed=3)
    Xo = O.lstsq(Anp, b)
    f = ctqr.qr_factor(A)
    X, rep = ctqr.reconstruct(f, ctqr.to_colmajor(b), A=A, method=ctqr.REFINE_CGLS)
    assert np.linalg.norm(_np(X) - Xo) / np.linalg.norm(Xo) <= 1e-10
    # residuals against an FP32 copy of A converge to the FP32 system's solution
    A32 = A.to(torch.float32)
    X32, _ = ctqr.reconstruct(f, ctqr.to_colmajor(b), A=A32, method=ctqr.REFINE_CGLS, check=False)
    A32np = _np(A32).astype(np.float64)
    Xo32 = O.lstsq(A32np, b)
    assert np.linalg.norm(_np(X32) - Xo32) / np.linalg.norm(Xo32) <= 1e-9


def test_reconstruct_scan_host_and_device_buffers_agree():
    g = I.CONFIG1["geom"]
    Ao = O.system_matrix(O.Geometry(*g.as_tuple()))
    b = Ao @ I.phantoms(g, [9, 10, 11])
    Xh, rep = ctqr.reconstruct_scan(g, b, prec=ctqr.Prec.F32)
    Xd, _ = ctqr.reconstruct_scan(g, ctqr.to_colmajor(b), prec=ctqr.Prec.F32)
    Xo = O.lstsq(Ao, b)
    assert np.linalg.norm(Xh.numpy() - Xo) / np.linalg.norm(Xo) <= 1e-10
    assert np.linalg.norm(_np(Xd) - Xo) / np.linalg.norm(Xo) <= 1e-10
    assert rep.ms_factor > 0 and rep.ms_build > 0 and rep.ms_solve > 0


# ---------------------------------------------------------------- tensor-core factor
@pytest.mark.parametrize("prec", [ctqr.Prec.TF32, ctqr.Prec.F16X3], ids=["tf32x3", "f16x3"])
@pytest.mark.parametrize("shape", [(300, 200), (700, 300), (1000, 513), (49000, 150), (90000, 150)])
def test_tf32_factor_is_close_to_oracle_and_refines_to_fp64(shape, prec):
    """3xTF32 (or FP16-split) outer updates give an FP32-quality factor (R within ~1e-4 of the
    oracle's, relative to max |R|); refinement then reaches the 1e-10 target.
    The inner panels' updates run as one cooperative launch each: every SM's
    rows in shared memory when its share fits 320, else streamed in chunks of
    320 rows (the 49000- and 90000-row cases); at 90000 rows the Cholesky-QR
    panel's FP32 copy of its rows no longer fits beside the FP64 one, so its
    Gram matrix and row solves run in FP64."""
    m, n = shape
    A = I.random_matrix(m, n, seed=31 + m)
    At = ctqr.to_colmajor(A)
    Af = At.to(torch.float32)
    torch.cuda.synchronize()
    ctqr.profile_reset()
    ctqr.profile_enable(True)
    f = ctqr.qr_factor(Af, prec=prec, nb=32)  # explicit width: no tuning runs inside
    torch.cuda.synchronize()
    ctqr.profile_enable(False)
    launches = {p_["name"]: p_["launches"] for p_ in ctqr.profile_kernels()}
    inner = sum(-(-min(128, n - J) // 32) - 1 for J in range(0, n, 128))
    assert launches.get("inner_update", 0) == inner, launches
    assert f.status() == ctqr.CT_OK
    F, tau = ctqr.factor_matrix(f)
    Fo, tauo = O.qr(A)
    R, Ro = np.triu(_np(F).astype(np.float64)[:n]), np.triu(Fo[:n])
    assert np.abs(R - Ro).max() <= 1e-4 * np.abs(Ro).max()
    b = A @ I.random_matrix(n, 2, seed=1)
    X, rep = ctqr.reconstruct(f, ctqr.to_colmajor(b), A=At)
    Xo = O.lstsq(A, b)
    assert np.linalg.norm(_np(X) - Xo) / np.linalg.norm(Xo) <= 1e-10, rep


def test_tf32_single_pass_option_is_less_accurate_but_refines():
    m, n = 600, 260
    A = I.random_matrix(m, n, seed=41)
    At = ctqr.to_colmajor(A)
    f1 = ctqr.qr_factor(At.to(torch.float32), prec=ctqr.Prec.TF32, tf32_passes=1)
    f3 = ctqr.qr_factor(At.to(torch.float32), prec=ctqr.Prec.TF32, tf32_passes=3)
    Fo, _ = O.qr(A)
    Ro = np.triu(Fo[:n])
    e1 = np.abs(np.triu(_np(ctqr.factor_matrix(f1)[0]).astype(np.float64)[:n]) - Ro).max()
    e3 = np.abs(np.triu(_np(ctqr.factor_matrix(f3)[0]).astype(np.float64)[:n]) - Ro).max()
    assert e3 < e1 / 20
    b = A @ I.random_matrix(n, 1, seed=2)
    X, rep = ctqr.reconstruct(f1, ctqr.to_colmajor(b), A=At)
    Xo = O.lstsq(A, b)
    assert np.linalg.norm(_np(X) - Xo) / np.linalg.norm(Xo) <= 1e-10, rep


@pytest.mark.parametrize("prec", [ctqr.Prec.TF32, ctqr.Prec.F16X3], ids=["tf32x3", "f16x3"])
def test_tf32_ct_reconstruction_config1_and_noisy_subset(prec):
    g = I.CONFIG1["geom"]
    A = ctqr.build_system(g, torch.float64)
    Anp = _np(A)
    b = np.hstack([Anp @ I.phantoms(g, [1]),
                   I.poisson_noise(Anp @ I.phantoms(g, [1001, 1002]), g.fov, 1e4, seed=9)])
    f = ctqr.qr_factor(A.to(torch.float32), prec=prec)
    X, rep = ctqr.reconstruct(f, ctqr.to_colmajor(b), A=A)
    Xo = O.lstsq(Anp, b)
    assert np.linalg.norm(_np(X) - Xo) / np.linalg.norm(Xo) <= 1e-10, rep


@pytest.mark.parametrize("prec", [ctqr.Prec.F64, ctqr.Prec.F32, ctqr.Prec.TF32, ctqr.Prec.F16X3])
def test_lambda_stacked_scan_matches_oracle(prec):
    """[A; lambda I] x = [b; 0] with a rank-deficient A (fan beam with 1.06
    rays per pixel): the stacked system is full rank and every precision path
    lands on the oracle's regularized least-squares solution."""
    g = I.fan_geometry(24, 18, 34)
    lam = 1e-3
    Ao = O.system_matrix(O.Geometry(*g.as_tuple()))
    b = Ao @ I.phantoms(g, [5, 6])
    As = np.vstack([Ao, lam * np.eye(g.n)])
    bs = np.vstack([b, np.zeros((g.n, 2))])
    Xo = O.lstsq(As, bs)
    X, rep = ctqr.reconstruct_scan(g, bs, prec=prec, lam=lam)
    assert np.linalg.norm(X.numpy() - Xo) / np.linalg.norm(Xo) <= 1e-10, rep


@pytest.mark.parametrize("n,k", [(200, 3), (1000, 17), (257, 70), (1300, 40), (700, 64)])
@pytest.mark.parametrize("transpose", [False, True])
def test_fp32_triangular_solve_matches_oracle(n, k, transpose):
    """ct_trsm_solve_f32 (the refinement's preconditioner solve, one
    persistent launch per 64 columns) on a factor whose R is known exactly:
    an upper triangular matrix with FP32-exact entries factors to R = +-A
    (the Householder panel keeps it, the Cholesky-QR panel flips every
    row's sign), so the oracle solves with +-A in FP64."""
    rng = np.random.default_rng(70 + n + k)
    A = np.triu(rng.uniform(-1.0, 1.0, (n, n)) / n)  # diagonally dominant: well conditioned
    A[np.diag_indices(n)] = rng.uniform(1.0, 2.0, n)
    A = A.astype(np.float32).astype(np.float64)
    f = ctqr.qr_factor(ctqr.to_colmajor(A, dtype=torch.float32), prec=ctqr.Prec.F32)
    F, _ = ctqr.factor_matrix(f)
    sign = 1.0 if _np(F)[0, 0] > 0 else -1.0  # which of the two exact R the panel produced
    R = sign * A
    Y = rng.standard_normal((n, k)).astype(np.float32)
    B = ctqr.to_colmajor(Y, dtype=torch.float32)
    ctqr.trsm_solve_f32(f, B, transpose=transpose)
    X = _np(B).astype(np.float64)
    if transpose:
        ref = np.linalg.solve(R.T, Y.astype(np.float64))   # lower triangular system, library solve
    else:
        ref = O.backsolve(np.asfortranarray(R), np.asfortranarray(Y.astype(np.float64)))
    err = np.linalg.norm(X - ref) / np.linalg.norm(ref)
    assert err <= 1e-5, err


@pytest.mark.parametrize("prec", [ctqr.Prec.TF32, ctqr.Prec.F16X3], ids=["tf32x3", "f16x3"])
@pytest.mark.parametrize("shape,k", [((700, 300), 3), ((1200, 520), 17)])
def test_tf32_factor_qt_by_outer_blocks(shape, k, prec):
    """Q^T of a two-level TF32 factor is applied by 128-column outer blocks
    (the block reflector through S = diag(1/tau) + striu(V^T V)); it matches
    the oracle's Q^T to the factor's FP32-level accuracy, and the per-panel
    application (the allocation-free entry point, k <= 64) to the same level."""
    m, n = shape
    A = I.random_matrix(m, n, seed=90 + n)
    B = I.random_matrix(m, k, seed=91 + n)
    f = ctqr.qr_factor(ctqr.to_colmajor(A, dtype=torch.float32), prec=prec)
    Y = _np(ctqr.apply_qt(f, ctqr.to_colmajor(B)))
    Yp = _np(ctqr.apply_qt_noalloc(f, ctqr.to_colmajor(B)))
    Fo, tau = O.qr(A)
    Yo = O.apply_qt(Fo, tau, B)
    # rows of Q^T B are fixed up to the sign of each reflector's R_ii: compare
    # with the signs of the two R diagonals aligned
    F, _ = ctqr.factor_matrix(f)
    sgn = np.sign(np.diag(_np(F).astype(np.float64)[:n])) * np.sign(np.diag(Fo[:n]))
    Yo_top = Yo[:n] * sgn[:, None]
    assert np.linalg.norm(Y[:n] - Yo_top) <= 1e-4 * np.linalg.norm(Yo_top)
    assert np.linalg.norm(Y - Yp) <= 1e-5 * np.linalg.norm(Y)
    assert abs(np.linalg.norm(Y) - np.linalg.norm(B)) <= 1e-5 * np.linalg.norm(B)  # orthogonal invariance


@pytest.mark.parametrize("prec,shape,k", [(ctqr.Prec.TF32, (1200, 520), 17), (ctqr.Prec.TF32, (700, 300), 3),
                                          (ctqr.Prec.TF32, (700, 300), 40), (ctqr.Prec.TF32, (24500, 260), 5),
                                          (ctqr.Prec.F32, (500, 200), 4), (ctqr.Prec.F16X3, (1200, 520), 17),
                                          (ctqr.Prec.F16X3, (24500, 260), 5)])
def test_fp32_qt_matches_oracle_with_the_factors_reflectors(prec, shape, k):
    """ct_apply_qt_f32 (Q^T B in FP32, the refinement's first solve) against
    the oracle's reflector-by-reflector Q^T built from the factor's own V and
    tau, i.e. the same orthogonal matrix in FP64.  TF32 factors with k <= 32
    whose rows fit 160 per SM take the one-launch path over all 128-column
    outer blocks (one qt_outer launch); k > 32, taller matrices and one-level
    factors take the block-by-block path (none)."""
    m, n = shape
    A = I.random_matrix(m, n, seed=30 + n)
    B = I.random_matrix(m, k, seed=31 + n).astype(np.float32)
    f = ctqr.qr_factor(ctqr.to_colmajor(A, dtype=torch.float32), prec=prec)
    F, tau = ctqr.factor_matrix(f)
    Yo = O.apply_qt(_np(F).astype(np.float64), _np(tau), B.astype(np.float64))
    Bg = ctqr.to_colmajor(B, dtype=torch.float32)
    torch.cuda.synchronize()
    ctqr.profile_reset()
    ctqr.profile_enable(True)
    ctqr.apply_qt_f32(f, Bg)
    torch.cuda.synchronize()
    ctqr.profile_enable(False)
    launches = {p_["name"]: p_["launches"] for p_ in ctqr.profile_kernels()}
    Y = _np(Bg).astype(np.float64)
    assert np.linalg.norm(Y - Yo) <= 2e-5 * np.linalg.norm(B), np.linalg.norm(Y - Yo) / np.linalg.norm(B)
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    one_launch = prec in (ctqr.Prec.TF32, ctqr.Prec.F16X3) and k <= 32 and -(-m // sms) <= 160 and n > 128
    assert launches.get("qt_outer", 0) == (1 if one_launch else 0), launches


def test_tf32_factor_with_lookahead_refines_to_fp64(monkeypatch):
    """The opt-in look-ahead (deferred outer-block updates on a second stream
    while the next panels run on reserved SMs) gives the same solution."""
    monkeypatch.setenv("CTQR_LOOKAHEAD", "1")
    m, n = 2100, 1000
    A = I.random_matrix(m, n, seed=77)
    At = ctqr.to_colmajor(A)
    f = ctqr.qr_factor(At.to(torch.float32), prec=ctqr.Prec.TF32)
    assert f.status() == ctqr.CT_OK
    b = A @ I.random_matrix(n, 3, seed=78)
    X, rep = ctqr.reconstruct(f, ctqr.to_colmajor(b), A=At)
    Xo = O.lstsq(A, b)
    assert np.linalg.norm(_np(X) - Xo) / np.linalg.norm(Xo) <= 1e-10, rep


def test_allocation_failure_is_reported_without_leaking(monkeypatch):
    """Host-side injection (CTQR_FAULT_NOMEM): the factorization reports
    CT_ERR_NOMEM and frees what it had allocated; the next call works."""
    A = ctqr.to_colmajor(I.random_matrix(400, 200, seed=5))
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    monkeypatch.setenv("CTQR_FAULT_NOMEM", "1")
    with pytest.raises(ctqr.CtError) as ei:
        ctqr.qr_factor(A)
    assert ei.value.status == ctqr.CT_ERR_NOMEM
    monkeypatch.delenv("CTQR_FAULT_NOMEM")
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 >= free0 - (1 << 20)
    f = ctqr.qr_factor(A)
    assert f.status() == ctqr.CT_OK


def test_refinement_cap_reports_noconverge():
    """A mixed-precision factor on noisy data with the refinement capped at
    one correction does not reach the tolerance: CT_ERR_NOCONVERGE, finite X."""
    g = I.CONFIG1["geom"]
    A = ctqr.build_system(g, torch.float64)
    Anp = _np(A)
    b = I.poisson_noise(Anp @ I.phantoms(g, [1001, 1002]), g.fov, 1e4, seed=9)
    f = ctqr.qr_factor(A.to(torch.float32), prec=ctqr.Prec.F32)
    X, rep = ctqr.reconstruct(f, ctqr.to_colmajor(b), A=A, max_iter=1, tol=1e-14, check=False)
    assert rep.status == ctqr.CT_ERR_NOCONVERGE
    assert np.all(np.isfinite(_np(X)))


@pytest.mark.parametrize("prec", [ctqr.Prec.TF32, ctqr.Prec.F16X3], ids=["tf32x3", "f16x3"])
@pytest.mark.parametrize("shape", [(400, 200), (900, 300), (1500, 700), (3000, 1100)])
def test_tf32_outer_blocks_of_256_and_128_agree_and_refine(shape, prec):
    """The trailing update with 256-column outer blocks (two 128-column
    halves merged into one compact-WY reflector, T = [[T_A, T_AB], [0, T_B]])
    against 128-column blocks: both R factors are FP32-quality copies of the
    oracle's (1e-4 relative to max |R|), and both refine to the oracle's
    solution (1e-10).  The shapes cover a second half narrower than 128, a
    first half that is the last block, and several whole 256-column blocks."""
    m, n = shape
    A = I.random_matrix(m, n, seed=400 + n)
    At = ctqr.to_colmajor(A)
    Fo, _ = O.qr(A)
    Ro = np.triu(Fo[:n])
    b = A @ I.random_matrix(n, 2, seed=401)
    Xo = O.lstsq(A, b)
    for outer in (128, 256):
        f = ctqr.qr_factor(At.to(torch.float32), prec=prec, outer_nb=outer)
        assert f.status() == ctqr.CT_OK
        F, _ = ctqr.factor_matrix(f)
        R = np.triu(_np(F).astype(np.float64)[:n])
        assert np.abs(R - Ro).max() <= 1e-4 * np.abs(Ro).max(), outer
        X, rep = ctqr.reconstruct(f, ctqr.to_colmajor(b), A=At)
        assert np.linalg.norm(_np(X) - Xo) / np.linalg.norm(Xo) <= 1e-10, (outer, rep)
        # Q^T by 128-column blocks uses the per-half V^T V and T the factor keeps
        B = I.random_matrix(m, 3, seed=402)
        Y = _np(ctqr.apply_qt(f, ctqr.to_colmajor(B)))
        assert abs(np.linalg.norm(Y) - np.linalg.norm(B)) <= 1e-5 * np.linalg.norm(B)


def test_qr_options_reject_bad_outer_width():
    A = ctqr.to_colmajor(I.random_matrix(300, 200, seed=1), dtype=torch.float32)
    with pytest.raises(ctqr.CtError) as e:
        ctqr.qr_factor(A, prec=ctqr.Prec.TF32, outer_nb=192)
    assert e.value.status == ctqr.CT_ERR_INVALID


@pytest.mark.parametrize("cond,bound", [(1e3, 2e-6), (1e6, 2e-5)])
def test_fp32_panel_gram_is_better_than_fp32(cond, bound):
    """One 32-column panel of an FP32-stored factor with condition number
    1e3: the Cholesky-QR panel forms its Gram matrix as compensated FP32
    products (about twice FP32's precision); in plain FP32 the Gram's error,
    amplified by kappa^2 = 1e6, would put R off by ~1e-1 relative.  R must
    match the oracle's R (of the same FP32-exact data) to FP32 storage level.
    With condition 1e6 the panel's kappa_1(R1) exceeds the Cholesky-QR limit
    and it falls back to per-column Householder, again to FP32 level."""
    rng = np.random.default_rng(int(cond))
    m, n = 5000, 32
    U, _ = np.linalg.qr(rng.standard_normal((m, n)))
    Vt, _ = np.linalg.qr(rng.standard_normal((n, n)))
    A = (U * np.logspace(0, -np.log10(cond), n)) @ Vt.T
    A = A.astype(np.float32).astype(np.float64)
    f = ctqr.qr_factor(ctqr.to_colmajor(A, dtype=torch.float32), prec=ctqr.Prec.F32, nb=32)
    F, _ = ctqr.factor_matrix(f)
    R = np.triu(_np(F).astype(np.float64)[:n])
    Fo, _ = O.qr(A)
    Ro = np.triu(Fo[:n])
    sgn = np.sign(np.diag(R)) * np.sign(np.diag(Ro))  # rows fixed up to sign
    err = np.abs(R - sgn[:, None] * Ro).max() / np.abs(Ro).max()
    assert err <= bound, err


def test_tf32_factor_widths_are_tuned_and_cached(tmp_path, monkeypatch):
    """With the widths left open, a TF32 factorization takes the panel and
    outer-block widths the tuner measured for its size class (16 or 32; 128
    or 256) and caches them in the JSON file; the second factorization of the
    same class reuses the cached pair (no measurement: no extra launches)."""
    cache = tmp_path / "tune.json"
    monkeypatch.setenv("CTQR_TUNE_CACHE", str(cache))
    monkeypatch.delenv("CTQR_NO_TUNE", raising=False)
    A = I.random_matrix(3000, 700, seed=61)
    Af = ctqr.to_colmajor(A, dtype=torch.float32)
    f1 = ctqr.qr_factor(Af, prec=ctqr.Prec.TF32)
    assert f1.info()["nb"] in (16, 32)
    import json
    text = json.loads(cache.read_text())
    # the key of this size class (log2 m = 12, log2 n = 9, 3xTF32); the file
    # also carries the classes tuned earlier in the process
    keys = [k for k in text if k.startswith("factor_tf32/") and k.endswith("/passes=3/log2m=12/log2n=9")]
    assert len(keys) == 1 and text[keys[0]] // 1000 == f1.info()["nb"] and text[keys[0]] % 1000 in (128, 256)
    torch.cuda.synchronize()
    ctqr.profile_reset()
    ctqr.profile_enable(True)
    f2 = ctqr.qr_factor(Af, prec=ctqr.Prec.TF32)
    torch.cuda.synchronize()
    ctqr.profile_enable(False)
    panels = {p_["name"]: p_["launches"] for p_ in ctqr.profile_kernels()}["panel_qr"]
    assert panels == -(-700 // f2.info()["nb"])  # one factorization's panels, no tuning runs
    b = A @ I.random_matrix(700, 1, seed=62)
    X, rep = ctqr.reconstruct(f2, ctqr.to_colmajor(b), A=ctqr.to_colmajor(A))
    Xo = O.lstsq(A, b)
    assert np.linalg.norm(_np(X) - Xo) / np.linalg.norm(Xo) <= 1e-10, rep


@pytest.mark.parametrize("shape,nb", [((1000, 513), 64), ((2700, 1024), 24), ((700, 300), 40)])
def test_fp64_two_level_factor_matches_oracle(shape, nb):
    """FP64 factorization with the trailing matrix updated once per outer
    block of (128 // nb) * nb columns (the form tall FP64 matrices take when
    their panels must be narrow): R, V and tau against the oracle (1e-11), the
    solution to 1e-10, and Q^T through the panel T blocks unchanged."""
    m, n = shape
    A = I.random_matrix(m, n, seed=800 + n)
    f = ctqr.qr_factor(ctqr.to_colmajor(A), nb=nb, outer_nb=128)
    assert f.status() == ctqr.CT_OK and f.info()["nb"] == nb
    F, tau = ctqr.factor_matrix(f)
    Fo, tauo = O.qr(A)
    F, tau = _np(F), _np(tau)
    scale = np.abs(Fo).max()
    assert np.abs(np.triu(F[:n]) - np.triu(Fo[:n])).max() <= 1e-11 * scale
    assert np.abs(np.tril(F, -1) - np.tril(Fo, -1)).max() <= 1e-11 * max(1.0, np.abs(np.tril(Fo, -1)).max())
    assert np.abs(tau - tauo).max() <= 1e-11
    b = I.random_matrix(m, 3, seed=801)
    X, _ = ctqr.reconstruct(f, ctqr.to_colmajor(b))
    Xo = O.lstsq(A, b)
    assert np.linalg.norm(_np(X) - Xo) / np.linalg.norm(Xo) <= 1e-10
