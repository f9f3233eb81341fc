"""Pins for the oracle's Householder QR, Q^T application and back substitution
(paper Eq. (QR) and Eq. (qr1)).  Each test checks the oracle against something
other than itself: exact rational arithmetic, LAPACK's dgeqrf, or an identity
that any correct QR must satisfy."""
from fractions import Fraction

import numpy as np
import pytest

from oracle import oracle as O
from paper_1907_01891_gb300 import inputs as I

EPS = np.finfo(np.float64).eps


def _exact_normal_equations(A, b):
    """x solving A^T A x = A^T b in exact rationals (Gauss-Jordan)."""
    m, n = A.shape
    Af = [[Fraction(int(v)) for v in row] for row in A]
    bf = [Fraction(int(v)) for v in b]
    M = [[sum(Af[r][i] * Af[r][j] for r in range(m)) for j in range(n)] +
         [sum(Af[r][i] * bf[r] for r in range(m))] for i in range(n)]
    for c in range(n):
        p = next(r for r in range(c, n) if M[r][c] != 0)
        M[c], M[p] = M[p], M[c]
        piv = M[c][c]
        M[c] = [v / piv for v in M[c]]
        for r in range(n):
            if r != c and M[r][c] != 0:
                f = M[r][c]
                M[r] = [a - f * b_ for a, b_ in zip(M[r], M[c])]
    return np.array([float(M[i][n]) for i in range(n)])


@pytest.mark.parametrize("seed", range(6))
def test_tiny_integer_systems_match_exact_normal_equations(seed):
    rng = np.random.default_rng(seed)
    n = int(rng.integers(1, 7))
    m = int(rng.integers(n, 9))
    while True:
        A = rng.integers(-5, 6, size=(m, n)).astype(np.float64)
        if np.linalg.matrix_rank(A) == n:
            break
    b = rng.integers(-9, 10, size=m).astype(np.float64)
    x_exact = _exact_normal_equations(A, b)
    x = O.lstsq(A, b)
    kappa = np.linalg.cond(A)
    assert np.linalg.norm(x - x_exact) <= 50 * kappa ** 2 * EPS * max(1.0, np.linalg.norm(x_exact))


@pytest.mark.parametrize("shape", [(1, 1), (5, 5), (17, 9), (64, 33), (200, 64), (130, 130)])
def test_matches_lapack_dgeqrf(shape):
    """LAPACK dgeqrf uses the same reflector convention (beta = -sign(alpha)*norm,
    v_0 = 1), so R, the stored reflectors and tau must all agree."""
    m, n = shape
    A = I.random_matrix(m, n, seed=m * 1000 + n)
    F, tau = O.qr(A)
    h, tau_ref = np.linalg.qr(A, mode="raw")
    H = h.T  # column-major packed output of dgeqrf
    scale = np.linalg.norm(A)
    tol = 100 * max(m, n) * EPS
    assert np.allclose(tau, tau_ref, rtol=0, atol=tol * 10)
    assert np.abs(np.triu(F) - np.triu(H)).max() <= tol * scale
    assert np.abs(np.tril(F, -1) - np.tril(H, -1)).max() <= tol * 10 * max(1.0, np.abs(np.tril(H, -1)).max())


@pytest.mark.parametrize("shape", [(40, 40), (90, 37), (257, 64)])
def test_q_orthogonal_and_reconstructs_a(shape):
    m, n = shape
    A = I.random_matrix(m, n, seed=7 + m)
    F, tau = O.qr(A)
    Qt = O.apply_qt(F, tau, np.eye(m))
    assert np.linalg.norm(Qt @ Qt.T - np.eye(m)) <= 10 * m * EPS
    R = np.zeros((m, n))
    R[:n] = np.triu(F[:n])
    QR = O.apply_q(F, tau, R)
    assert np.linalg.norm(A - QR) / np.linalg.norm(A) <= 10 * m * n * EPS


def test_qt_a_is_upper_triangular_r():
    A = I.random_matrix(120, 50, seed=3)
    F, tau = O.qr(A)
    QtA = O.apply_qt(F, tau, A)
    assert np.abs(np.tril(QtA, -1)).max() <= 1e3 * EPS * np.linalg.norm(A)
    assert np.abs(np.triu(QtA[:50]) - np.triu(F[:50])).max() <= 1e3 * EPS * np.linalg.norm(A)


def test_orthogonal_invariance_of_norm():
    A = I.random_matrix(300, 80, seed=11)
    B = I.random_matrix(300, 4, seed=12)
    F, tau = O.qr(A)
    QtB = O.apply_qt(F, tau, B)
    assert np.allclose(np.linalg.norm(QtB, axis=0), np.linalg.norm(B, axis=0), rtol=1e-13)


def test_exact_recovery_on_ct_system():
    """Noiseless b = A x on the 32x32 parallel-beam system: x comes back to
    within a small multiple of kappa(A)*eps."""
    g = I.CONFIG1["geom"]
    A = O.system_matrix(O.Geometry(*g.as_tuple()))
    x = I.phantoms(g, [1, 2])
    b = A @ x
    xr = O.lstsq(A, b)
    kappa = np.linalg.cond(A)
    err = np.linalg.norm(xr - x) / np.linalg.norm(x)
    assert err <= 10 * kappa * EPS * np.sqrt(g.n)
    assert err < 1e-11


def test_least_squares_optimality_noisy():
    """For an inconsistent b the solution satisfies A^T (b - A x) = 0."""
    g = I.CONFIG1["geom"]
    A = O.system_matrix(O.Geometry(*g.as_tuple()))
    b = I.poisson_noise(A @ I.phantoms(g, [5]), g.fov, 1e4, seed=5)
    x = O.lstsq(A, b)
    r = b - A @ x
    ref = np.linalg.lstsq(A, b, rcond=None)[0]
    assert np.linalg.norm(A.T @ r) / (np.linalg.norm(A, 2) * np.linalg.norm(r)) <= 1e3 * EPS * np.linalg.cond(A)
    assert np.linalg.norm(x - ref) / np.linalg.norm(ref) < 1e-11


def test_backsolve_residual():
    rng = np.random.default_rng(4)
    n = 60
    F = np.asfortranarray(np.triu(rng.standard_normal((n, n))) + 5 * np.eye(n))
    Y = rng.standard_normal((n, 3))
    X = O.backsolve(F, Y)
    R = np.triu(F)
    assert np.linalg.norm(R @ X - Y) / (np.linalg.norm(R) * np.linalg.norm(X)) <= 10 * n * EPS
    assert np.allclose(X, np.linalg.solve(R, Y), rtol=1e-10)


def test_rank_deficient_detected():
    A = I.random_matrix(20, 6, seed=9)
    A[:, 3] = 0.0
    F, tau = O.qr(A)
    with pytest.raises(np.linalg.LinAlgError):
        O.backsolve(F, np.ones((20, 1)))
    A = I.random_matrix(20, 6, seed=9)
    A[:, 4] = A[:, 1]
    F, tau = O.qr(A)
    with pytest.raises(np.linalg.LinAlgError):
        O.backsolve(F, np.ones((20, 1)))


def test_column_already_reduced_gives_identity_reflector():
    """A column with zeros below the diagonal needs no reflection: tau = 0 and
    R keeps the entry as is (dgeqrf does the same)."""
    A = I.random_matrix(10, 4, seed=2)
    A[1:, 0] = 0.0
    A[0, 0] = -3.0
    F, tau = O.qr(A)
    h, tau_ref = np.linalg.qr(A, mode="raw")
    assert tau[0] == 0.0 and tau_ref[0] == 0.0
    assert F[0, 0] == -3.0
    assert np.allclose(np.triu(F), np.triu(h.T), atol=1e-13)
