"""The convolutional surrogate and its FP64 gate through the C ABI
(ct_surrogate_*), against the oracle model of oracle/surrogate.py.

Tolerances.  The library stores weights and activations in BF16 and
accumulates in FP32; the oracle rounds to BF16 at the same points and computes
in FP64 in between.  The two then differ only where an FP32 and an FP64 value
round to different BF16 neighbours (one BF16 ulp, 2^-8 relative, on a small
fraction of the elements) and by FP32 accumulation (about 1e-6 relative), so
network outputs and gradients are held to 2e-3 and 5e-3 relative (Frobenius)
and the loss to 1e-4.  The gate's residuals are FP64 on both sides (1e-10),
the slices it accepts are the network output bit for bit, and the slices it
sends back are the QR solution within 1e-10 of the oracle's.
"""
import dataclasses

import numpy as np
import pytest
import torch

from oracle import oracle as O
from oracle import surrogate as S
from paper_1907_01891_gb300 import ctqr
from paper_1907_01891_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def _np(t: torch.Tensor) -> np.ndarray:
    torch.cuda.synchronize()
    return t.detach().cpu().numpy()


def _og(g):
    return O.Geometry(*g.as_tuple())


def _he_params(seed: int, bias_scale: float = 0.1) -> np.ndarray:
    """Seeded parameters: weights U(-a, a), a = sqrt(6 / fan_in), biases
    bias_scale * N(0, 1)."""
    rng = np.random.default_rng(seed)
    parts = []
    for ci, co in S.layer_shapes():
        a = np.sqrt(6.0 / (9 * ci))
        parts.append(rng.uniform(-a, a, co * ci * 9))
        parts.append(bias_scale * rng.standard_normal(co))
    return np.concatenate(parts).astype(np.float32)


def _images(G: np.ndarray, geom) -> np.ndarray:
    """n x k column-major image matrix -> (k, ny, nx) (pixel iy * nx + ix)."""
    return np.ascontiguousarray(G.T).reshape(G.shape[1], geom.ny, geom.nx)


RAGGED = dataclasses.replace(I.parallel_geometry(40, 30, 59), ny=24)  # 2.5 x 1.5 tiles of 16


def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


# ----------------------------------------------------------- network parity
@pytest.mark.parametrize("k", [1, 3])
def test_forward_matches_oracle(k):
    geom = RAGGED
    s = ctqr.Surrogate(geom, in_scale=0.5, out_scale=2.0, seed=1)
    p = _he_params(11)
    s.set_params(p)
    G = np.random.default_rng(12).standard_normal((geom.n, k))
    X = _np(s.forward(ctqr.to_colmajor(G)))
    y, _ = S.forward(p.astype(np.float64), _images(G, geom), 0.5)
    ref = 2.0 * y[:, 0].reshape(k, -1).T
    assert X.shape == ref.shape
    assert _rel(X, ref) < 2e-3
    assert np.abs(X - ref).max() < 1e-2 * np.abs(ref).max()


def test_forward_chunks_large_batches():
    # more images than one network launch holds (256)
    geom = I.parallel_geometry(16, 8, 23)
    s = ctqr.Surrogate(geom, in_scale=1.0, out_scale=1.0)
    p = _he_params(13)
    s.set_params(p)
    k = 260
    G = np.random.default_rng(14).standard_normal((geom.n, k))
    X = _np(s.forward(ctqr.to_colmajor(G)))
    y, _ = S.forward(p.astype(np.float64), _images(G, geom), 1.0)
    ref = y[:, 0].reshape(k, -1).T
    assert _rel(X, ref) < 2e-3
    assert _rel(X[:, 256:], ref[:, 256:]) < 2e-3


def test_gradient_matches_oracle():
    geom = RAGGED
    s = ctqr.Surrogate(geom, in_scale=0.5, out_scale=2.0)
    p = _he_params(21)
    s.set_params(p)
    rng = np.random.default_rng(22)
    k = 2
    G = rng.standard_normal((geom.n, k))
    X = rng.standard_normal((geom.n, k))
    loss, grad = s.grad(ctqr.to_colmajor(G), ctqr.to_colmajor(X))
    lref, gref = S.loss_and_grad(p.astype(np.float64), _images(G, geom), _images(X, geom), 0.5, 2.0)
    assert abs(loss - lref) <= 1e-4 * lref
    off = 0
    for ci, co in S.layer_shapes():
        for n in (co * ci * 9, co):  # weights, then biases
            a, b = grad[off:off + n].astype(np.float64), gref[off:off + n]
            assert _rel(a, b) < 5e-3, (ci, co, n)
            off += n
    assert off == grad.size


def test_train_step_is_adam_on_the_gradient():
    geom = I.parallel_geometry(24, 10, 35)
    s = ctqr.Surrogate(geom, in_scale=1.0, out_scale=1.0)
    p = _he_params(31)
    s.set_params(p)
    rng = np.random.default_rng(32)
    G = rng.standard_normal((geom.n, 4))
    X = rng.standard_normal((geom.n, 4))
    lr = 1e-3
    loss0 = s.train_step(ctqr.to_colmajor(G), ctqr.to_colmajor(X), lr)
    p1 = s.get_params().astype(np.float64)
    lref, gref = S.loss_and_grad(p.astype(np.float64), _images(G, geom), _images(X, geom), 1.0, 1.0)
    pref, _, _ = S.adam_step(p.astype(np.float64), 0.0, 0.0, gref, 1, lr)
    assert abs(loss0 - lref) <= 1e-4 * lref
    # the first Adam step moves every parameter by about lr * sign(gradient):
    # the two sides agree wherever their gradients have the same sign
    same = np.sign(p1 - p) == np.sign(pref - p)
    assert same.mean() > 0.99
    assert np.abs((p1 - pref)[same]).max() < 1e-3 * lr + 1e-6


def test_training_reduces_the_loss():
    geom = I.parallel_geometry(16, 12, 23)
    s = ctqr.Surrogate(geom, in_scale=1.0, out_scale=1.0, seed=5)
    rng = np.random.default_rng(41)
    G = ctqr.to_colmajor(rng.standard_normal((geom.n, 32)))
    X = ctqr.to_colmajor(np.asarray(G.cpu()) * 0.5 + 0.25)  # an affine target the network can fit
    losses = [s.train_step(G, X, 3e-3) for _ in range(150)]
    assert losses[-1] < 0.1 * losses[0]
    assert np.all(np.isfinite(losses))


# ------------------------------------------------------------------- the gate
GATE_GEOM = I.CONFIG1["geom"]


@pytest.fixture(scope="module")
def gate_case():
    geom = GATE_GEOM
    A = O.system_matrix(_og(geom))
    half = np.full(geom.n, 0.5)
    x_ph = I.phantoms(geom, [7, 8])
    cols = [A @ half,                         # x_hat = 0.5 is exact: passes
            (1.0 + 1e-4) * (A @ half),        # residual 1e-4 / (1 + 1e-4): passes at 1e-3
            (1.0 + 1e-2) * (A @ half),        # residual ~1e-2: falls back
            A @ x_ph[:, 0],                   # a phantom: falls back
            np.zeros(geom.m),                 # b = 0: ||A x_hat|| > 0 falls back, QR gives 0
            A @ x_ph[:, 1]]
    B = np.asfortranarray(np.stack(cols, axis=1))
    res, ok = S.gate(A, np.tile(half[:, None], (1, B.shape[1])), B, 1e-3)
    return dict(geom=geom, A=A, B=B, res=res, ok=ok)


def _constant_network(geom, value: float, out_scale: float = 1.0) -> ctqr.Surrogate:
    """All weights zero and the output bias `value`: x_hat = value * out_scale."""
    s = ctqr.Surrogate(geom, in_scale=1.0, out_scale=out_scale)
    p = np.zeros(s.num_params(), dtype=np.float32)
    p[-1] = value
    s.set_params(p)
    return s


@pytest.mark.parametrize("prec", [ctqr.Prec.F64, ctqr.Prec.TF32])
def test_gate_keeps_passing_slices_and_solves_the_rest(gate_case, prec):
    geom, A, B = gate_case["geom"], gate_case["A"], gate_case["B"]
    s = _constant_network(geom, 0.5)
    Ad = ctqr.build_system(geom, torch.float64 if prec == ctqr.Prec.F64 else torch.float32)
    f = ctqr.qr_factor(Ad, prec)
    X, resid, rep = s.infer(ctqr.to_colmajor(B), tol=1e-3, factor=f)
    X, resid = _np(X), _np(resid)
    ok = gate_case["ok"]
    assert list(ok) == [True, True, False, False, False, False]
    assert np.allclose(resid, gate_case["res"], rtol=1e-10, atol=1e-13)
    assert rep["fallbacks"] == int((~ok).sum()) and rep["slices"] == B.shape[1]
    assert np.array_equal(X[:, ok], np.full((geom.n, ok.sum()), 0.5))
    ref = O.lstsq(A, B[:, ~ok])
    got = X[:, ~ok]
    for j in range(ref.shape[1]):
        scale = max(np.linalg.norm(ref[:, j]), 1.0)
        assert np.linalg.norm(got[:, j] - ref[:, j]) <= 1e-10 * scale
    assert rep["max_residual"] == pytest.approx(gate_case["res"][ok].max(), rel=1e-10, abs=1e-15)


def test_gate_without_factor_keeps_network_output(gate_case):
    geom, B = gate_case["geom"], gate_case["B"]
    s = _constant_network(geom, 0.5)
    X, resid, rep = s.infer(ctqr.to_colmajor(B), tol=1e-3, factor=None)
    assert np.array_equal(_np(X), np.full((geom.n, B.shape[1]), 0.5))
    assert rep["fallbacks"] == 4


def test_nonfinite_network_output_falls_back(gate_case):
    geom, A, B = gate_case["geom"], gate_case["A"], gate_case["B"]
    s = _constant_network(geom, float("nan"))
    f = ctqr.qr_factor(ctqr.build_system(geom, torch.float64))
    X, resid, rep = s.infer(ctqr.to_colmajor(B), tol=1e-3, factor=f)
    assert np.all(np.isnan(_np(resid)))
    assert rep["fallbacks"] == B.shape[1]
    ref = O.lstsq(A, B)
    X = _np(X)
    for j in range(B.shape[1]):
        assert np.linalg.norm(X[:, j] - ref[:, j]) <= 1e-10 * max(np.linalg.norm(ref[:, j]), 1.0)


def test_gate_with_lambda_stacked_factor(gate_case):
    geom, A, B = gate_case["geom"], gate_case["A"], gate_case["B"]
    lam = 1e-3
    s = _constant_network(geom, 0.5)
    f = ctqr.qr_factor(ctqr.build_system(geom, torch.float64, lam=lam))
    X, resid, rep = s.infer(ctqr.to_colmajor(B), tol=1e-3, factor=f, lam=lam)
    ok = gate_case["ok"]
    As = np.vstack([A, lam * np.eye(geom.n)])
    Bs = np.vstack([B, np.zeros((geom.n, B.shape[1]))])
    ref = O.lstsq(As, Bs[:, ~ok])
    got = _np(X)[:, ~ok]
    for j in range(ref.shape[1]):
        assert np.linalg.norm(got[:, j] - ref[:, j]) <= 1e-10 * max(np.linalg.norm(ref[:, j]), 1.0)


def test_gate_chunks_and_strided_output():
    # 300 slices (two gate chunks), alternately passing and failing, written
    # into an X with padding rows
    geom = GATE_GEOM
    A = O.system_matrix(_og(geom))
    half = np.full(geom.n, 0.5)
    ph = I.phantoms(geom, range(300, 450))
    B = np.empty((geom.m, 300), order="F")
    B[:, 0::2] = (A @ half)[:, None]
    B[:, 1::2] = A @ ph
    s = _constant_network(geom, 0.5)
    f = ctqr.qr_factor(ctqr.build_system(geom, torch.float64))
    Xd = ctqr.colmajor(geom.n, 300, ld=geom.n + 6, fill=-7.0)
    X, resid, rep = s.infer(ctqr.to_colmajor(B), tol=1e-3, factor=f, X=Xd)
    X = _np(X)
    assert rep["fallbacks"] == 150
    assert np.array_equal(X[:, 0::2], np.full((geom.n, 150), 0.5))
    ref = O.lstsq(A, B[:, 1::2])
    assert np.linalg.norm(X[:, 1::2] - ref) <= 1e-10 * np.linalg.norm(ref)
    full = _np(Xd.as_strided((geom.n + 6, 300), (1, geom.n + 6)))
    assert np.all(full[geom.n:] == -7.0)  # padding rows untouched


def test_project_and_backproject_match_oracle():
    geom = I.fan_geometry(24, 30, 37)
    A = O.system_matrix(_og(geom))
    s = ctqr.Surrogate(geom)
    X = I.phantoms(geom, [1, 2, 3])
    B = _np(s.project(ctqr.to_colmajor(X)))
    assert np.abs(B - A @ X).max() <= 1e-12 * np.abs(A @ X).max()
    R = np.random.default_rng(3).standard_normal((geom.m, 3))
    G = _np(s.backproject(ctqr.to_colmajor(R)))
    assert np.abs(G - A.T @ R).max() <= 1e-12 * np.abs(A.T @ R).max()


def test_invalid_arguments():
    geom = GATE_GEOM
    s = ctqr.Surrogate(geom)
    B = ctqr.colmajor(geom.m, 2, fill=0.0)
    f_other = ctqr.qr_factor(ctqr.build_system(I.parallel_geometry(16, 12, 23), torch.float64))
    with pytest.raises(ctqr.CtError):
        s.infer(B, tol=1e-3, factor=f_other)  # factor of another geometry
    with pytest.raises(ctqr.CtError):
        s.infer(B, tol=-1.0)
    with pytest.raises(ctqr.CtError):
        ctqr.Surrogate(geom, in_scale=0.0)


# --------------------------------------------------------------------- gain
def test_trained_surrogate_gain_report():
    """Train on QR reconstructions of noiseless scans of the 32 x 32 parallel
    geometry and report what the gate accepts, the error against the QR
    solution, and slices/s with and without the network."""
    import time
    geom = GATE_GEOM
    s0 = ctqr.Surrogate(geom)
    Ad = ctqr.build_system(geom, torch.float64)
    f = ctqr.qr_factor(Ad)
    ntrain, batch = 4096, 64
    Xtr = ctqr.to_colmajor(I.phantoms(geom, range(10_000, 10_000 + ntrain)))
    Btr = s0.project(Xtr)
    Qtr, _ = ctqr.reconstruct(f, Btr)  # the method's reconstructions are the targets
    Gtr = s0.backproject(Btr)
    in_scale = 1.0 / float(Gtr.abs().mean())
    s = ctqr.Surrogate(geom, in_scale=in_scale, out_scale=1.0, seed=3)
    first = last = None
    for it in range(600):
        j = (it * batch) % ntrain
        l = s.train_step(Gtr[:, j:j + batch], Qtr[:, j:j + batch], 1e-3 if it < 400 else 3e-4)
        first = l if first is None else first
        last = l
    assert last < 0.2 * first

    k = 256
    Xte = ctqr.to_colmajor(I.phantoms(geom, range(50_000, 50_000 + k)))
    Bte = s0.project(Xte)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    Xq, _ = ctqr.reconstruct(f, Bte)
    torch.cuda.synchronize()
    t_qr = time.perf_counter() - t0
    Xn = s.forward(s.backproject(Bte))
    t0 = time.perf_counter()
    Xg, resid, rep = s.infer(Bte, tol=1e-3, factor=f)
    torch.cuda.synchronize()
    t_sur = time.perf_counter() - t0
    Xq, Xn, Xg, resid = _np(Xq), _np(Xn), _np(Xg), _np(resid)
    err_net = np.linalg.norm(Xn - Xq, axis=0) / np.linalg.norm(Xq, axis=0)
    err_gated = np.linalg.norm(Xg - Xq, axis=0) / np.linalg.norm(Xq, axis=0)
    passed = resid <= 1e-3
    print(f"\nsurrogate gain (32x32, {ntrain} training pairs, {k} test slices): "
          f"loss {first:.3e} -> {last:.3e}; network error vs QR median {np.median(err_net):.3e}; "
          f"gate residual median {np.median(resid):.3e}; fallback {rep['fallbacks']}/{k}; "
          f"gated error vs QR max {err_gated.max():.3e}; "
          f"QR {k / t_qr:.1f} slices/s, gated surrogate {k / t_sur:.1f} slices/s")
    assert rep["fallbacks"] == int((~passed).sum())
    assert np.all(err_gated[~passed] <= 1e-10)
    assert np.all(np.median(err_net) < 1.0)
