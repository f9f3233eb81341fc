"""Parity on the full multi-slice and batched workloads (paper Eq. (qr1):
one factor, many right-hand sides; Tables tasks_qr_ab / tasks_solve_ab: many
systems in one launch), against the oracle.

* 512 Poisson-noisy sinograms (I0 = 1e4) of the 32 x 32 parallel-beam system
  (2700 x 1024) through one factor in one multi-RHS call, FP64 factor and the
  3xTF32 factor refined with FP64 residuals: every column of X against the
  oracle's least-squares solution to the 1e-10 target.
* The largest system of the 64-system uneven batch (96^2 image, [A; 1e-3 I],
  26752 x 9216) in one persistent launch beside the smallest: its oracle
  solution takes minutes on the host cores, so it is checked by a property
  that holds at any size -- the FP64 normal equations of the oracle's own
  system matrix, ||A^T (b - A x) - lam^2 x|| / (||A||_F^2 ||x||) at
  rounding level -- and against the independent single-system FP64 path
  (whose solutions match the oracle at smaller sizes); the smallest system is
  compared with the oracle element by element.
"""
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


def _err(X, Xo):
    return (np.linalg.norm(X - Xo) / np.linalg.norm(Xo), np.abs(X - Xo).max() / np.abs(Xo).max())


@pytest.fixture(scope="module")
def config4a():
    g = I.CONFIG4A["geom"]
    Ao = O.system_matrix(O.Geometry(*g.as_tuple()))
    seeds = I.CONFIG4A["seeds"]
    assert len(seeds) == 512
    b = I.poisson_noise(Ao @ I.phantoms(g, seeds), g.fov, I.CONFIG4A["noise_i0"], seed=seeds[0])
    Xo = O.lstsq(Ao, b)
    return g, Ao, b, Xo


@pytest.mark.parametrize("prec", [ctqr.Prec.F64, ctqr.Prec.TF32], ids=["f64", "tf32_refined"])
def test_config4a_512_noisy_slices_in_one_call_match_oracle(config4a, prec):
    g, Ao, b, Xo = config4a
    A = ctqr.build_system(g, torch.float64)
    f = ctqr.qr_factor(A if prec == ctqr.Prec.F64 else A.to(torch.float32), prec=prec)
    X, rep = ctqr.reconstruct(f, ctqr.to_colmajor(b), A=None if prec == ctqr.Prec.F64 else A)
    Xg = _np(X)
    fro, elem = _err(Xg, Xo)
    assert fro <= 1e-10 and elem <= 1e-10, (fro, elem)
    # each column is its own least-squares problem: the worst column too
    col = (np.linalg.norm(Xg - Xo, axis=0) / np.linalg.norm(Xo, axis=0)).max()
    assert col <= 1e-10, col


def test_largest_uneven_batch_system_solves_its_normal_equations():
    cfg = I.CONFIG4B
    geoms = I.uneven_systems(cfg["count"], cfg["seed"])
    order = sorted(range(len(geoms)), key=lambda q: geoms[q].m * geoms[q].n)
    small, big = order[0], order[-1]
    lam = cfg["lam"]
    assert geoms[big].nx == 96
    As, Bs, ref = [], [], []
    for q in (small, big):
        g = geoms[q]
        Ao = O.system_matrix(O.Geometry(*g.as_tuple()))
        b = np.vstack([Ao @ I.phantoms(g, [cfg["seed0"] + q]), np.zeros((g.n, 1))])
        As.append(ctqr.build_system(g, torch.float64, lam=lam))
        Bs.append(ctqr.to_colmajor(b))
        ref.append((Ao, b, g))
    st, rep = ctqr.qr_solve_batched(As, Bs, tile=0)
    assert st == ctqr.CT_OK
    torch.cuda.synchronize()
    # smallest: the oracle's least-squares solution
    Ao, b, g = ref[0]
    Xs = Bs[0].cpu().numpy()[:g.n]
    Xo = O.lstsq(np.vstack([Ao, lam * np.eye(g.n)]), b)
    fro, elem = _err(Xs, Xo)
    assert fro <= 1e-10 and elem <= 1e-10, (fro, elem)
    # largest: FP64 normal equations of the oracle's matrix
    Ao, b, g = ref[1]
    x = Bs[1].cpu().numpy()[:g.n]
    r = b[:g.m] - Ao @ x
    gres = Ao.T @ r - lam * lam * x
    ne = np.linalg.norm(gres) / (np.linalg.norm(Ao) ** 2 * np.linalg.norm(x))
    assert ne <= 1e-15, ne
    # and the single-system FP64 path on the same system
    Asys = ctqr.build_system(g, torch.float64, lam=lam)
    f = ctqr.qr_factor(Asys)
    X1, _ = ctqr.reconstruct(f, ctqr.to_colmajor(b))
    fro, elem = _err(x, _np(X1))
    assert fro <= 1e-10 and elem <= 1e-10, (fro, elem)
