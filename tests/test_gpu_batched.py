"""Batched factor + solve of uneven systems (ct_qr_solve_batched): the paper's
algorithm-by-blocks (tile QR and the tile solve) in one persistent launch,
against the oracle.  x is unique under full rank and must match the oracle's
least-squares solution to 1e-10 relative; R is unique up to the sign of each
row, so |R| is compared (1e-10 relative to max |R|)."""
import json
import os

import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_1907_01891_gb300 import ctqr
from paper_1907_01891_gb300 import inputs as I

pytestmark = pytest.mark.gpu

SHAPES = [(130, 70, 2), (300, 200, 1), (97, 97, 3), (520, 333, 5), (64, 64, 1), (1000, 257, 17), (65, 33, 0)]


@pytest.mark.parametrize("tile", [32, 64])
def test_batched_uneven_random_systems_match_oracle(tile):
    As, Bs, ref = [], [], []
    for q, (m, n, k) in enumerate(SHAPES):
        A = I.random_matrix(m, n, seed=300 + q)
        B = I.random_matrix(m, k, seed=400 + q) if k else None
        As.append(ctqr.to_colmajor(A))
        Bs.append(ctqr.to_colmajor(B) if k else None)
        ref.append((A, B))
    st, rep = ctqr.qr_solve_batched(As, Bs, tile=tile)
    assert rep.tile == tile and rep.tasks > 0
    torch.cuda.synchronize()
    for (A, B), At, Bt, (m, n, k) in zip(ref, As, Bs, SHAPES):
        Fo, tau = O.qr(A)
        R, Ro = np.triu(At.cpu().numpy()[:n]), np.triu(Fo[:n])
        assert np.abs(np.abs(R) - np.abs(Ro)).max() <= 1e-10 * np.abs(Ro).max(), (m, n)
        if k:
            X = Bt.cpu().numpy()[:n]
            Xo = O.lstsq(A, B)
            assert np.linalg.norm(X - Xo) / np.linalg.norm(Xo) <= 1e-10, (m, n)


def test_batched_lambda_stacked_ct_systems_match_oracle():
    """Config-4b style: [A_s; 1e-3 I] for uneven fan/parallel geometries."""
    lam = 1e-3
    geoms = [I.parallel_geometry(16, 18, 23), I.fan_geometry(20, 24, 29), I.parallel_geometry(12, 11, 17),
             I.fan_geometry(24, 30, 35)]
    As, Bs, ref = [], [], []
    for q, g in enumerate(geoms):
        A = ctqr.build_system(g, torch.float64, lam=lam)
        Ao = O.system_matrix(O.Geometry(*g.as_tuple()))
        Asys = np.vstack([Ao, lam * np.eye(g.n)])
        b = np.vstack([Ao @ I.phantoms(g, [q + 1, q + 2]), np.zeros((g.n, 2))])
        As.append(A)
        Bs.append(ctqr.to_colmajor(b))
        ref.append((Asys, b))
    ctqr.qr_solve_batched(As, Bs, tile=32)
    torch.cuda.synchronize()
    for (Asys, b), Bt, g in zip(ref, Bs, geoms):
        X = Bt.cpu().numpy()[:g.n]
        Xo = O.lstsq(Asys, b)
        assert np.linalg.norm(X - Xo) / np.linalg.norm(Xo) <= 1e-10


def test_batched_autotune_caches_its_choice(tmp_path, monkeypatch):
    cache = tmp_path / "tune.json"
    monkeypatch.setenv("CTQR_TUNE_CACHE", str(cache))
    As = [ctqr.to_colmajor(I.random_matrix(400, 150, seed=9)), ctqr.to_colmajor(I.random_matrix(380, 140, seed=10))]
    Bs = [ctqr.to_colmajor(I.random_matrix(400, 2, seed=11)), ctqr.to_colmajor(I.random_matrix(380, 2, seed=12))]
    st, rep = ctqr.qr_solve_batched(As, Bs, tile=0)
    assert rep.tile in (32, 64)
    data = json.loads(cache.read_text())
    assert any(k.startswith("tile_qr/") and v == rep.tile for k, v in data.items())


def test_batched_reports_rank_deficiency():
    A = I.random_matrix(90, 40, seed=3)
    A[:, 17] = 0.0
    st, rep = ctqr.qr_solve_batched([ctqr.to_colmajor(A)], [ctqr.to_colmajor(np.ones((90, 1)))], tile=32,
                                    check=False)
    assert st == ctqr.CT_ERR_RANK


def test_uneven_lambda_stacked_batch_smallest_systems_match_oracle():
    """The four smallest systems of the 64-system uneven batch (fan beam,
    images 32^2-96^2, [A; 1e-3 I]) in one launch with the tuned tile, against
    the oracle's least-squares solution."""
    cfg = I.CONFIG4B
    geoms = I.uneven_systems(cfg["count"], cfg["seed"])
    idx = sorted(range(len(geoms)), key=lambda q: geoms[q].m * geoms[q].n)[:4]
    lam = cfg["lam"]
    As, Bs, ref = [], [], []
    for q in idx:
        g = geoms[q]
        Ao = O.system_matrix(O.Geometry(*g.as_tuple()))
        b = np.vstack([Ao @ I.phantoms(g, [cfg["seed0"] + q]), np.zeros((g.n, 1))])
        As.append(ctqr.build_system(g, torch.float64, lam=lam))
        Bs.append(ctqr.to_colmajor(b))
        ref.append((np.vstack([Ao, lam * np.eye(g.n)]), b, g))
    st, rep = ctqr.qr_solve_batched(As, Bs, tile=0)
    torch.cuda.synchronize()
    for (Asys, b, g), Bt in zip(ref, Bs):
        X = Bt.cpu().numpy()[:g.n]
        Xo = O.lstsq(Asys, b)
        assert np.linalg.norm(X - Xo) / np.linalg.norm(Xo) <= 1e-10, (g.nx, g.m)


def test_batched_stalled_task_times_out_and_context_survives(monkeypatch):
    """A task whose dependency never arrives (host-side injection) makes the
    persistent launch give up after the bounded wait with CT_ERR_TIMEOUT; the
    next call on the same context succeeds."""
    A = I.random_matrix(300, 120, seed=21)
    B = I.random_matrix(300, 2, seed=22)
    monkeypatch.setenv("CTQR_WAIT_LIMIT_MS", "200")
    monkeypatch.setenv("CTQR_FAULT_STALL_TASK", "7")
    st, _ = ctqr.qr_solve_batched([ctqr.to_colmajor(A)], [ctqr.to_colmajor(B)], tile=32, check=False)
    assert st == ctqr.CT_ERR_TIMEOUT
    monkeypatch.delenv("CTQR_FAULT_STALL_TASK")
    At, Bt = ctqr.to_colmajor(A), ctqr.to_colmajor(B)
    st, _ = ctqr.qr_solve_batched([At], [Bt], tile=32)
    assert st == ctqr.CT_OK
    torch.cuda.synchronize()
    X = Bt.cpu().numpy()[:120]
    Xo = O.lstsq(A, B)
    assert np.linalg.norm(X - Xo) / np.linalg.norm(Xo) <= 1e-10


def test_mixed_precision_batch_matches_oracle_and_keeps_A():
    """ct_qr_solve_batched with CT_PREC_TF32: every system through the
    tensor-core factorization and FP64 refinement against its own FP64 A
    (left unchanged): the four smallest systems of the uneven 64-system batch
    and two random ones, against the oracle's least-squares solutions."""
    cfg = I.CONFIG4B
    geoms = I.uneven_systems(cfg["count"], cfg["seed"])
    idx = sorted(range(len(geoms)), key=lambda q: geoms[q].m * geoms[q].n)[:4]
    lam = cfg["lam"]
    As, Bs, ref = [], [], []
    for q in idx:
        g = geoms[q]
        Ao = O.system_matrix(O.Geometry(*g.as_tuple()))
        b = np.vstack([Ao @ I.phantoms(g, [cfg["seed0"] + q]), np.zeros((g.n, 1))])
        As.append(ctqr.build_system(g, torch.float64, lam=lam))
        Bs.append(ctqr.to_colmajor(b))
        ref.append((np.vstack([Ao, lam * np.eye(g.n)]), b, g.n))
    for q, (m, n, k) in enumerate([(700, 300, 3), (1300, 650, 2)]):
        A = I.random_matrix(m, n, seed=600 + q)
        B = I.random_matrix(m, k, seed=610 + q)
        As.append(ctqr.to_colmajor(A))
        Bs.append(ctqr.to_colmajor(B))
        ref.append((A, B, n))
    before = [A.clone() for A in As]
    st, rep = ctqr.qr_solve_batched(As, Bs, prec=ctqr.Prec.TF32)
    assert st == ctqr.CT_OK and rep.tasks == 0 and rep.iterations >= 1
    torch.cuda.synchronize()
    for (Asys, b, n), Bt, A0, A1 in zip(ref, Bs, before, As):
        assert torch.equal(A0, A1)
        X = Bt.cpu().numpy()[:n]
        Xo = O.lstsq(Asys, b)
        assert np.linalg.norm(X - Xo) / np.linalg.norm(Xo) <= 1e-10, n

@pytest.mark.slow
def test_largest_uneven_batch_system_solves_its_normal_equations():
    """The largest system of the 64-system uneven batch (96^2 image, [A; 1e-3 I],
    26752 x 9216) in one persistent launch beside the smallest.  Its oracle
    solution takes minutes on the host cores, so it is held to a property
    that holds at any size -- the FP64 normal equations of the oracle's own
    system matrix, ||A^T (b - A x) - lam^2 x|| / (||A||_F^2 ||x||), at the
    level of a backward-stable QR's backward error (20 sqrt(n) u = 2e-13 for
    n = 9216; the tile runtime gives ~5e-14) -- and to the single-system FP64
    path (whose
    solutions match the oracle at smaller sizes); the smallest system is
    compared with the oracle element by element."""
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
    fro, elem = _rel_err(Xs, Xo)
    assert fro <= 1e-10 and elem <= 1e-10, (fro, elem)
    # largest: FP64 normal equations of the oracle's matrix
    Ao, b, g = ref[1]
    x = Bs[1].cpu().numpy()[:g.n]
    r = b[:g.m] - Ao @ x
    gres = Ao.T @ r - lam * lam * x
    ne = np.linalg.norm(gres) / (np.linalg.norm(Ao) ** 2 * np.linalg.norm(x))
    assert ne <= 2e-13, ne
    # and the single-system FP64 path on the same system
    Asys = ctqr.build_system(g, torch.float64, lam=lam)
    f = ctqr.qr_factor(Asys)
    X1, _ = ctqr.reconstruct(f, ctqr.to_colmajor(b))
    torch.cuda.synchronize()
    fro, elem = _rel_err(x, X1.cpu().numpy())
    assert fro <= 1e-10 and elem <= 1e-10, (fro, elem)


def _rel_err(X, Xo):
    return (np.linalg.norm(X - Xo) / np.linalg.norm(Xo), np.abs(X - Xo).max() / np.abs(Xo).max())


@pytest.mark.parametrize("pos", [4, 12])
def test_tile32_factor_of_ct_systems_with_noise_level_columns_matches_oracle(pos):
    """Two systems of the uneven batch (38^2 and 45^2 images, [A; 1e-3 I]) whose
    32-wide tile factorization meets columns that are rounding remainders of
    exact zeros, down to magnitudes where their sums of squares underflow:
    R and the solution against the oracle (R up to row signs, relative to
    max |R|, 1e-11; x 1e-10).  Built from such columns, the triangle-on-square
    reflectors were not orthogonal and lost up to 2.6e-2 of R."""
    cfg = I.CONFIG4B
    geoms = I.uneven_systems(cfg["count"], cfg["seed"])
    order = sorted(range(len(geoms)), key=lambda q: geoms[q].m * geoms[q].n)
    q = order[pos]
    g = geoms[q]
    lam = cfg["lam"]
    Ao = O.system_matrix(O.Geometry(*g.as_tuple()))
    As = np.vstack([Ao, lam * np.eye(g.n)])
    b = np.vstack([Ao @ I.phantoms(g, [cfg["seed0"] + q]), np.zeros((g.n, 1))])
    Fo, _ = O.qr(As)
    Ro = np.triu(Fo[:g.n])
    Xo = O.lstsq(As, b)
    At, Bt = ctqr.to_colmajor(As), ctqr.to_colmajor(b)
    st, _ = ctqr.qr_solve_batched([At], [Bt], tile=32)
    assert st == ctqr.CT_OK
    torch.cuda.synchronize()
    R = np.triu(At.cpu().numpy()[:g.n])
    sg = np.sign(np.diag(R)) * np.sign(np.diag(Ro))
    assert np.abs(R * sg[:, None] - Ro).max() <= 1e-11 * np.abs(Ro).max()
    fro, elem = _rel_err(Bt.cpu().numpy()[:g.n], Xo)
    assert fro <= 1e-10 and elem <= 1e-10, (fro, elem)


def test_repeat_calls_replay_the_kept_plan_with_new_buffers():
    """Calls with the same sizes reuse the task list and graph kept on the
    device: each call's systems sit in fresh buffers (new pointers) with new
    data, and every result matches the oracle; a call with other sizes, a call
    after ct_qr_solve_batched_release and an uncached call do too."""
    shapes = [(300, 120, 2), (520, 333, 1), (97, 97, 3)]

    def run(seed, shp, **kw):
        As, Bs, ref = [], [], []
        for q, (m, n, k) in enumerate(shp):
            A = I.random_matrix(m, n, seed=seed + q)
            B = I.random_matrix(m, k, seed=seed + 50 + q)
            As.append(ctqr.to_colmajor(A))
            Bs.append(ctqr.to_colmajor(B))
            ref.append((A, B))
        st, rep = ctqr.qr_solve_batched(As, Bs, tile=32, **kw)
        assert st == ctqr.CT_OK
        torch.cuda.synchronize()
        for (A, B), Bt, (m, n, k) in zip(ref, Bs, shp):
            X = Bt.cpu().numpy()[:n]
            Xo = O.lstsq(A, B)
            assert np.linalg.norm(X - Xo) / np.linalg.norm(Xo) <= 1e-10, (seed, m, n)
        return rep.tasks

    t0 = run(1000, shapes)
    assert run(2000, shapes) == t0 and run(3000, shapes) == t0
    run(4000, shapes[:2])
    ctqr.qr_solve_batched_release()
    assert run(5000, shapes) == t0
    assert run(6000, shapes, cache=False) == t0
    ctqr.qr_solve_batched_release()
    ctqr.qr_solve_batched_release()
