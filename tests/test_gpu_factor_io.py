"""A factor written to a file and read back (ct_factor_save / ct_factor_load),
then used: the paper computes the factorization once and keeps it for every
later batch of slices (Sec. II-B).  The loaded factor must be bitwise the
saved one (same F, tau) and must reconstruct against the oracle within the
1e-10 relative bound of the other reconstruction tests; a damaged file must be
refused."""
import os

import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_1907_01891_gb300 import ctqr
from paper_1907_01891_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def _np(t):
    torch.cuda.synchronize()
    return t.detach().cpu().numpy()


def test_fp64_factor_round_trip_reconstructs_against_oracle(tmp_path):
    g = I.CONFIG1["geom"]
    A = ctqr.build_system(g, torch.float64)
    f = ctqr.qr_factor(A)
    tag = ctqr.geometry_hash(g)
    path = str(tmp_path / "fan.ctqr")
    ctqr.factor_save(f, path, tag)
    info = ctqr.factor_file_info(path)
    assert info == dict(m=g.m, n=g.n, nb=f.info()["nb"], prec=ctqr.Prec.F64, tag=tag)
    f2, tag2 = ctqr.factor_load(path)
    assert tag2 == tag and f2.info() == f.info()
    F1, t1 = ctqr.factor_matrix(f)
    F2, t2 = ctqr.factor_matrix(f2)
    assert torch.equal(F1, F2) and torch.equal(t1, t2)
    Ao = O.system_matrix(O.Geometry(*g.as_tuple()))
    x = I.phantoms(g, [1, 2, 3])
    b = Ao @ x
    X, _ = ctqr.reconstruct(f2, ctqr.to_colmajor(b))
    xo = O.lstsq(Ao, b)
    assert np.linalg.norm(_np(X) - xo) / np.linalg.norm(xo) <= 1e-10


def test_mixed_factor_round_trip_refines_to_oracle(tmp_path):
    g = I.fan_geometry(40, 64, 59)
    lam = 1e-3
    A32 = ctqr.build_system(g, torch.float32, lam=lam)
    f = ctqr.qr_factor(A32, ctqr.Prec.TF32)
    path = str(tmp_path / "mixed.ctqr")
    ctqr.factor_save(f, path, ctqr.geometry_hash(g, lam))
    f2, tag = ctqr.factor_load(path)
    assert tag == ctqr.geometry_hash(g, lam)
    assert f2.info()["prec"] == ctqr.Prec.TF32
    F1, t1 = ctqr.factor_matrix(f)
    F2, t2 = ctqr.factor_matrix(f2)
    assert torch.equal(F1, F2) and torch.equal(t1, t2)
    Ao = O.system_matrix(O.Geometry(*g.as_tuple()))
    x = I.phantoms(g, [7, 8])
    b = Ao @ x
    Asys = np.vstack([Ao, lam * np.eye(g.n)])
    bsys = np.vstack([b, np.zeros((g.n, 2))])
    A64 = ctqr.to_colmajor(Ao)
    # the same refinement through the original and through the loaded factor
    X1, r1 = ctqr.reconstruct(f, ctqr.to_colmajor(bsys), A=A64, lam=lam)
    X2, r2 = ctqr.reconstruct(f2, ctqr.to_colmajor(bsys), A=A64, lam=lam)
    assert torch.equal(X1, X2) and r1.iterations == r2.iterations
    xo = O.lstsq(Asys, bsys)
    assert np.linalg.norm(_np(X2) - xo) / np.linalg.norm(xo) <= 1e-10


def test_damaged_factor_file_is_refused(tmp_path):
    A = ctqr.to_colmajor(I.random_matrix(300, 100, seed=3))
    f = ctqr.qr_factor(A)
    path = str(tmp_path / "f.ctqr")
    ctqr.factor_save(f, path)
    raw = bytearray(open(path, "rb").read())
    bad = tmp_path / "flipped.ctqr"
    raw2 = bytearray(raw)
    raw2[128 + 8 * 1234 + 3] ^= 0x10  # one payload bit
    bad.write_bytes(bytes(raw2))
    with pytest.raises(ctqr.CtError) as e:
        ctqr.factor_load(str(bad))
    assert e.value.status == ctqr.CT_ERR_INVALID
    short = tmp_path / "short.ctqr"
    short.write_bytes(bytes(raw[:-8]))
    with pytest.raises(ctqr.CtError) as e:
        ctqr.factor_load(str(short))
    assert e.value.status == ctqr.CT_ERR_INVALID
    # the intact file still loads
    f2, _ = ctqr.factor_load(path)
    assert torch.equal(ctqr.factor_matrix(f2)[0], ctqr.factor_matrix(f)[0])
    os.remove(path)
