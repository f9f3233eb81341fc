"""Joseph's projector (ct_project_joseph, the paper's sinogram simulator,
Sec. III) and the image-quality measures (ct_image_quality: Eq. MSE, psnr,
ssim) against the oracle.  Both sides compute the same FP64 expressions
(up to fused multiply-adds), so the sinograms must agree to 1e-12 relative to
their largest entry, the measures to 1e-10 relative.  The last test
reconstructs Joseph sinograms with the Siddon system matrix: the model
mismatch of a real scan, which the paper's PSNR / SSIM tables measure."""
import math

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


@pytest.mark.parametrize("geom", [I.parallel_geometry(24, 30, 35), I.fan_geometry(32, 40, 47),
                                  I.scanner_geometry(20, 28, 31),
                                  I.ScanGeometry(0, 9, 7, 0.8, 4, 13, 0.0, math.pi, 0.0, 9.0)],
                         ids=["parallel24", "fan32", "scanner20", "axis_views_nonsquare"])
def test_joseph_matches_oracle(geom):
    X = I.phantoms(geom, [5, 6, 7]) if geom.nx == geom.ny else np.random.default_rng(1).uniform(0, 1, (geom.n, 3))
    B = ctqr.project_joseph(geom, ctqr.to_colmajor(X))
    Bo = O.joseph_project(O.Geometry(*geom.as_tuple()), X)
    assert np.abs(_np(B) - Bo).max() <= 1e-12 * max(1.0, np.abs(Bo).max())


def test_image_quality_matches_oracle():
    g = I.fan_geometry(40, 8, 9)
    ref = I.phantoms(g, [11, 12, 13])
    rng = np.random.default_rng(3)
    X = ref + 0.02 * rng.standard_normal(ref.shape)
    X[:, 2] = ref[:, 2]                   # identical slice: MSE 0, SSIM 1
    q = _np(ctqr.image_quality(ctqr.to_colmajor(X), ctqr.to_colmajor(ref), 40, 40))
    for c in range(3):
        mse, psnr, ssim = O.quality(X[:, c], ref[:, c], 40, 40)
        assert q[c, 0] == pytest.approx(mse, rel=1e-10, abs=1e-300)
        if math.isinf(psnr):
            assert math.isinf(q[c, 1])
        else:
            assert q[c, 1] == pytest.approx(psnr, rel=1e-10)
        assert q[c, 2] == pytest.approx(ssim, rel=1e-10)
    assert q[2, 2] == pytest.approx(1.0, abs=1e-12)


def test_joseph_sinograms_reconstructed_with_the_siddon_matrix():
    """The paper's data path: sinograms from Joseph's projector, reconstruction
    with the system matrix (here Siddon's).  The least-squares solution is the
    oracle's to 1e-10 (it is a well-defined problem whatever produced b); its
    PSNR against the phantom is finite and far below the ~200 dB of a
    consistent b = A x, which is the model mismatch."""
    g = I.CONFIG1["geom"]
    x = I.phantoms(g, [21, 22])
    B = ctqr.project_joseph(g, ctqr.to_colmajor(x))
    A = ctqr.build_system(g, torch.float64)
    f = ctqr.qr_factor(A)
    X, _ = ctqr.reconstruct(f, B)
    Ao = O.system_matrix(O.Geometry(*g.as_tuple()))
    Xo = O.lstsq(Ao, O.joseph_project(O.Geometry(*g.as_tuple()), x))
    assert np.linalg.norm(_np(X) - Xo) / np.linalg.norm(Xo) <= 1e-10
    q = _np(ctqr.image_quality(X, ctqr.to_colmajor(x), g.nx, g.ny))
    assert np.all(np.isfinite(q[:, 1])) and np.all(q[:, 1] < 100.0)
    Xc, _ = ctqr.reconstruct(f, ctqr.to_colmajor(Ao @ x))       # consistent data
    qc = _np(ctqr.image_quality(Xc, ctqr.to_colmajor(x), g.nx, g.ny))
    assert np.all(qc[:, 1] > 180.0) and np.all(qc[:, 2] > 0.999999)
