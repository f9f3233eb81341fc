"""The batched runtime's task list (ct_batch_plan, host logic only, no GPU).

For uneven systems, the list must hold exactly the tile tasks of the paper's
algorithm-by-blocks (Table tasks_qr_ab: one GEQRT per diagonal tile, an UNMQR
for every tile right of it, a TSQRT for every tile below it, a TSMQR for every
tile below and right; Table tasks_solve_ab: the two Apply tasks on every tile
of B, one Trsm_lunn per block row and a Gemm_nn_mo per tile above the
diagonal of R, per block column of B), and its order must let the persistent
launch run: taking the tasks one after another in list order, every
dependency is already met when a task is taken, and met exactly (a reader sees
precisely the writes planned before it, a writer precisely the reads and
writes planned before it), so the reordering by earliest start kept the
planned versions.  The launch only ever waits on tasks taken before, which is
why it cannot deadlock."""
import numpy as np
import pytest

from paper_1907_01891_gb300 import ctqr

SHAPES = [(130, 70, 2), (300, 200, 1), (97, 97, 3), (520, 333, 5), (64, 64, 1), (1000, 257, 17), (65, 33, 0)]
NAMES = ["GEQRT", "UNMQR", "TSQRT", "TSMQR", "B_UNMQR", "B_TSMQR", "TRSM", "GEMM"]


def _expected_counts(shapes, b):
    cnt = dict.fromkeys(NAMES, 0)
    for m, n, k in shapes:
        mt, nt, kt = -(-m // b), -(-n // b), -(-k // b)
        for q in range(min(mt, nt)):
            cnt["GEQRT"] += 1
            cnt["UNMQR"] += nt - q - 1
            cnt["TSQRT"] += mt - q - 1
            cnt["TSMQR"] += (mt - q - 1) * (nt - q - 1)
            cnt["B_UNMQR"] += kt
            cnt["B_TSMQR"] += kt * (mt - q - 1)
        cnt["TRSM"] += kt * nt
        cnt["GEMM"] += kt * nt * (nt - 1) // 2
    return cnt


@pytest.mark.parametrize("tile", [32, 64])
@pytest.mark.parametrize("shapes", [SHAPES, [(2387, 1024, 1), (900, 400, 64), (40, 40, 1)]], ids=["random", "ct"])
def test_plan_holds_the_papers_tile_tasks(shapes, tile):
    plan, nparts = ctqr.batch_plan(shapes, tile)
    types = plan[:, 0]
    want = _expected_counts(shapes, tile)
    got = {name: int((types == t).sum()) for t, name in enumerate(NAMES)}
    assert got == want
    assert nparts > 0 and plan[:, 1].min() >= 0 and plan[:, 1].max() == len(shapes) - 1


@pytest.mark.parametrize("tile", [32, 64])
def test_plan_order_meets_every_dependency_exactly(tile):
    plan, nparts = ctqr.batch_plan(SHAPES + [(2387, 1024, 1)], tile)
    cnt = np.zeros(2 * nparts, dtype=np.int64)
    for q, r in enumerate(plan):
        nd, ni = r[5], r[6]
        dep_c, dep_v, inc_c = r[7:7 + nd], r[13:13 + nd], r[19:19 + ni]
        assert (dep_c >= 0).all() and (dep_c < 2 * nparts).all()
        assert np.array_equal(cnt[dep_c], dep_v), (q, r.tolist())
        cnt[inc_c] += 1
    # the counters hold every task's increments, and some part was both read
    # and written (the dependencies are not vacuous)
    assert cnt.sum() == plan[:, 6].sum()
    assert (cnt[0::2] > 1).any() and (cnt[1::2] > 1).any()


def test_plan_rejects_bad_input():
    with pytest.raises(ctqr.CtError):
        ctqr.batch_plan([(10, 20, 1)], 32)   # m < n
    with pytest.raises(ctqr.CtError):
        ctqr.batch_plan([(100, 20, 1)], 48)  # tile not 32 or 64
