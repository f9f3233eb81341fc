"""Factor one seeded random matrix and print the library's per-kernel launch
counts and device times (ct_profile_*), e.g. to size or profile the panel and
update kernels on a given shape:

    python -m paper_1907_01891_gb300.factor_probe --m 23168 --n 512 --prec tf32

The matrix is factored twice; the second factorization is the one reported
(the first loads the kernels and sizes the scratch).  With ``--rhs K`` (FP32
and TF32 factors) it then applies Q^T to K seeded right-hand sides in FP32
(``ct_apply_qt_f32``) and solves with R and R^T (``ct_trsm_solve_f32``), twice
each, and reports the second round's per-kernel counts and times as well.
"""
from __future__ import annotations

import argparse
import json

import torch

from . import ctqr
from . import inputs as I


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--m", type=int, default=23168)
    ap.add_argument("--n", type=int, default=512)
    ap.add_argument("--prec", choices=["f64", "f32", "tf32"], default="tf32")
    ap.add_argument("--seed", type=int, default=5)
    ap.add_argument("--rhs", type=int, default=0)
    args = ap.parse_args(argv)
    prec = {"f64": ctqr.Prec.F64, "f32": ctqr.Prec.F32, "tf32": ctqr.Prec.TF32}[args.prec]
    dtype = torch.float64 if prec == ctqr.Prec.F64 else torch.float32
    A = ctqr.to_colmajor(I.random_matrix(args.m, args.n, seed=args.seed), dtype=dtype)
    ctqr.qr_factor(A, prec)
    torch.cuda.synchronize()
    ctqr.profile_reset()
    ctqr.profile_enable(True)
    f = ctqr.qr_factor(A, prec)
    torch.cuda.synchronize()
    ctqr.profile_enable(False)
    stats = _stats()
    out = {"m": args.m, "n": args.n, "prec": args.prec, "status": f.status(), "kernels": stats}
    if args.rhs > 0 and prec != ctqr.Prec.F64:
        B = ctqr.to_colmajor(I.random_matrix(args.m, args.rhs, seed=args.seed + 1), dtype=torch.float32)
        Y = ctqr.to_colmajor(I.random_matrix(args.n, args.rhs, seed=args.seed + 2), dtype=torch.float32)
        for rnd in range(2):
            torch.cuda.synchronize()
            ctqr.profile_reset()
            ctqr.profile_enable(rnd == 1)
            ctqr.apply_qt_f32(f, B)
            ctqr.trsm_solve_f32(f, Y)
            ctqr.trsm_solve_f32(f, Y, transpose=True)
            torch.cuda.synchronize()
        ctqr.profile_enable(False)
        out["solve_kernels"] = _stats()
    print(json.dumps(out))


def _stats():
    return {k["name"]: {"launches": k["launches"], "ms": round(k["ms"], 4),
                        "us_per_launch": round(1e3 * k["ms"] / k["launches"], 2)}
            for k in ctqr.profile_kernels() if k["launches"]}


if __name__ == "__main__":
    main()
