"""Factor one seeded random matrix and print the library's per-kernel launch
counts and device times (ct_profile_*), e.g. to size or profile the panel and
update kernels on a given shape:

    python -m paper_1907_01891_gb300.factor_probe --m 23168 --n 512 --prec tf32

The matrix is factored twice; the second factorization is the one reported
(the first loads the kernels and sizes the scratch).
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
    stats = {k["name"]: {"launches": k["launches"], "ms": round(k["ms"], 4),
                         "us_per_launch": round(1e3 * k["ms"] / k["launches"], 2)}
             for k in ctqr.profile_kernels() if k["launches"]}
    print(json.dumps({"m": args.m, "n": args.n, "prec": args.prec, "status": f.status(), "kernels": stats}))


if __name__ == "__main__":
    main()
