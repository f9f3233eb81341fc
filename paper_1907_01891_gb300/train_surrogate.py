"""Train the convolutional surrogate (``ct_surrogate_*``) on one scan geometry
and report what its FP64 gate accepts on unseen slices.

    python -m paper_1907_01891_gb300.train_surrogate [--n-train 20000] [--epochs 3]

Steps (all on the GPU through the library): build A in FP32 and factor it in
TF32 with FP64 panels; for every training phantom x compute the sinogram
b = A x (exact sparse A), its QR reconstruction (the gated call with tolerance
0, i.e. every slice solved through the factor with FP64-residual refinement)
and the backprojection A^T b; train on (A^T b, QR reconstruction) pairs; then
run the gated reconstruction on a batch of unseen phantoms and print one JSON
line: training time and loss, gate residuals, fallback rate, error of the
network and of the gated output against the QR solution, and slices/s with
and without the network.  Phantoms are the seeded random-ellipse phantoms of
``inputs``; the workload is the 128 x 128 fan-beam scan (128 views x 181 bins)
with noiseless sinograms.
"""
from __future__ import annotations

import argparse
import json
import time

import numpy as np
import torch

from . import ctqr
from . import inputs as I


def _sync():
    torch.cuda.synchronize()


def make_pairs(geom, f, s_proj, seeds, chunk: int = 1024):
    """(G, Q): backprojections and QR reconstructions of the phantoms `seeds`,
    as n x len(seeds) FP64 CUDA tensors (ld = n)."""
    n = geom.n
    N = len(seeds)
    G = ctqr.colmajor(n, N, ld=n)
    Q = ctqr.colmajor(n, N, ld=n)
    seeds = list(seeds)
    for c0 in range(0, N, chunk):
        cs = seeds[c0:c0 + chunk]
        X = ctqr.to_colmajor(I.phantoms(geom, cs))
        B = s_proj.project(X)
        s_proj.backproject(B, G[:, c0:c0 + len(cs)])
        s_proj.infer(B, tol=0.0, factor=f, X=Q[:, c0:c0 + len(cs)])
    return G, Q


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--n-train", type=int, default=20000)
    ap.add_argument("--epochs", type=int, default=3)
    ap.add_argument("--batch", type=int, default=32)
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--tol", type=float, default=I.CONFIG5["tol"])
    ap.add_argument("--k", type=int, default=len(I.CONFIG5["seeds"]))
    ap.add_argument("--seed", type=int, default=0)
    args = ap.parse_args(argv)

    cfg = I.CONFIG5
    geom = cfg["geom"]
    torch.manual_seed(args.seed)
    t0 = time.perf_counter()
    A = ctqr.build_system(geom, torch.float32)
    f = ctqr.qr_factor(A, ctqr.Prec.TF32, in_place=True)
    _sync()
    t_factor = time.perf_counter() - t0
    proj = ctqr.Surrogate(geom)

    t0 = time.perf_counter()
    train_seeds = list(cfg["train_seeds"])[:args.n_train]
    G, Q = make_pairs(geom, f, proj, train_seeds)
    _sync()
    t_data = time.perf_counter() - t0
    in_scale = 1.0 / float(G.abs().mean())
    out_scale = float(Q.abs().mean()) * 2.0
    net = ctqr.Surrogate(geom, in_scale=in_scale, out_scale=out_scale, seed=args.seed)

    N = len(train_seeds)
    gen = torch.Generator().manual_seed(args.seed)
    losses = []
    t0 = time.perf_counter()
    steps = 0
    total_steps = args.epochs * (N // args.batch)
    for ep in range(args.epochs):
        perm = torch.randperm(N, generator=gen).cuda()
        Gs = G.t()[perm].t()  # shuffled copies, column-major n x N
        Qs = Q.t()[perm].t()
        for b0 in range(0, N - args.batch + 1, args.batch):
            # cosine decay of the step size over the whole run
            lr = args.lr * 0.5 * (1.0 + np.cos(np.pi * steps / max(total_steps, 1)))
            l = net.train_step(Gs[:, b0:b0 + args.batch], Qs[:, b0:b0 + args.batch], lr)
            steps += 1
            if steps % 50 == 0 or steps == 1:
                losses.append((steps, l))
    _sync()
    t_train = time.perf_counter() - t0

    # unseen slices: QR reference, network alone, gated
    Xte = ctqr.to_colmajor(I.phantoms(geom, cfg["seeds"][:args.k]))
    Bte = proj.project(Xte)
    _sync()
    t0 = time.perf_counter()
    Xq, _, _ = proj.infer(Bte, tol=0.0, factor=f)
    _sync()
    t_qr = time.perf_counter() - t0
    t0 = time.perf_counter()
    Xn = net.forward(net.backproject(Bte))
    _sync()
    t_net = time.perf_counter() - t0
    t0 = time.perf_counter()
    Xg, resid, rep = net.infer(Bte, tol=args.tol, factor=f)
    _sync()
    t_gated = time.perf_counter() - t0
    nq = torch.linalg.vector_norm(Xq, dim=0)
    err_net = (torch.linalg.vector_norm(Xn - Xq, dim=0) / nq).cpu().numpy()
    err_gated = (torch.linalg.vector_norm(Xg - Xq, dim=0) / nq).cpu().numpy()
    err_truth = (torch.linalg.vector_norm(Xq - Xte, dim=0) / torch.linalg.vector_norm(Xte, dim=0)).cpu().numpy()
    resid = resid.cpu().numpy()
    k = args.k
    out = dict(
        workload=cfg["name"], geometry=dict(nx=geom.nx, ny=geom.ny, views=geom.n_views, bins=geom.n_bins,
                                            m=geom.m, n=geom.n),
        n_train=N, epochs=args.epochs, batch=args.batch, steps=steps, lr=args.lr, tol=args.tol,
        s_factor=round(t_factor, 3), s_training_data=round(t_data, 3), s_train=round(t_train, 3),
        train_images_per_s=round(steps * args.batch / t_train, 1),
        loss_curve=[(s_, float(f"{l_:.4e}")) for s_, l_ in losses],
        test_slices=k, fallbacks=int(rep["fallbacks"]), fallback_rate=rep["fallbacks"] / k,
        gate_residual=dict(min=float(resid.min()), median=float(np.median(resid)), max=float(resid.max())),
        pass_fraction_at=[(t_, float((resid <= t_).mean())) for t_ in (1e-3, 1e-2, 5e-2, 1e-1, 2e-1)],
        network_error_vs_qr=dict(median=float(np.median(err_net)), max=float(err_net.max())),
        gated_error_vs_qr_max=float(err_gated.max()),
        qr_error_vs_phantom_max=float(err_truth.max()),
        slices_per_s=dict(qr=round(k / t_qr, 2), network_only=round(k / t_net, 2), gated=round(k / t_gated, 2)),
        gated_ms=dict(network=round(rep["ms_network"], 3), gate=round(rep["ms_gate"], 3),
                      fallback=round(rep["ms_fallback"], 3)),
    )
    print(json.dumps(out))
    return out


if __name__ == "__main__":
    main()
