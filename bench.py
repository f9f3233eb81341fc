"""Benchmark: QR-based CT reconstruction on one GB300 (arXiv 1907.01891).

One step is one pass of the whole method over one batch of slices: build the
system matrix A on the GPU, factor A = QR, apply Q^T to the batch of
sinograms, back-solve, and (mixed precision) refine with FP64 residuals --
all through ct_reconstruct_scan of the C ABI, with the sinograms already in
HBM.  value = slices reconstructed per second (whole job, all ranks).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--workload NAME] [--prec P]
  python bench.py --impl reference ...   # the plain CPU oracle on the host
  python bench.py --probe M N [--rhs K]  # per-kernel launch list of one factorization

The default workload is the 256 x 256 fan-beam system stacked over 1e-3 I
(135232 x 65536, 64 slices) with the tensor-core factor whose products split
every FP32 operand into two FP16 parts (--prec f16x3; --prec tf32 selects the
three-pass TF32 split) and FP64 refinement; after the timed steps the plain
FP64 QR path reconstructs the same scan once, for the relative error and the
FP64 path's slices/s.

Multi-GPU (torchrun): every rank reconstructs its own scan (independent
replicas, weak scaling); there is no data-path collective.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_1907_01891_gb300 import inputs as I  # noqa: E402

METRIC = "slices/s & QR TFLOP/s: mixed-prec+refine vs FP64 QR, 1 GB300, rel err ≤1e-10"
WORKLOADS = {"fan128": I.CONFIG2, "fan256": I.CONFIG3, "parallel32": I.CONFIG1, "batch64": I.CONFIG4B}
PREC = {"f64": 0, "f32": 1, "tf32": 2, "f16x3": 3}
DTYPE_NAME = {"f64": "f64", "f32": "f32+f64", "tf32": "tf32+f64", "f16x3": "f16x3+f64"}


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=2)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", choices=["ours", "reference"], default="ours")
    p.add_argument("--workload", choices=sorted(WORKLOADS), default="fan256")
    p.add_argument("--prec", choices=sorted(PREC), default="f16x3")
    p.add_argument("--e2e-steps", type=int, default=1)
    p.add_argument("--cpu-seconds", type=float, default=15.0, help="budget of the oracle sample")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--fp64-check", type=int, default=1,
                   help="after the timed steps, reconstruct the scan once through the plain FP64 QR "
                        "path (relative error and FP64 slices/s; about 15 min on the 256x256 system)")
    p.add_argument("--probe", type=int, nargs=2, metavar=("M", "N"), default=None,
                   help="factor one seeded M x N matrix and print its per-kernel launch list")
    p.add_argument("--rhs", type=int, default=0, help="--probe: also time Q^T and R^-1, R^-T on K columns")
    p.add_argument("--seed", type=int, default=5, help="--probe: seed of the matrix")
    p.add_argument("--ooc", action="store_true",
                   help="out-of-core table: the paper's scanner (Table scanner, Eq. angulos) at 128 x 128, "
                        "Joseph sinograms, FP64 factor in host memory streamed through a small HBM budget, "
                        "seconds per slice for S = 256..2048 with and without copy/compute overlap")
    p.add_argument("--ooc-npix", type=int, default=128)
    p.add_argument("--ooc-budget", type=float, default=0.1, help="HBM budget as a fraction of the matrix")
    return p.parse_args()


# ncu DRAM traffic (read + write) over algorithmic bytes, per (kernel class,
# precision), each from one capture of that kernel on a smaller case of the
# same shape family (launch, rows, columns in the value); absent: not
# captured since the kernel last changed.  The roofline's traffic is this ratio times the
# dominant class's algorithmic bytes per launch.
TRAFFIC_RATIO = {
    # k_tc_update16<2>, C -= V W' of a 134,976 x 768 block with K = 256 (the
    # ninth tensor-core update launch of `bench.py --probe 135232 1024`, C
    # larger than L2): 562.1 MB read + 360.9 MB written against 968.3 MB of
    # algorithmic bytes (C read and written once, FP16 operand parts once)
    ("tc_update", "f16x3"): {"ratio": 922.946816 / 968.2944,
                  "capture": "k_tc_update16 on a 134976 x 768 x 256 block (ncu --set full)"},
}


def qr_flops(m, n):
    return 2.0 * m * n * n - 2.0 * n ** 3 / 3.0


def solve_flops(m, n, k):
    return (4.0 * m * n - 2.0 * n * n + n * n) * k


# ---------------------------------------------------------------- clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id: str | None):
        self.proc = None
        self.gpu_id = gpu_id

    def start(self):
        cmd = ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "200"]
        if self.gpu_id:
            cmd += ["-i", self.gpu_id]
        try:
            self.proc = subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.splitlines():
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "samples": len(sm),
                "reasons": sorted(reasons)}


# ---------------------------------------------------------------- distributed
def dist_setup(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def reduce_max(value: float, world: int, device) -> float:
    if world == 1:
        return value
    import torch
    import torch.distributed as dist
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier(world: int):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def replica_seeds(seeds, rank: int):
    """Every rank reconstructs its own scan: the same phantom recipe with the
    seeds shifted by 100000 per rank (independent replicas, no exchange)."""
    return [s + 100000 * rank for s in seeds]


def job_throughput(world: int, units_per_rank: int, steps: int, ms_max: float) -> float:
    """Whole-job units per second: all ranks' units over the slowest rank's time."""
    return world * units_per_rank * steps / (ms_max / 1e3)


# ---------------------------------------------------------------- oracle timing
class OracleSampler:
    """Bounded samples of one step of the workload run by the plain CPU oracle
    on the host cores: (1) the system matrix of a subset of the views (scaled
    by rays to the whole scan) and (2) unblocked Householder QR, Q^T and
    back-solve of the k slices on the first ns columns of a seeded m x ns
    matrix at the system's full height (scaled by flops to n columns).  The
    sample size is calibrated once so that one sample takes about `target_s`
    seconds; every sample reports its measured time and the time a full step
    would take at the measured rates (labelled as extrapolated)."""

    def __init__(self, cfg, k: int, m: int, n: int, target_s: float):
        from oracle import oracle as O
        self.O, self.cfg, self.k, self.m, self.n = O, cfg, k, m, n
        g = cfg["geom"]
        self.views = max(1, min(g.n_views, int(g.n_views * min(1.0, 2048.0 / max(g.m, 1)))))
        self.gs = O.Geometry(g.beam, g.nx, g.ny, g.pixel, self.views, g.n_bins, g.angle0,
                             g.angle_span * self.views / g.n_views, g.src_iso, g.det_span, g.angle_rule)
        self.cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
        self.rng = np.random.default_rng(0)
        # calibrate ns: grow until one QR + solve sample takes ~target_s / 2
        ns, t = 32, 0.0
        while True:
            t = self._qr_solve(ns)
            if t > target_s / 4 or ns >= n:
                break
            ns = min(n, int(ns * min(4.0, max(1.25, math.sqrt(target_s / 2 / max(t, 1e-3))))))
        self.ns = ns

    def _qr_solve(self, ns: int) -> float:
        A = np.asfortranarray(self.rng.standard_normal((self.m, ns)))
        B = np.asfortranarray(self.rng.standard_normal((self.m, self.k)))
        t0 = time.perf_counter()
        F, tau = self.O.qr(A)
        Y = self.O.apply_qt(F, tau, B)
        self.O.backsolve(F, Y)
        return time.perf_counter() - t0

    def sample(self):
        """One sample: (measured seconds, extrapolated seconds of a full step)."""
        g = self.cfg["geom"]
        t0 = time.perf_counter()
        self.O.system_matrix(self.gs)
        t_build = time.perf_counter() - t0
        t_qr = self._qr_solve(self.ns)
        full = (t_build * g.m / self.gs.m +
                t_qr * (qr_flops(self.m, self.n) + solve_flops(self.m, self.n, self.k)) /
                (qr_flops(self.m, self.ns) + solve_flops(self.m, self.ns, self.k)))
        return t_build + t_qr, full

    def describe(self) -> str:
        g = self.cfg["geom"]
        return (f"oracle on {self.cores} host cores: system matrix for {self.views} of {g.n_views} views "
                f"(scaled by rays) + unblocked Householder QR, Q^T and back-solve of {self.k} slices on the "
                f"first {self.ns} of {self.n} columns at full height m={self.m} (scaled by flops); "
                f"the full step is extrapolated from the measured rates")

    def lapack(self, target_s: float):
        """The strong CPU baseline: LAPACK's blocked Householder QR
        least-squares solve (dgeqrf, dormqr, dtrtrs through scipy) of an
        m x ns sample (ns grown from 32 until one solve takes about
        target_s / 4), flop-scaled to n columns.  Returns (extrapolated
        seconds of a full step's QR + solve, threads, description)."""
        from scipy.linalg import lapack
        ns, t = 32, 0.0
        rng = np.random.default_rng(1)
        B = np.asfortranarray(rng.standard_normal((self.m, self.k)))

        def solve(A):
            qr, tau, _, _ = lapack.dgeqrf(A, overwrite_a=1)
            lwork = int(lapack.dormqr("L", "T", qr, tau, B, -1)[1][0].real)
            c, _, _ = lapack.dormqr("L", "T", qr, tau, B, max(lwork, 1))
            lapack.dtrtrs(qr[:ns, :ns], c[:ns], lower=0)

        while True:
            A = np.asfortranarray(rng.standard_normal((self.m, ns)))
            t0 = time.perf_counter()
            solve(A)
            t = time.perf_counter() - t0
            if t > target_s / 4 or ns >= self.n:
                break
            ns = min(self.n, int(ns * min(4.0, max(1.25, math.sqrt(target_s / 2 / max(t, 1e-3))))))
        full = t * (qr_flops(self.m, self.n) + solve_flops(self.m, self.n, self.k)) / (
            qr_flops(self.m, ns) + solve_flops(self.m, ns, self.k))
        threads = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
        return full, threads, (
            f"LAPACK dgeqrf + dormqr + dtrtrs (scipy) on the first {ns} of {self.n} columns at full height, "
            f"measured {t:.2f} s, flop-scaled (QR + solve only)")


def _oracle_worker(workload, k, m, n, target_s):
    """The oracle sample (runs in a spawned process)."""
    t0 = time.perf_counter()
    sampler = OracleSampler(WORKLOADS[workload], k, m, n, target_s=target_s)
    print(f"[cpu baseline] oracle calibrated to {sampler.ns} columns in {time.perf_counter() - t0:.1f} s",
          file=sys.stderr, flush=True)
    t_meas, t_full = sampler.sample()
    return {"value": k / t_full, "unit": "slices/s", "cores": sampler.cores, "kind": "oracle",
            "sample": sampler.describe() + f" (sample measured {t_meas:.1f} s)"}


def _lapack_worker(workload, k, m, n, target_s):
    """The LAPACK sample (runs in a spawned process)."""
    sampler = OracleSampler.__new__(OracleSampler)
    sampler.m, sampler.n, sampler.k = m, n, k
    t_lp, thr, desc = sampler.lapack(target_s)
    return {"value": k / t_lp, "unit": "slices/s", "threads": thr, "sample": desc}


def _bounded(fn, args, timeout_s):
    """fn(*args) in a spawned process, stopped after timeout_s seconds;
    (result, None) or (None, reason)."""
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    pool = ctx.Pool(1)
    try:
        return pool.apply_async(fn, args).get(timeout=timeout_s), None
    except mp.TimeoutError:
        return None, f"did not finish within {timeout_s:.0f} s"
    except Exception as exc:  # the CPU baselines are context only
        return None, str(exc)[:200]
    finally:
        pool.terminate()
        pool.join()


def cpu_baseline_bounded(workload, k, m, n, target_s, timeout_s):
    """cpu_baseline object: the oracle sample and, beside it, the LAPACK
    sample, each in its own spawned process stopped after timeout_s seconds
    (the host-side samples can never hold the GPU job)."""
    cpu, why = _bounded(_oracle_worker, (workload, k, m, n, target_s), timeout_s)
    if cpu is None:
        return {"unavailable": "the oracle sample " + why}
    lp, why = _bounded(_lapack_worker, (workload, k, m, n, target_s), min(timeout_s, 90.0))
    cpu["lapack"] = lp if lp is not None else {"unavailable": "the LAPACK sample " + why}
    return cpu


_T0 = time.perf_counter()


def log(msg: str) -> None:
    """Progress on stderr with the seconds since the start."""
    print(f"[bench {time.perf_counter() - _T0:7.1f} s] {msg}", file=sys.stderr, flush=True)


def reference_main(args, cfg, k, m_sys, n_sys, world, rank):
    """The reference arm: the plain CPU oracle on the host cores, W warm-up
    and K timed steps, each step one bounded sample of the workload (see
    OracleSampler); value = slices per second extrapolated from the samples'
    measured rates.  Only rank 0 runs."""
    if rank != 0:
        return 0
    g = cfg["geom"]
    sampler = OracleSampler(cfg, k, m_sys, n_sys, target_s=args.cpu_seconds / 3)
    for _ in range(args.warmup):
        sampler.sample()
    meas, full = [], []
    for _ in range(args.steps):
        t, f = sampler.sample()
        meas.append(t)
        full.append(f)
    value = k * len(full) / sum(full)
    ms = 1e3 * sum(meas) / len(meas)
    line = {"metric": METRIC, "value": value, "unit": "slices/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic: seeded ellipse phantoms", "impl": "reference",
            "config": {"workload": f"{cfg['name']} ({m_sys}x{n_sys}, {k} slices)", "prec": "f64",
                       "parallelism": "host cores"},
            "step_is_sample": {"measured_ms_per_sample": ms,
                               "extrapolated_ms_per_full_step": 1e3 * sum(full) / len(full)},
            "cpu_baseline": {"value": value, "unit": "slices/s", "cores": sampler.cores, "kind": "oracle",
                             "sample": sampler.describe()},
            "e2e": {"value": value, "unit": "slices/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def probe_main(args):
    """Factor one seeded random M x N matrix twice and print the second
    factorization's per-kernel launch counts and device times; with --rhs K
    (FP32 / TF32 factors) also Q^T of K columns in FP32 and the R^-1 and R^-T
    solves, twice, the second round reported.  Used for the ncu captures."""
    import torch
    from paper_1907_01891_gb300 import ctqr
    ctqr.load()
    m, n = args.probe
    prec = ctqr.Prec(PREC[args.prec])
    dtype = torch.float64 if prec == ctqr.Prec.F64 else torch.float32
    A = ctqr.to_colmajor(I.random_matrix(m, n, seed=args.seed), dtype=dtype)

    def stats():
        return {k["name"]: {"launches": k["launches"], "ms": round(k["ms"], 4),
                            "us_per_launch": round(1e3 * k["ms"] / k["launches"], 2)}
                for k in ctqr.profile_kernels() if k["launches"]}

    ctqr.qr_factor(A, prec)
    torch.cuda.synchronize()
    ctqr.profile_reset()
    ctqr.profile_enable(True)
    f = ctqr.qr_factor(A, prec)
    torch.cuda.synchronize()
    ctqr.profile_enable(False)
    out = {"m": m, "n": n, "prec": args.prec, "status": f.status(), "kernels": stats()}
    if args.rhs > 0 and prec != ctqr.Prec.F64:
        B = ctqr.to_colmajor(I.random_matrix(m, args.rhs, seed=args.seed + 1), dtype=torch.float32)
        Y = ctqr.to_colmajor(I.random_matrix(n, args.rhs, seed=args.seed + 2), dtype=torch.float32)
        for rnd in range(2):
            torch.cuda.synchronize()
            ctqr.profile_reset()
            ctqr.profile_enable(rnd == 1)
            ctqr.apply_qt_f32(f, B)
            ctqr.trsm_solve_f32(f, Y)
            ctqr.trsm_solve_f32(f, Y, transpose=True)
            torch.cuda.synchronize()
        ctqr.profile_enable(False)
        out["solve_kernels"] = stats()
    print(json.dumps(out))
    return 0


def ooc_main(args):
    """The paper's experiment of Table time_per_slice on GB300: the factor of
    the scanner's system matrix lives in host memory (the paper: on disk) and
    streams through an HBM budget (the paper: a RAM block cache) once per
    solve, with (O-OOC) and without (B-OOC) a copy stream overlapping the
    transfers; solve time per slice for S = 256, 512, 1024, 2048 slices."""
    import torch
    from paper_1907_01891_gb300 import ctqr
    ctqr.load()
    npix = args.ooc_npix
    g = I.scanner_geometry(npix, 260 * npix // 512, 1025 * npix // 512 | 1)
    lam = 1e-3
    m, n = ctqr.system_size(g, lam)
    log(f"scanner {npix}x{npix}: {g.n_views} views x {g.n_bins} bins, system {m} x {n} = [A; {lam:g} I]")
    Ad = ctqr.build_system(g, torch.float64, lam=lam)
    H = torch.empty((n, m), dtype=torch.float64).pin_memory().t()   # page-locked host matrix
    budget = int(args.ooc_budget * m * n * 8)
    S_list = [256, 512, 1024, 2048]
    seeds = list(range(70000, 70000 + max(S_list)))
    Xt = torch.as_tensor(I.phantoms(g, seeds), device="cuda")
    Bj = ctqr.project_joseph(g, ctqr.to_colmajor(Xt))   # the paper's sinograms: Joseph's projector
    B = ctqr.colmajor(m, max(S_list), fill=0.0)
    B[:g.m].copy_(Bj)
    del Bj
    out = {"metric": "out-of-core solve s/slice (factor in host memory, streamed through an HBM budget)",
           "unit": "s/slice", "higher_is_better": False, "n_gpus": 1, "dtype": "f64",
           "data": "synthetic: seeded ellipse phantoms, sinograms by Joseph's projector",
           "config": {"workload": f"scanner{npix} (Table scanner proportions, Eq. angulos views; "
                                  f"{g.n_views} views x {g.n_bins} bins; system {m}x{n} = [A; {lam:g} I])",
                      "hbm_budget_bytes": budget, "matrix_bytes": m * n * 8}}
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    stream = torch.cuda.current_stream()
    rows = {}
    for overlap in (False, True):
        H.copy_(Ad)   # the system matrix in host memory (the factor overwrites it)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        f = ctqr.qr_factor_host(H, device_bytes=budget, overlap=overlap)
        t_fact = time.perf_counter() - t0
        st = f.status()
        mode = "O-OOC" if overlap else "B-OOC"
        res = {"factor_s": t_fact, "status": st, "qr_tflops": qr_flops(m, n) / t_fact / 1e12}
        for S in S_list:
            Bs = B[:, :S]
            ctqr.reconstruct(f, Bs)     # warm-up of this size
            e0.record(stream)
            X, _ = ctqr.reconstruct(f, Bs)
            e1.record(stream)
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1)
            res[f"S={S}"] = {"s_per_slice": ms / 1e3 / S, "slices_per_s": S / (ms / 1e3), "solve_ms": ms}
            if S == max(S_list):
                Xl = X.clone()
        rows[mode] = res
        log(f"{mode}: factor {t_fact:.1f} s; " + ", ".join(
            f"S={S}: {res[f'S={S}']['s_per_slice'] * 1e3:.3f} ms/slice" for S in S_list))
        f.destroy()
    # accuracy: the streamed solution against the in-HBM FP64 factor's, and
    # image quality against the phantoms (Joseph data: the model mismatch)
    fd = ctqr.qr_factor(Ad)
    Bs = B[:, :64]
    Xd, _ = ctqr.reconstruct(fd, Bs)
    rel = float(torch.linalg.norm(Xl[:, :64] - Xd) / torch.linalg.norm(Xd))
    e0.record(stream)
    ctqr.reconstruct(fd, B)
    e1.record(stream)
    torch.cuda.synchronize()
    in_hbm = e0.elapsed_time(e1) / 1e3 / max(S_list)
    q = ctqr.image_quality(Xl, ctqr.to_colmajor(Xt), g.nx, g.ny).cpu().numpy()
    out["value"] = rows["O-OOC"][f"S={max(S_list)}"]["s_per_slice"]
    out["table"] = rows
    out["in_hbm_s_per_slice_S2048"] = in_hbm
    out["rel_err_streamed_vs_in_hbm"] = rel
    out["quality_vs_phantom"] = {"psnr_db_median": float(np.median(q[:, 1])), "ssim_median": float(np.median(q[:, 2]))}
    out["paper_context"] = ("Table time_per_slice, i7-7800X + SSD, 512x512 scanner: O-OOC 1.65 / 1.00 / 0.83 / "
                            "0.72 s per slice, B-OOC + HDD 14.54 / 7.72 / 4.33 / 2.50 s (S = 256..2048): other "
                            "hardware and size")
    print(json.dumps(out))
    return 0


def load_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except OSError:
        return {}


def roofline(dom, prec, ms_step, peaks):
    """Roofline object of the dominant kernel class (the one with the most
    device time in the profiled step)."""
    sm_max_ghz = (peaks.get("sm_max_mhz") or 2070.0) / 1e3
    fp64_peak = 152 * 2 * 2 * sm_max_ghz * 1e9 / 1e12      # 2 DFMA/clk/SM (measured 1.204 TF/s)
    fp32_peak = 152 * 128 * 2 * sm_max_ghz * 1e9 / 1e12    # 128 FFMA/clk/SM
    hbm = peaks.get("hbm_gbs")
    hbm_src = "measured (MEASURED_PEAKS.json hbm_gbs)" if hbm else "fallback 6800 GB/s"
    hbm = hbm or 6800.0
    # Tensor peak of the products' input type.  TF32: cuBLAS TF32 8192^3
    # measured on this machine's GB300 (1040 TFLOP/s), above the BF16-derived
    # figure (sustained BF16 x 1.1/2.25).  FP16 (the FP16-split factor): the
    # measured sustained BF16 rate (FP16 and BF16 MMAs run at the same rate;
    # the factorization is a seconds-long step).
    if prec == "f16x3":
        t_peak = peaks.get("bf16_tflops_sustained") or 1700.0
        t_src = ("measured sustained cuBLAS BF16 (MEASURED_PEAKS.json bf16_tflops_sustained; FP16 runs at "
                 "the BF16 rate)" if peaks.get("bf16_tflops_sustained") else "fallback 1.7 PFLOP/s sustained")
        t_note = "algorithmic flops 2MNK; the FP16 split issues three FP16 MMAs per product"
    else:
        t_peak, t_src = TF32_MEASURED_TFLOPS, "measured cuBLAS TF32 (8192^3) on a GB300 of this pool"
        t_note = "algorithmic flops 2MNK; 3xTF32 issues three MMAs per product"
    name = dom["name"]
    if name in ("zero_fill", "copy", "system_matrix", "tc_update", "tc_fused"):
        roof = {"bound": "hbm", "achieved": dom["bytes"] / (dom["ms"] / 1e3) / 1e9, "peak": hbm, "unit": "GB/s",
                "peak_source": hbm_src}
        if name in ("tc_update", "tc_fused"):
            roof["tensor_rate"] = {"achieved": dom["flops"] / (dom["ms"] / 1e3) / 1e12, "peak": t_peak,
                                   "unit": "TFLOP/s", "issued_x": 3, "peak_source": t_src, "note": t_note}
    elif name == "tc_gemm":
        roof = {"bound": "tensor", "achieved": dom["flops"] / (dom["ms"] / 1e3) / 1e12, "peak": t_peak,
                "unit": "TFLOP/s", "peak_source": t_src, "note": t_note}
    else:
        alu = fp64_peak if prec == "f64" or name == "panel_qr" else fp32_peak
        roof = {"bound": "alu", "achieved": dom["flops"] / (dom["ms"] / 1e3) / 1e12, "peak": alu,
                "unit": "TFLOP/s",
                "peak_source": "derived: 152 SMs x %s FMA/clk x 2 x %.2f GHz" % (
                    "2 FP64" if alu == fp64_peak else "128 FP32", sm_max_ghz)}
    roof["frac"] = roof["achieved"] / roof["peak"]
    roof["kernel"] = name
    roof["launches_per_step"] = dom["launches"]
    roof["share_of_step"] = dom["ms"] / ms_step
    roof["timed_in"] = "one extra step with CUDA events around every launch of the class"
    ratio = TRAFFIC_RATIO.get((name, prec))
    if ratio is not None and dom["launches"]:
        roof["traffic"] = ratio["ratio"] * dom["bytes"] / dom["launches"]
        roof["traffic_source"] = ("ncu dram read + write of " + ratio["capture"] +
                                  " over its algorithmic bytes (%.3f), times this step's algorithmic "
                                  "bytes per launch" % ratio["ratio"])
    else:
        roof["traffic"] = None
    return roof


# cuBLAS TF32 GEMM (8192^3) measured on a GB300 of this machine, TFLOP/s.
TF32_MEASURED_TFLOPS = 1040.0


# ---------------------------------------------------------------- main
def main():
    args = parse()
    if args.probe:
        return probe_main(args)
    if args.ooc:
        return ooc_main(args)
    world, rank, local = dist_setup(args)
    cfg = WORKLOADS[args.workload]
    if args.workload == "batch64":
        return main_batch(args, world, rank, local, cfg)
    g = cfg["geom"]
    k = len(cfg["seeds"])
    lam = cfg.get("lam", 0.0)
    m_sys = g.m + (g.n if lam > 0 else 0)
    n_sys = g.n

    if args.impl == "reference":
        return reference_main(args, cfg, k, m_sys, n_sys, world, rank)

    import torch
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    from paper_1907_01891_gb300 import ctqr
    ctqr.load()
    assert ctqr.system_size(g, lam) == (m_sys, n_sys)

    # ---- inputs (outside the timed region): phantoms, sinograms B = A x (+ noise)
    seeds = replica_seeds(cfg["seeds"], rank)
    Xtrue = I.phantoms(g, seeds)
    A = ctqr.build_system(g, torch.float64)  # rays only, for the inputs and the checks
    B = ctqr.colmajor(m_sys, k, fill=0.0)     # [b; 0] when lambda*I is stacked
    B[:g.m].copy_(A @ torch.as_tensor(Xtrue, device=dev))
    torch.cuda.synchronize()
    if cfg["noise_i0"]:
        Bn = I.poisson_noise(B[:g.m].cpu().numpy(), g.fov, cfg["noise_i0"], seed=seeds[0])
        B[:g.m].copy_(torch.as_tensor(Bn))
    torch.cuda.synchronize()
    X = ctqr.colmajor(n_sys, k)
    prec = ctqr.Prec(PREC[args.prec])

    def step():
        return ctqr.reconstruct_scan(g, B, X=X, prec=prec, lam=lam)

    log(f"inputs ready ({m_sys} x {n_sys}, {k} slices); warm-up")
    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    log("warm-up done; timed steps")
    # Accuracy at any size: optimality of the (regularized) least-squares
    # solution, ||A^T (b - A x) - lam^2 x|| / (||A||_F^2 ||x||).
    r = B[:g.m] - A @ X
    gres = A.t() @ r - (lam * lam) * X
    normal_eq = float(torch.linalg.norm(gres) / (torch.linalg.norm(A) ** 2 * torch.linalg.norm(X)))
    del r, gres, A
    torch.cuda.empty_cache()

    gpu_id = None
    try:
        gpu_id = "GPU-" + str(torch.cuda.get_device_properties(dev).uuid)
    except Exception:
        gpu_id = None
    clocks = ClockSampler(gpu_id)
    ctqr.profile_reset()
    stream = torch.cuda.current_stream()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    barrier(world)
    torch.cuda.synchronize()
    clocks.start()
    reps = []
    e0.record(stream)
    for _ in range(args.steps):
        _, r = step()
        reps.append(r)
    e1.record(stream)
    torch.cuda.synchronize()
    barrier(world)
    clk = clocks.stop()
    launches = ctqr.kernel_launches()  # launches of the timed steps (counted, not timed)
    ms = e0.elapsed_time(e1)
    ms_max = reduce_max(ms, world, dev)
    value = job_throughput(world, k, args.steps, ms_max)
    X_mixed = X.clone()
    # Per-kernel device times come from one more step with CUDA events around
    # every launch (outside the timed region: the events add host work).
    ctqr.profile_reset()
    ctqr.profile_enable(True)
    step()
    torch.cuda.synchronize()
    ctqr.profile_enable(False)
    kstats = ctqr.profile_kernels()
    ms_factor = statistics.median(r.ms_factor for r in reps)
    ms_solve = statistics.median(r.ms_solve for r in reps)
    ms_build = statistics.median(r.ms_build for r in reps)
    peaks = load_peaks()
    dom = max(kstats, key=lambda s_: s_["ms"])
    roof = roofline(dom, args.prec, ms / args.steps, peaks)

    log("timed steps done; end to end from host buffers")
    # ---- end to end through the public API with host buffers
    Bh = B.cpu()
    Bp = torch.empty((k, m_sys), dtype=torch.float64).pin_memory().t()
    Bp.copy_(Bh)
    Xp = torch.empty((k, n_sys), dtype=torch.float64).pin_memory().t()
    barrier(world)
    t0 = time.perf_counter()
    for _ in range(args.e2e_steps):
        ctqr.reconstruct_scan(g, Bp, X=Xp, prec=prec, lam=lam)
    t_e2e = reduce_max(time.perf_counter() - t0, world, dev)
    e2e = None
    if args.e2e_steps > 0:
        e2e = {"value": world * k * args.e2e_steps / t_e2e, "unit": "slices/s",
               "h2d_bytes_per_step": m_sys * k * 8, "d2h_bytes_per_step": n_sys * k * 8}
    del Bp, Xp

    # ---- the plain FP64 QR path on the same scan, once (after the timed
    # region): relative error of the mixed-precision result against it and
    # its own slices/s
    fp64 = None
    if args.fp64_check and args.prec != "f64":
        log("FP64 QR path on the same scan")
        torch.cuda.empty_cache()
        f0 = torch.cuda.Event(enable_timing=True)
        f1 = torch.cuda.Event(enable_timing=True)
        f0.record(stream)
        X64, rep64 = ctqr.reconstruct_scan(g, B, prec=ctqr.Prec.F64, lam=lam)
        f1.record(stream)
        torch.cuda.synchronize()
        ms64 = f0.elapsed_time(f1)
        d = X_mixed - X64
        fp64 = {"rel_err_vs_fp64_qr": float(torch.linalg.norm(d) / torch.linalg.norm(X64)),
                "max_abs_err_vs_fp64_qr_rel": float(d.abs().max() / X64.abs().max()),
                "fp64_qr_slices_per_s": k / (ms64 / 1e3), "fp64_ms_per_step": ms64,
                "fp64_qr_tflops": qr_flops(m_sys, n_sys) / (rep64.ms_factor / 1e3) / 1e12,
                "fp64_phase_ms": {"build": rep64.ms_build, "factor": rep64.ms_factor, "solve": rep64.ms_solve},
                "speedup_mixed_vs_fp64": (ms64 / 1e3) / (ms_max / args.steps / 1e3),
                "measured": "one FP64 reconstruct_scan of the same scan after the timed steps, CUDA events"}
        del X64

    line = {"metric": METRIC, "value": value, "unit": "slices/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": DTYPE_NAME[args.prec],
            "data": "synthetic: seeded ellipse phantoms" + (
                f", Poisson noise I0={cfg['noise_i0']:g}" if cfg["noise_i0"] else ", noiseless b = Ax"),
            "config": {"workload": f"{cfg['name']} (system {m_sys}x{n_sys}"
                                   + (f" = [A; {lam:g} I]" if lam else "") + f", {k} slices per scan)",
                       "prec": args.prec, "parallelism": f"replicas x{world}",
                       "l2": f"inputs larger than L2 (A {g.m * g.n * 8 / 1e9:.2f} GB FP64 per step)"},
            "qr_tflops": qr_flops(m_sys, n_sys) / (ms_factor / 1e3) / 1e12,
            "solve_slices_per_s": k / (ms_solve / 1e3),
            "phase_ms": {"build": ms_build, "factor": ms_factor, "solve": ms_solve},
            "rel_err_vs_fp64_qr": fp64["rel_err_vs_fp64_qr"] if fp64 else None,
            "fp64_qr": fp64,
            "normal_eq_residual": normal_eq,
            "refine_iterations": reps[-1].iterations,
            "panel_arithmetic": ("FP32-stored factors: Cholesky-QR panels whose Gram matrix and row solves are "
                                 "compensated FP32 (Dot2) products, the 32x32 algebra, tau and T in FP64"
                                 if args.prec != "f64" else "FP64 per-column Householder panels"),
            "update_arithmetic": {
                "f16x3": "tcgen05 kind::f16: each FP32 operand split into two FP16 parts (per-column power-of-two "
                         "scales), three FP16 products with FP32 accumulation, TMEM chunks summed every 256 rows",
                "tf32": "tcgen05 kind::tf32: each FP32 operand split into TF32 high and low parts, three products "
                        "with FP32 accumulation, TMEM chunks summed every 256 rows",
                "f32": "FP32 on the CUDA cores", "f64": "FP64 on the CUDA cores"}[args.prec],
            "roofline": roof, "e2e": e2e, "clocks": clk, "gpu_launches": launches,
            "kernels": {s_["name"]: {"launches": s_["launches"], "ms": round(s_["ms"], 3)}
                        for s_ in kstats if s_["launches"]}}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        log("CPU baselines (oracle, LAPACK) in a spawned process")
        line["cpu_baseline"] = cpu_baseline_bounded(args.workload, k, m_sys, n_sys, args.cpu_seconds,
                                                    timeout_s=6 * args.cpu_seconds + 60)
    if rank == 0:
        print(json.dumps(line))
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


# ---------------------------------------------------------------- batched workload
def batch_inputs(cfg):
    """Geometries, phantoms and systems of the uneven batch (host side)."""
    geoms = I.uneven_systems(cfg["count"], cfg["seed"])
    X = [I.phantoms(g, [cfg["seed0"] + q]) for q, g in enumerate(geoms)]
    return geoms, X


def oracle_batch_sample(cfg, budget_s: float):
    """The oracle's QR + solve of the smallest system of the batch (measured),
    scaled by flops to the whole batch.  Returns (seconds, cores, description)."""
    from oracle import oracle as O
    geoms, X = batch_inputs(cfg)
    lam = cfg["lam"]
    q = min(range(len(geoms)), key=lambda i: geoms[i].m * geoms[i].n)
    g = geoms[q]
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    t0 = time.perf_counter()
    A = O.system_matrix(O.Geometry(*g.as_tuple()))
    Asys = np.vstack([A, lam * np.eye(g.n)])
    b = np.vstack([A @ X[q], np.zeros((g.n, 1))])
    O.lstsq(Asys, b)
    dt = time.perf_counter() - t0
    total = sum(qr_flops(x.m + x.n, x.n) + solve_flops(x.m + x.n, x.n, 1) for x in geoms)
    mine = qr_flops(g.m + g.n, g.n) + solve_flops(g.m + g.n, g.n, 1)
    desc = (f"oracle system matrix + unblocked Householder QR + solve of the smallest system "
            f"({g.m + g.n}x{g.n}, measured {dt:.1f} s), flop-scaled to the {len(geoms)} systems")
    return dt * total / mine, cores, desc


def main_batch(args, world, rank, local, cfg):
    """64 uneven [A; lambda I] systems factored and solved in one persistent
    graph-captured launch per step (ct_qr_solve_batched); value = systems/s."""
    count, lam = cfg["count"], cfg["lam"]
    metric = "systems/s & QR TFLOP/s: 64 uneven [A; 1e-3 I] systems, one persistent launch, 1 GB300"
    geoms, Xtrue = batch_inputs(cfg)
    flops = sum(qr_flops(g.m + g.n, g.n) + solve_flops(g.m + g.n, g.n, 1) for g in geoms)
    wl = f"{cfg['name']} ({count} systems {min(g.m + g.n for g in geoms)}..{max(g.m + g.n for g in geoms)} rows)"
    if args.impl == "reference":
        if rank != 0:
            return 0
        t, cores, desc = oracle_batch_sample(cfg, args.cpu_seconds)
        value = count / t
        print(json.dumps({"metric": metric, "value": value, "unit": "systems/s", "n_gpus": args.gpus,
                          "steps": args.steps, "warmup": args.warmup, "ms_per_step": t * 1e3,
                          "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
                          "data": "synthetic: seeded ellipse phantoms, noiseless", "impl": "reference",
                          "config": {"workload": wl, "parallelism": "host cores"},
                          "cpu_baseline": {"value": value, "unit": "systems/s", "cores": cores, "kind": "oracle",
                                           "sample": desc},
                          "e2e": {"value": value, "unit": "systems/s", "h2d_bytes_per_step": 0,
                                  "d2h_bytes_per_step": 0}}))
        return 0
    import torch
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    from paper_1907_01891_gb300 import ctqr
    ctqr.load()
    # FP64: the persistent tile-task launch; tf32: per-system tensor-core
    # factor + FP64 refinement
    bprec = ctqr.Prec(PREC[args.prec]) if args.prec in ("tf32", "f16x3") else ctqr.Prec.F64
    A0, B0, As, Bs = [], [], [], []
    for g, x in zip(geoms, Xtrue):
        A = ctqr.build_system(g, torch.float64, lam=lam)
        b = ctqr.colmajor(g.m + g.n, 1, fill=0.0)
        b[:g.m].copy_(A[:g.m] @ torch.as_tensor(x, device=dev))
        A0.append(A)
        B0.append(b)
        As.append(ctqr.colmajor(g.m + g.n, g.n))
        Bs.append(ctqr.colmajor(g.m + g.n, 1))
    torch.cuda.synchronize()

    def step():
        for A, Aw, b, bw in zip(A0, As, B0, Bs):
            Aw.copy_(A)
            bw.copy_(b)
        return ctqr.qr_solve_batched(As, Bs, tile=0, prec=bprec)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    # accuracy: least-squares optimality of every system (a property at any size)
    worst = 0.0
    for g, A, b, bw in zip(geoms, A0, B0, Bs):
        x = bw[:g.n]
        r = b - A @ x
        worst = max(worst, float(torch.linalg.norm(A.t() @ r) / (torch.linalg.norm(A) ** 2 * torch.linalg.norm(x))))
    gpu_id = None
    try:
        gpu_id = "GPU-" + str(torch.cuda.get_device_properties(dev).uuid)
    except Exception:
        pass
    clocks = ClockSampler(gpu_id)
    ctqr.profile_reset()
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier(world)
    torch.cuda.synchronize()
    clocks.start()
    reps = []
    e0.record(stream)
    for _ in range(args.steps):
        reps.append(step()[1])
    e1.record(stream)
    torch.cuda.synchronize()
    barrier(world)
    clk = clocks.stop()
    kstats = ctqr.profile_kernels()  # launch counts of the timed steps
    ms = reduce_max(e0.elapsed_time(e1), world, dev)
    value = job_throughput(world, count, args.steps, ms)
    ms_kernel = statistics.median(r.ms for r in reps)
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except OSError:
        pass
    sm_max_ghz = (peaks.get("sm_max_mhz") or 2070.0) / 1e3
    fp64_peak = 152 * 2 * 2 * sm_max_ghz * 1e9 / 1e12
    achieved = flops / (ms_kernel / 1e3) / 1e12
    roof = {"bound": "alu", "achieved": achieved, "peak": fp64_peak, "unit": "TFLOP/s",
            "frac": achieved / fp64_peak, "traffic": None, "kernel": "tile_runtime",
            "peak_source": "derived: 152 SMs x 2 FP64 FMA/clk x 2 x %.2f GHz" % sm_max_ghz,
            "note": "algorithmic flops of Householder QR + Q^T + back-solve per system (2mn^2 - 2n^3/3 + ...)",
            "share_of_step": ms_kernel * args.steps / ms}
    if args.prec != "f64":
        roof.update({"bound": "tensor", "peak": TF32_MEASURED_TFLOPS, "frac": achieved / TF32_MEASURED_TFLOPS,
                     "kernel": "per-system tensor-core factor + FP64 refinement",
                     "peak_source": "measured cuBLAS TF32 (8192^3) on a GB300 of this pool",
                     "note": "algorithmic flops of QR + solve over the wall time of all systems' factor and "
                             "refinement (3xTF32 issues three MMAs per product)"})
    # end to end: systems and right-hand sides from pinned host memory, X back
    Ah = [torch.empty((g.n, g.m + g.n), dtype=torch.float64).pin_memory().t() for g in geoms]
    for h, A in zip(Ah, A0):
        h.copy_(A)
    Bh = [torch.empty((1, g.m + g.n), dtype=torch.float64).pin_memory().t() for g in geoms]
    for h, b in zip(Bh, B0):
        h.copy_(b)
    Xh = [torch.empty((1, g.n), dtype=torch.float64).pin_memory().t() for g in geoms]
    torch.cuda.synchronize()
    barrier(world)
    t0 = time.perf_counter()
    for _ in range(args.e2e_steps):
        for h, Aw, hb, bw in zip(Ah, As, Bh, Bs):
            Aw.copy_(h, non_blocking=True)
            bw.copy_(hb, non_blocking=True)
        ctqr.qr_solve_batched(As, Bs, tile=0, prec=bprec)
        for xh, bw, g in zip(Xh, Bs, geoms):
            xh.copy_(bw[:g.n], non_blocking=True)
        torch.cuda.synchronize()
    t_e2e = reduce_max(time.perf_counter() - t0, world, dev)
    e2e = None
    if args.e2e_steps > 0:
        e2e = {"value": world * count * args.e2e_steps / t_e2e, "unit": "systems/s",
               "h2d_bytes_per_step": sum((g.m + g.n) * (g.n + 1) * 8 for g in geoms),
               "d2h_bytes_per_step": sum(g.n * 8 for g in geoms)}
    line = {"metric": metric, "value": value, "unit": "systems/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64" if args.prec == "f64" else "tf32+f64",
            "data": "synthetic: seeded ellipse phantoms, noiseless b = Ax",
            "config": {"workload": wl, "tile": reps[-1].tile, "tasks": reps[-1].tasks, "prec": args.prec,
                       "refine_iterations_max": reps[-1].iterations,
                       "parallelism": f"replicas x{world}",
                       "l2": "inputs larger than L2 (%.1f GB of FP64 systems)" % (
                           sum((g.m + g.n) * g.n * 8 for g in geoms) / 1e9)},
            "qr_tflops": achieved, "kernel_ms": ms_kernel, "normal_eq_residual_max": worst,
            "roofline": roof, "e2e": e2e, "clocks": clk,
            "gpu_launches": sum(s["launches"] for s in kstats),
            "kernels": {s["name"]: {"launches": s["launches"], "ms": round(s["ms"], 3)}
                        for s in kstats if s["launches"]}}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        t_cpu, cores, desc = oracle_batch_sample(cfg, args.cpu_seconds)
        line["cpu_baseline"] = {"value": count / t_cpu, "unit": "systems/s", "cores": cores, "kind": "oracle",
                                "sample": desc}
    if rank == 0:
        print(json.dumps(line))
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
