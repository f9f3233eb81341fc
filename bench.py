"""Benchmark: QR-based CT reconstruction on one GB300 (arXiv 1907.01891).

One step is one pass of the whole method over one batch of slices: build the
system matrix A on the GPU, factor A = QR, apply Q^T to the batch of
sinograms, back-solve, and (mixed precision) refine with FP64 residuals --
all through ct_reconstruct_scan of the C ABI, with the sinograms already in
HBM.  value = slices reconstructed per second (whole job, all ranks).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--workload NAME] [--prec P]
  python bench.py --impl reference ...   # the plain CPU oracle on the host

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
PREC = {"f64": 0, "f32": 1, "tf32": 2}
DTYPE_NAME = {"f64": "f64", "f32": "f32+f64", "tf32": "tf32+f64"}


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=2)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", choices=["ours", "reference"], default="ours")
    p.add_argument("--workload", choices=sorted(WORKLOADS), default="fan128")
    p.add_argument("--prec", choices=sorted(PREC), default="tf32")
    p.add_argument("--e2e-steps", type=int, default=1)
    p.add_argument("--cpu-seconds", type=float, default=15.0, help="budget of the oracle sample")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--fp64-check", type=int, default=None,
                   help="also run the FP64 QR path once for the relative-error column "
                        "(default: on unless the workload is the 256x256 one, where it takes ~15 min)")
    return p.parse_args()


# DRAM bytes (read + write) of one Cholesky-QR panel launch of 22976 rows x 32
# columns, from the ncu capture summarised in profiles/panel_qr_fan128.md
PANEL_CAPTURE_BYTES, PANEL_CAPTURE_ROWS, PANEL_NB = 3.076e6, 22976, 32


def panel_traffic_per_launch(m, n, nb=PANEL_NB):
    """The captured panel's DRAM bytes scaled by rows to the average panel of
    an m x n factorization (panel j0 has m - j0 rows)."""
    if m <= 0 or n <= 0:
        return None
    rows = [m - j0 for j0 in range(0, n, nb)]
    return PANEL_CAPTURE_BYTES * (sum(rows) / len(rows)) / PANEL_CAPTURE_ROWS


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
def oracle_sample(cfg, k: int, budget_s: float):
    """Time the plain CPU oracle on a bounded sample of the workload and scale
    it (by rays for the build, by flops for QR and solve) to one full step.
    Returns (seconds per full step, cores, description)."""
    from oracle import oracle as O

    g = cfg["geom"]
    m, n = g.m, g.n
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    # (1) system matrix for a subset of the views, scaled by rays
    views = max(1, min(g.n_views, int(g.n_views * min(1.0, 4096.0 / max(m, 1)))))
    gs = O.Geometry(g.beam, g.nx, g.ny, g.pixel, views, g.n_bins, g.angle0,
                    g.angle_span * views / g.n_views, g.src_iso, g.det_span)
    t0 = time.perf_counter()
    As = O.system_matrix(gs)
    t_build = (time.perf_counter() - t0) * (m / gs.m)
    del As
    # (2) QR + Q^T + back-solve of k slices on the first ns columns, full height
    rng = np.random.default_rng(0)
    A = None
    ns = 64
    spent = 0.0
    t_qr_rate = None
    while True:
        A = np.asfortranarray(rng.standard_normal((m, ns)))
        B = np.asfortranarray(rng.standard_normal((m, k)))
        t0 = time.perf_counter()
        F, tau = O.qr(A)
        Y = O.apply_qt(F, tau, B)
        O.backsolve(F, Y)
        dt = time.perf_counter() - t0
        spent += dt
        t_qr_rate = (qr_flops(m, ns) + solve_flops(m, ns, k)) / dt
        if dt > budget_s / 4 or ns >= n or spent > budget_s:
            break
        ns = min(n, int(ns * min(4.0, max(1.5, math.sqrt(budget_s / 3 / max(dt, 1e-3))))))
    t_full = t_build + (qr_flops(m, n) + solve_flops(m, n, k)) / t_qr_rate
    desc = (f"oracle system matrix for {views} of {g.n_views} views (measured, scaled by rays) + "
            f"unblocked Householder QR, Q^T and back-solve of {k} slices on the first {ns} of {n} "
            f"columns at full height m={m} (measured {dt:.1f} s, flop-scaled to n={n})")
    return t_full, cores, desc


# ---------------------------------------------------------------- main
def main():
    args = parse()
    world, rank, local = dist_setup(args)
    cfg = WORKLOADS[args.workload]
    if args.workload == "batch64":
        return main_batch(args, world, rank, local, cfg)
    if args.fp64_check is None:
        args.fp64_check = 0 if args.workload == "fan256" else 1
    g = cfg["geom"]
    k = len(cfg["seeds"])

    if args.impl == "reference":
        if rank != 0:
            return 0
        t_step, cores, desc = oracle_sample(cfg, k, args.cpu_seconds)
        value = k / t_step
        line = {"metric": METRIC, "value": value, "unit": "slices/s", "n_gpus": args.gpus,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_step * 1e3,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
                "data": "synthetic: seeded ellipse phantoms", "impl": "reference",
                "config": {"workload": f"{cfg['name']} ({g.m}x{g.n}, {k} slices)", "prec": "f64",
                           "parallelism": "host cores"},
                "cpu_baseline": {"value": value, "unit": "slices/s", "cores": cores, "kind": "oracle",
                                 "sample": desc},
                "e2e": {"value": value, "unit": "slices/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
        print(json.dumps(line))
        return 0

    import torch
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    from paper_1907_01891_gb300 import ctqr
    ctqr.load()

    # ---- inputs (outside the timed region): phantoms, sinograms B = A x (+ noise)
    lam = cfg.get("lam", 0.0)
    m_sys, n_sys = ctqr.system_size(g, lam)
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

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    # Accuracy: optimality of the (regularized) least-squares solution,
    # ||A^T (b - A x) - lam^2 x|| / (||A||_F^2 ||x||), a property that holds at any
    # size; and, where the FP64 QR path is affordable, the relative error vs it.
    r = B[:g.m] - A @ X
    gres = A.t() @ r - (lam * lam) * X
    normal_eq = float(torch.linalg.norm(gres) / (torch.linalg.norm(A) ** 2 * torch.linalg.norm(X)))
    del r, gres
    rel_err, fp64_qr_tflops = None, None
    if args.fp64_check:
        del A
        torch.cuda.empty_cache()
        X64, rep64 = ctqr.reconstruct_scan(g, B, prec=ctqr.Prec.F64, lam=lam)
        torch.cuda.synchronize()
        rel_err = float(torch.linalg.norm(X - X64) / torch.linalg.norm(X64))
        fp64_qr_tflops = qr_flops(m_sys, n_sys) / (rep64.ms_factor / 1e3) / 1e12
        del X64
    else:
        del A
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
    # Per-kernel device times come from one more step with CUDA events around
    # every launch (outside the timed region: the events add host work).
    ctqr.profile_reset()
    ctqr.profile_enable(True)
    step()
    torch.cuda.synchronize()
    ctqr.profile_enable(False)
    kstats = ctqr.profile_kernels()
    ms = e0.elapsed_time(e1)
    ms_max = reduce_max(ms, world, dev)
    value = job_throughput(world, k, args.steps, ms_max)
    ms_factor = statistics.median(r.ms_factor for r in reps)
    ms_solve = statistics.median(r.ms_solve for r in reps)
    ms_build = statistics.median(r.ms_build for r in reps)

    # ---- roofline of the dominant kernel class
    dom = max(kstats, key=lambda s: s["ms"])
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except OSError:
        pass
    sm_max_ghz = (peaks.get("sm_max_mhz") or 2070.0) / 1e3
    fp64_peak = 152 * 2 * 2 * sm_max_ghz * 1e9 / 1e12      # 2 DFMA/clk/SM (measured 1.204 TF/s)
    fp32_peak = 152 * 128 * 2 * sm_max_ghz * 1e9 / 1e12    # 128 FFMA/clk/SM
    bf16 = peaks.get("bf16_tflops_sustained") or 1705.3
    tf32_peak = bf16 * 1.1 / 2.25
    if dom["name"] in ("zero_fill", "copy", "system_matrix", "tc_update"):
        roof = {"bound": "hbm", "achieved": dom["bytes"] / (dom["ms"] / 1e3) / 1e9,
                "peak": peaks.get("hbm_gbs") or 6809.3, "unit": "GB/s"}
        if dom["name"] == "tc_update":
            roof["note"] = ("C -= V W' streams C (read + write) and the TF32 operands; achieved counts those "
                            "algorithmic bytes; tensor rate %.1f TFLOP/s algorithmic" % (
                                dom["flops"] / (dom["ms"] / 1e3) / 1e12))
    elif dom["name"] == "tc_gemm":
        roof = {"bound": "tensor", "achieved": dom["flops"] / (dom["ms"] / 1e3) / 1e12,
                "peak": tf32_peak, "unit": "TFLOP/s",
                "peak_source": "measured bf16 sustained x nominal tf32/bf16 ratio (1.1/2.25)",
                "note": "achieved counts algorithmic flops 2MNK; 3xTF32 issues 3 MMAs per product"}
    else:
        alu = fp64_peak if args.prec == "f64" or dom["name"] == "panel_qr" else fp32_peak
        roof = {"bound": "alu", "achieved": dom["flops"] / (dom["ms"] / 1e3) / 1e12, "peak": alu,
                "unit": "TFLOP/s",
                "peak_source": "derived: 152 SMs x %s FMA/clk x 2 x %.2f GHz" % (
                    "2 FP64" if alu == fp64_peak else "128 FP32", sm_max_ghz)}
        if dom["name"] == "panel_qr":
            roof["note"] = ("algorithmic flops 3*mr*nbp^2 per panel against the FP64 peak; the Gram matrix and "
                            "the row solves run as compensated FP32 products, the 32x32 Cholesky, inverses and "
                            "modified LU in FP64 (dependent steps: latency-bound)")
    roof["frac"] = roof["achieved"] / roof["peak"]
    roof["kernel"] = dom["name"]
    roof["launches_per_step"] = dom["launches"]
    roof["share_of_step"] = dom["ms"] / (ms / args.steps)
    roof["timed_in"] = "one extra step with CUDA events around every launch of the class"
    roof["traffic"] = None
    if dom["name"] == "panel_qr" and args.prec != "f64":
        t = panel_traffic_per_launch(m_sys, n_sys)
        if t is not None:
            roof["traffic"] = t
            roof["traffic_source"] = ("ncu capture of one 22976-row panel (dram read + write %.3g MB, "
                                      "profiles/panel_qr_fan128.md) scaled by rows to this step's average panel"
                                      % (PANEL_CAPTURE_BYTES / 1e6))

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
            "rel_err_vs_fp64_qr": rel_err,
            "normal_eq_residual": normal_eq,
            "refine_iterations": reps[-1].iterations,
            "fp64_qr_tflops": fp64_qr_tflops,
            "roofline": roof, "e2e": e2e, "clocks": clk, "gpu_launches": launches,
            "kernels": {s["name"]: {"launches": s["launches"], "ms": round(s["ms"], 3)}
                        for s in kstats if s["launches"]}}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        t_cpu, cores, desc = oracle_sample(cfg, k, args.cpu_seconds)
        line["cpu_baseline"] = {"value": k / t_cpu, "unit": "slices/s", "cores": cores, "kind": "oracle",
                                "sample": desc}
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
        return ctqr.qr_solve_batched(As, Bs, tile=0)

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
        ctqr.qr_solve_batched(As, Bs, tile=0)
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
            "vs_baseline": None, "dtype": "f64", "data": "synthetic: seeded ellipse phantoms, noiseless b = Ax",
            "config": {"workload": wl, "tile": reps[-1].tile, "tasks": reps[-1].tasks,
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
