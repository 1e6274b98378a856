#!/usr/bin/env python3
"""Helmholtz right-hand sides solved per second to 1e-6 relative residual.

Workload (one step): the batched multi-source, multi-frequency solve of
Sec. 3.1-3.4 on a 512x256 seeded layered medium (h = 20 m, 32-cell absorbing
layer on the left, right and bottom), 64 point sources on row 2 and three
frequencies (3, 4.5, 6 Hz) = 192 right-hand sides in one batched launch
sequence: the per-medium set-up (medium upload + Galerkin multigrid hierarchy
for every frequency) followed by MG-FGMRES(10) with the shifted-Laplacian
V-cycle until every right-hand side reaches ||b - H x|| <= 1e-6 ||b|| in FP64.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line.  Under torchrun (N > 1) every rank solves its own copy
of the batch (independent problems, no collective on the data path: weak
scaling); the time is the max over ranks.  ``--impl reference`` times the CPU
FP64 oracle (sparse direct solve) on the host cores instead.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_2405_17696_gb300 import media  # noqa: E402

METRIC = "Helmholtz RHS solved/sec to 1e-6 rel. residual: CNN-FGMRES vs MG-FGMRES, 1 GB300"
UNIT = "RHS/s"
TOL = 1e-6
FALLBACK_HBM_GBS = 6800.0


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


# --------------------------------------------------------------------------
# clocks sampled with nvidia-smi during the timed region
# --------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "200",
                 "-i", str(self.index)], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.lines:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for name, val in zip(names, parts[4:8]):
                if val.lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# --------------------------------------------------------------------------
# CPU oracle (the reference arm and the cpu_baseline field)
# --------------------------------------------------------------------------
def oracle_sample(w):
    """One bounded sample of the workload on the host: the direct solve of one
    frequency's share (one sparse LU factorisation + 64 back-solves), which is
    one third of the 192-RHS batch.  Returns (RHS solved, seconds)."""
    from oracle import helmholtz as H
    j = len(w.freqs_hz) - 1
    rhs = w.rhs()[w.freq_index() == j]
    t0 = time.perf_counter()
    solver = H.DirectSolver(w.kappa.astype(np.float64), w.gamma.astype(np.float64),
                            float(np.float32(w.omegas[j])), w.h, w.h)
    solver.solve(rhs)
    return rhs.shape[0], time.perf_counter() - t0


SAMPLE_DESC = ("direct sparse LU (SuperLU, FP64) of the 6 Hz operator plus its 64 back-solves: one third "
               "of the 512x256, 192-RHS batch")


def run_reference(args, rank, world):
    if rank != 0:
        return
    w = media.workload_batched()
    for _ in range(args.warmup):
        oracle_sample(w)
    n_tot, t_tot = 0, 0.0
    for _ in range(args.steps):
        n, t = oracle_sample(w)
        n_tot += n
        t_tot += t
    value = n_tot / t_tot
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t_tot / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": config_of(w),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": SAMPLE_DESC},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def config_of(w):
    return {"workload": w.name, "nx": w.nx, "nz": w.nz, "h_m": w.h, "freqs_hz": w.freqs_hz,
            "n_sources": len(w.positions), "n_rhs": len(w.positions) * len(w.freqs_hz),
            "medium": "seeded 12-layer model, 1.5-4.5 km/s, smoothed N(0, 0.1) km/s noise",
            "precond": "shifted-Laplacian V-cycle (Galerkin, 3 levels, 2+2 damped Jacobi, coarse GMRES(10))",
            "krylov": "FGMRES(10), complex64 vectors, FP64 Hessenberg/Givens/residual, complex128 iterate",
            "tol": TOL, "l2": "inputs larger than L2 (201 MB RHS batch, 4.6 GB Krylov workspace)",
            "parallelism": "independent replicas per GPU"}


# --------------------------------------------------------------------------
# our arm
# --------------------------------------------------------------------------
def run_ours(args, rank, world):
    import torch
    import torch.distributed as dist
    from paper_2405_17696_gb300 import native

    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)

    w = media.workload_batched(args.sources)
    nb = len(w.positions) * len(w.freqs_hz)
    kappa = torch.from_numpy(w.kappa).to(dev)
    gamma = torch.from_numpy(w.gamma).to(dev)
    omegas = torch.from_numpy(np.asarray(w.omegas, dtype=np.float32)).to(dev)
    rhs_host = w.rhs()
    rhs = torch.from_numpy(rhs_host).to(dev)
    fi = w.freq_index()
    x = torch.empty((nb, w.nz, w.nx), dtype=torch.complex128, device=dev)
    opts = native.helm_default_opts(mg_levels=3, max_rhs=nb, stream=stream.cuda_stream)
    ctx = native.helm_setup(kappa, gamma, w.nx, w.nz, w.h, w.h, omegas, opts=opts)

    iters_all = []

    def step(rhs_arg, x_arg, kappa_arg, gamma_arg, om_arg):
        native.helm_set_medium(ctx, kappa_arg, gamma_arg, om_arg)
        st, iters, rel, stat = native.helm_solve(ctx, rhs_arg, x_arg, nb, fi, TOL, native.HELM_SOLVE_ZERO_X0)
        if st != native.HELM_OK:
            raise RuntimeError(f"solve did not converge: status {st}, per-RHS {np.unique(stat)}, "
                               f"iterations {iters.min()}-{iters.max()}, max rel. residual {rel.max():.3e}")
        iters_all.append(iters.copy())
        return rel

    for _ in range(max(args.warmup, 0)):
        step(rhs, x, kappa, gamma, omegas)
    torch.cuda.synchronize(dev)

    sampler = ClockSampler(local)
    sampler.start()
    time.sleep(0.3)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize(dev)
    launches0 = native.helm_launch_count()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    iters_all.clear()
    ev0.record(stream)
    rels = []
    for _ in range(args.steps):
        rels.append(step(rhs, x, kappa, gamma, omegas))
    ev1.record(stream)
    torch.cuda.synchronize(dev)
    if world > 1:
        dist.barrier()
    launches = native.helm_launch_count() - launches0
    clocks = sampler.stop()
    ms = ev0.elapsed_time(ev1)
    t = torch.tensor([ms], dtype=torch.float64, device=dev)
    if world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    ms_max = float(t.item())
    value = world * nb * args.steps / (ms_max / 1e3)
    its = np.concatenate(iters_all)

    if args.no_extras:
        native.helm_destroy(ctx)
        if rank == 0:
            print(json.dumps({"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                              "warmup": args.warmup, "ms_per_step": ms_max / args.steps,
                              "config": config_of(w), "note": "timing only (--no-extras)"}), flush=True)
        return

    # one profiled step (per-kernel-class CUDA events + algorithmic bytes)
    native.helm_profile_enable(ctx, True)
    step(rhs, x, kappa, gamma, omegas)
    prof = native.helm_profile_read(ctx)
    native.helm_profile_enable(ctx, False)

    # end to end through the C ABI with host buffers (pinned), copies inside
    rhs_pin = torch.from_numpy(rhs_host).pin_memory()
    x_pin = torch.empty((nb, w.nz, w.nx), dtype=torch.complex128).pin_memory()
    k_pin = torch.from_numpy(w.kappa).pin_memory()
    g_pin = torch.from_numpy(w.gamma).pin_memory()
    o_pin = torch.from_numpy(np.asarray(w.omegas, dtype=np.float32)).pin_memory()
    e2e_steps = max(1, min(args.steps, 3))
    step(rhs_pin, x_pin, k_pin, g_pin, o_pin)          # warm the staging path
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        step(rhs_pin, x_pin, k_pin, g_pin, o_pin)
    torch.cuda.synchronize(dev)
    e2e_s = (time.perf_counter() - t0) / e2e_steps
    h2d = rhs_pin.numel() * 8 + (k_pin.numel() + g_pin.numel() + o_pin.numel()) * 4 + nb * 4
    d2h = x_pin.numel() * 16
    native.helm_destroy(ctx)

    if rank != 0:
        return
    peak, peak_kind = peaks()
    dom = max(prof.items(), key=lambda kv: kv[1][0])
    name, (kms, kl, kbytes) = dom
    achieved = kbytes / (kms / 1e3) / 1e9 if kms > 0 else 0.0
    traffic = traffic_from_profiles(name)
    roofline = {"bound": "hbm", "kernel": name, "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "peak_source": f"hbm_gbs of {peak_kind}",
                "traffic": traffic, "launches": kl, "avg_launch_us": 1e3 * kms / max(kl, 1),
                "algorithmic_bytes_per_launch": kbytes / max(kl, 1)}
    cpu = None
    if world == 1:
        n, tcpu = oracle_sample(w)
        cpu = {"value": n / tcpu, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": SAMPLE_DESC}
    total_ms = sum(v[0] for v in prof.values())
    kernels = {k: {"ms": round(v[0], 3), "share": round(v[0] / total_ms, 4) if total_ms else 0.0,
                   "launches": v[1], "GBps": round(v[2] / (v[0] / 1e3) / 1e9, 1) if v[0] > 0 and v[2] > 0 else None}
               for k, v in sorted(prof.items(), key=lambda kv: -kv[1][0]) if v[1] > 0}
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "c64/f64", "data": "synthetic", "config": config_of(w),
        "impl": "ours", "precond": "mg",
        "iterations": {"mean": float(its.mean()), "max": int(its.max()), "min": int(its.min())},
        "max_rel_residual": float(max(np.max(r) for r in rels)),
        "roofline": roofline, "cpu_baseline": cpu,
        "e2e": {"value": nb / e2e_s, "unit": UNIT, "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h)},
        "gpu_launches": int(launches), "clocks": clocks, "kernels": kernels,
    }
    print(json.dumps(line), flush=True)


def traffic_from_profiles(kernel: str):
    """DRAM bytes per launch of ``kernel`` from a committed ncu summary
    (profiles/<kernel>*.md, a line 'traffic_bytes_per_launch: <n>'), else None."""
    pdir = os.path.join(ROOT, "profiles")
    if not os.path.isdir(pdir):
        return None
    for fn in sorted(os.listdir(pdir)):
        if fn.startswith(kernel) and fn.endswith(".md"):
            for line in open(os.path.join(pdir, fn)):
                if line.strip().startswith("traffic_bytes_per_launch:"):
                    try:
                        return float(line.split(":", 1)[1])
                    except ValueError:
                        return None
    return None


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--sources", type=int, default=64,
                    help="sources per frequency (64 = the benchmark workload; fewer only for profiling runs)")
    ap.add_argument("--no-extras", action="store_true",
                    help="time the solve only: no profiled step, end-to-end leg or CPU baseline (profiling runs)")
    args = ap.parse_args()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
        dist.init_process_group("nccl")
    try:
        run_ours(args, rank, world)
    finally:
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()


if __name__ == "__main__":
    main()
