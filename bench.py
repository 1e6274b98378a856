#!/usr/bin/env python3
"""Helmholtz right-hand sides solved per second to 1e-6 relative residual:
CNN-FGMRES against MG-FGMRES on one GPU.

Default workload (``--workload cnn``): the encoder-solver preconditioned solve
of Sec. 3.4 (Eq. 3.14) on a 1024x512 seeded layered medium (h = 12.5 m,
32-cell absorbing layer on the left, right and bottom), 128 point sources on
row 2 at 8 Hz.  Set-up, not timed: the network (widths 16/32/64/128, seeded
He initialisation) is trained on this medium by Alg. 2 (Eq. 4.3 data from
Gaussian x, Adam on Eq. 4.2) for ``--train-steps`` steps.  One step: the
per-medium set-up (medium upload, Galerkin multigrid hierarchy, encoder
context features) followed by FGMRES(10) until every right-hand side reaches
||b - H x|| <= 1e-6 ||b|| in FP64.  ``value`` is CNN-FGMRES; the MG-FGMRES
arm (shifted-Laplacian V-cycle alone) runs on the same batch in the same
process and is reported beside it.

``--workload mg``: the batched MG-FGMRES solve on a 512x256 medium with 64
sources at 3, 4.5 and 6 Hz (192 right-hand sides).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--workload cnn|mg] [--train-steps T]

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
CHECKPOINT = os.path.join(ROOT, "paper_2405_17696_gb300", "weights", "encoder_solver_1024x512_8hz.ckpt")
UNIT = "RHS/s"
TOL = 1e-6
FALLBACK_HBM_GBS = 6800.0
FALLBACK_BF16_TFLOPS = 1900.0
FALLBACK_BF16_TFLOPS_SUSTAINED = 1700.0


def peaks(sustained: bool = False):
    """(HBM GB/s, BF16 TFLOP/s, source) from the measured peaks file, else the fallback.
    sustained: the BF16 figure of a seconds-long GEMM loop (for kernels timed inside a
    long step) instead of the burst figure (for a kernel timed alone)."""
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        key = "bf16_tflops_sustained" if sustained and "bf16_tflops_sustained" in d else "bf16_tflops"
        return float(d["hbm_gbs"]), float(d.get(key, FALLBACK_BF16_TFLOPS)), f"{key} of measured"
    except Exception:
        return FALLBACK_HBM_GBS, FALLBACK_BF16_TFLOPS_SUSTAINED if sustained else FALLBACK_BF16_TFLOPS, "fallback"


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
def _oracle_worker(job):
    """One host process of the CPU baseline: its own sparse LU factorisation of H
    (SuperLU, FP64) and the back-solves of its share of the batch.  Returns
    (factorisation seconds, back-solve seconds, RHS solved)."""
    kappa, gamma, omega, h, rhs = job
    from oracle import helmholtz as H
    t0 = time.perf_counter()
    solver = H.DirectSolver(kappa, gamma, omega, h, h)
    t1 = time.perf_counter()
    solver.solve(rhs)
    return t1 - t0, time.perf_counter() - t1, int(rhs.shape[0])


def _host_memory_bytes():
    """Memory this process may use: MemAvailable, capped by a cgroup limit if one is set."""
    avail = None
    try:
        for line in open("/proc/meminfo"):
            if line.startswith("MemAvailable:"):
                avail = int(line.split()[1]) * 1024
    except OSError:
        pass
    for path in ("/sys/fs/cgroup/memory.max", "/sys/fs/cgroup/memory/memory.limit_in_bytes"):
        try:
            v = open(path).read().strip()
            if v.isdigit():
                avail = min(avail, int(v)) if avail else int(v)
        except OSError:
            pass
    return avail


class OraclePool:
    """The CPU oracle on the host cores: a pool of spawned processes (spawned, so that a
    pool started after CUDA work is safe), one per core up to what memory allows
    (a SuperLU factorisation of the 1024x512 operator peaks near 3.5 GB).  A sample
    solves the whole batch of one frequency: the RHS are split over the workers, each
    of which factors H itself and back-solves its share, so that the wall time is one
    factorisation plus B / workers back-solves."""

    PEAK_BYTES_PER_WORKER = 5 * 1024 ** 3

    def __init__(self, max_workers=None):
        import multiprocessing as mp
        ncores = os.cpu_count() or 1
        mem = _host_memory_bytes()
        by_mem = max(1, int(mem // self.PEAK_BYTES_PER_WORKER)) if mem else 1
        self.workers = max(1, min(ncores, by_mem, max_workers or ncores))
        self.nproc = ncores
        # one BLAS thread per worker process: the workers already fill the cores, and
        # oversubscribed BLAS thread pools spin against each other
        keys = ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")
        saved = {k: os.environ.get(k) for k in keys}
        os.environ.update({k: "1" for k in keys})
        try:
            self.pool = mp.get_context("spawn").Pool(self.workers)
        finally:
            for k, v in saved.items():
                if v is None:
                    os.environ.pop(k, None)
                else:
                    os.environ[k] = v

    def sample(self, w, rhs_sel=None):
        """(RHS solved, wall seconds, mean factorisation seconds, max back-solve seconds)
        for the batch of the workload's last frequency."""
        j = len(w.freqs_hz) - 1
        rhs = w.rhs()[w.freq_index() == j]
        if rhs_sel is not None:
            rhs = rhs[:rhs_sel]
        parts = [p for p in np.array_split(rhs, self.workers) if p.shape[0] > 0]
        kap, gam = w.kappa.astype(np.float64), w.gamma.astype(np.float64)
        om = float(np.float32(w.omegas[j]))
        t0 = time.perf_counter()
        res = self.pool.map(_oracle_worker, [(kap, gam, om, w.h, p) for p in parts])
        wall = time.perf_counter() - t0
        return (sum(r[2] for r in res), wall, float(np.mean([r[0] for r in res])), max(r[1] for r in res))

    def close(self):
        self.pool.close()
        self.pool.join()


def oracle_desc(w, pool, n):
    return (f"direct sparse LU (SuperLU, FP64) of the {w.freqs_hz[-1]:g} Hz {w.nx}x{w.nz} operator and the "
            f"back-solves of {n} RHS (the whole batch of that frequency) over {pool.workers} spawned processes "
            f"of {pool.nproc} host cores; each process factors H itself and back-solves its share")


def cpu_baseline_of(w):
    """One timed sample of the CPU oracle on all host cores (run on rank 0 at N = 1)."""
    pool = OraclePool()
    try:
        pool.sample(w, rhs_sel=pool.workers)      # warm the workers' imports
        n, wall, fact, solve = pool.sample(w)
    finally:
        pool.close()
    return {"value": n / wall, "unit": UNIT, "cores": pool.workers, "nproc": pool.nproc, "kind": "oracle",
            "sample": oracle_desc(w, pool, n),
            "without_factorisation": {"value": n / solve, "unit": UNIT},
            "factorisation_s": fact}


def oracle_workload(workload):
    return media.workload_cnn() if workload in ("cnn", "net") else media.workload_batched()


def run_reference(args, rank, world):
    if rank != 0:
        return
    w = oracle_workload(args.workload)
    pool = OraclePool()
    try:
        for _ in range(min(args.warmup, 1)):   # the host path needs one warm-up (worker imports)
            pool.sample(w)
        n_tot, t_tot, s_tot = 0, 0.0, 0.0
        for _ in range(args.steps):
            n, t, _, s = pool.sample(w)
            n_tot += n
            t_tot += t
            s_tot += s
    finally:
        pool.close()
    value = n_tot / t_tot
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t_tot / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": config_of(w, args.workload),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": pool.workers, "nproc": pool.nproc, "kind": "oracle",
                         "sample": oracle_desc(w, pool, n_tot // max(args.steps, 1)),
                         "without_factorisation": {"value": n_tot / s_tot, "unit": UNIT}},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def config_of(w, workload):
    cfg = {"workload": w.name, "nx": w.nx, "nz": w.nz, "h_m": w.h, "freqs_hz": w.freqs_hz,
           "n_sources": len(w.positions), "n_rhs": len(w.positions) * len(w.freqs_hz),
           "medium": "seeded 12-layer model, 1.5-4.5 km/s, smoothed N(0, 0.1) km/s noise, 32-cell absorbing layer",
           "multigrid": "shifted-Laplacian V-cycle (Galerkin, 3 levels, 2+2 damped Jacobi, coarse GMRES(10))",
           "krylov": "FGMRES(10), complex64 vectors, FP64 Hessenberg/Givens/residual, complex128 iterate",
           "tol": TOL, "parallelism": "independent replicas per GPU",
           "restart_cycles": "CUDA graph replay (MG-FGMRES)"}
    if workload in ("cnn", "net"):
        cfg["precond"] = ("CNN-FGMRES: M_VU(r) = a e0 + V(r - a H e0), a minimising ||r - a H e0||, "
                          "e0 = encoder-solver U-Net (16/32/64/128, BF16)")
        cfg["l2"] = "inputs larger than L2 (537 MB RHS batch, 6 GB Krylov workspace)"
    else:
        cfg["precond"] = "MG-FGMRES"
        cfg["l2"] = "inputs larger than L2 (201 MB RHS batch, 4.6 GB Krylov workspace)"
    return cfg


# --------------------------------------------------------------------------
# our arm
# --------------------------------------------------------------------------
class Problem:
    """Device copies of one workload's inputs and the solve step through the C ABI."""

    def __init__(self, native, w, dev):
        import torch
        self.native, self.w = native, w
        self.nb = len(w.positions) * len(w.freqs_hz)
        self.kappa = torch.from_numpy(w.kappa).to(dev)
        self.gamma = torch.from_numpy(w.gamma).to(dev)
        self.omegas = torch.from_numpy(np.asarray(w.omegas, dtype=np.float32)).to(dev)
        self.rhs_host = w.rhs()
        self.rhs = torch.from_numpy(self.rhs_host).to(dev)
        self.fi = w.freq_index()
        self.x = torch.empty((self.nb, w.nz, w.nx), dtype=torch.complex128, device=dev)
        self.iters = []
        self.solved = []   # RHS per step that reached the tolerance

    def step(self, ctx, rhs=None, x=None, kappa=None, gamma=None, om=None):
        n = self.native
        n.helm_set_medium(ctx, self.kappa if kappa is None else kappa, self.gamma if gamma is None else gamma,
                          self.omegas if om is None else om)
        st, iters, rel, stat = n.helm_solve(ctx, self.rhs if rhs is None else rhs, self.x if x is None else x,
                                            self.nb, self.fi, TOL, n.HELM_SOLVE_ZERO_X0)
        if st not in (n.HELM_OK, n.HELM_ENOCONV):
            raise RuntimeError(f"solve failed: status {st}, per-RHS {np.unique(stat)}, "
                               f"iterations {iters.min()}-{iters.max()}, max rel. residual {rel.max():.3e}")
        # an RHS that hits the iteration cap is not counted as solved
        self.iters.append(iters.copy())
        self.solved.append(int(np.count_nonzero(np.asarray(stat) == n.HELM_OK)))
        return rel


def reduce_over_ranks(ms, solved, world, device="cpu"):
    """Whole-job figures of a timed region: the slowest rank's milliseconds and the
    RHS that reached the tolerance on all ranks together (all-reduce MAX and SUM over
    the default process group when world > 1)."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    n = torch.tensor([float(solved)], dtype=torch.float64, device=device)
    if world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        dist.all_reduce(n, op=dist.ReduceOp.SUM)
    return float(t.item()), int(n.item())


def timed(prob, ctx, steps, warmup, dev, world, stream, sampler=None):
    """Device time (ms, max over ranks) of `steps` solve steps after `warmup`, with
    a barrier and a synchronize on both sides; per-RHS iterations and residuals."""
    import torch
    import torch.distributed as dist
    from paper_2405_17696_gb300 import native
    for _ in range(max(warmup, 0)):
        prob.step(ctx)
    torch.cuda.synchronize(dev)
    if sampler:
        sampler.start()
        time.sleep(0.3)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize(dev)
    launches0 = native.helm_launch_count()
    prob.iters.clear()
    prob.solved.clear()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    rels = [prob.step(ctx) for _ in range(steps)]
    ev1.record(stream)
    torch.cuda.synchronize(dev)
    if world > 1:
        dist.barrier()
    launches = native.helm_launch_count() - launches0
    clocks = sampler.stop() if sampler else None
    its = np.concatenate(prob.iters)
    # slowest rank's time; RHS that reached the tolerance in the timed steps, summed over ranks
    ms, timed.solved = reduce_over_ranks(ev0.elapsed_time(ev1), sum(prob.solved), world, dev)
    return ms, its, float(max(np.max(r) for r in rels)), launches, clocks


def e2e_of(prob, ctx, steps, dev):
    """The same solve through the C ABI from pinned host buffers (copies inside)."""
    import torch
    w = prob.w
    rhs_pin = torch.from_numpy(prob.rhs_host).pin_memory()
    x_pin = torch.empty((prob.nb, w.nz, w.nx), dtype=torch.complex128).pin_memory()
    k_pin = torch.from_numpy(w.kappa).pin_memory()
    g_pin = torch.from_numpy(w.gamma).pin_memory()
    o_pin = torch.from_numpy(np.asarray(w.omegas, dtype=np.float32)).pin_memory()
    args = dict(rhs=rhs_pin, x=x_pin, kappa=k_pin, gamma=g_pin, om=o_pin)
    prob.step(ctx, **args)   # warm the staging path
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    for _ in range(steps):
        prob.step(ctx, **args)
    torch.cuda.synchronize(dev)
    sec = (time.perf_counter() - t0) / steps
    solved = sum(prob.solved[-steps:]) / steps   # RHS per step that reached the tolerance
    h2d = rhs_pin.numel() * 8 + (k_pin.numel() + g_pin.numel() + o_pin.numel()) * 4 + prob.nb * 4
    d2h = x_pin.numel() * 16
    return {"value": solved / sec, "unit": UNIT, "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h)}


def autotune_of(native, ctx, nb, on):
    """Set-up (untimed): the fastest tiling of every convolution shape, timed on the GPU."""
    if not on:
        return None
    t0 = time.perf_counter()
    n = native.cnn_autotune(ctx, nb)
    return {"shapes": n, "seconds": round(time.perf_counter() - t0, 3)}


def profile_step(native, prob, ctx):
    native.helm_profile_enable(ctx, True)
    prob.step(ctx)
    prof = native.helm_profile_read(ctx)
    flops = native.helm_profile_flops(ctx)
    native.helm_profile_enable(ctx, False)
    return prof, flops


def kernel_table(prof, flops):
    total = sum(v[0] for v in prof.values())
    out = {}
    for k, v in sorted(prof.items(), key=lambda kv: -kv[1][0]):
        if v[1] <= 0:
            continue
        e = {"ms": round(v[0], 3), "share": round(v[0] / total, 4) if total else 0.0, "launches": v[1],
             "GBps": round(v[2] / (v[0] / 1e3) / 1e9, 1) if v[0] > 0 and v[2] > 0 else None}
        if flops.get(k, 0.0) > 0 and v[0] > 0:
            e["TFLOPs"] = round(flops[k] / (v[0] / 1e3) / 1e12, 2)
        out[k] = e
    return out


def roofline_of(prof, flops):
    """Roofline of the dominant kernel class: algorithmic bytes (or flops) per
    launch over the class's average CUDA-event launch time.  The class is timed
    inside a whole solve step, so its tensor companion takes the sustained BF16 peak."""
    hbm, bf16, kind = peaks(sustained=True)
    name, (kms, kl, kbytes) = max(prof.items(), key=lambda kv: kv[1][0])
    secs = kms / 1e3
    r = {"bound": "hbm", "kernel": name, "achieved": kbytes / secs / 1e9 if secs > 0 else 0.0, "peak": hbm,
         "unit": "GB/s", "peak_source": "hbm_gbs of " + ("measured" if "measured" in kind else "fallback"),
         "launches": kl,
         "avg_launch_us": 1e3 * kms / max(kl, 1), "algorithmic_bytes_per_launch": kbytes / max(kl, 1),
         "traffic": traffic_from_profiles(name)}
    r["frac"] = r["achieved"] / r["peak"]
    fl = flops.get(name, 0.0)
    if fl > 0 and secs > 0:
        r["tensor"] = {"achieved": fl / secs / 1e12, "peak": bf16, "unit": "TFLOP/s",
                       "frac": fl / secs / 1e12 / bf16, "peak_source": kind,
                       "algorithmic_flops_per_launch": fl / max(kl, 1)}
    return r


def run_retrain_series(args, native, dev, stream, world, rank):
    """CNN-FGMRES iterations along the medium path m_t (t = 0..8, Gaussian-smoothed to true,
    a stand-in for the models an FWI visits) on the 1024x512, 8 Hz batch (every fourth of
    the 128 sources): MG-FGMRES, the network as loaded, and the network retrained by Alg. 2
    for --retrain-steps steps on each m_t (cumulative) before its solve."""
    import torch
    from paper_2405_17696_gb300 import retrain as RT
    w = media.workload_cnn(args.sources_cnn)
    c_true = media.layered_velocity(w.nx, w.nz, seed=media.SEED_MODEL)
    kappas = media.medium_sequence(c_true, 8, 10.0)
    pos = w.positions[::4]
    rhs = torch.from_numpy(media.point_source_rhs(w.nx, w.nz, pos, w.h, w.h)).to(dev)
    nb = rhs.shape[0]
    gam = torch.from_numpy(w.gamma).to(dev)
    om = torch.tensor(w.omegas, dtype=torch.float32, device=dev)
    retrain_steps = args.retrain_steps or 200
    nets = {"cnn_no_retraining": native.cnn_load(args.checkpoint), "cnn_retrained": native.cnn_load(args.checkpoint)}
    rows, t_retrain = [], 0.0
    for t, kap in enumerate(kappas):
        k = torch.from_numpy(kap).to(dev)
        row = {"t": t}
        for label, net in [("mg", None)] + list(nets.items()):
            ctx = native.helm_setup(k, gam, w.nx, w.nz, w.h, w.h, om, net=net, opts=native.helm_default_opts(
                mg_levels=3, max_iter=1000, max_rhs=nb, stream=stream.cuda_stream,
                precond=native.HELM_PC_CNN if net else native.HELM_PC_MG))
            try:
                if label == "cnn_retrained" and retrain_steps > 0:
                    t0 = time.perf_counter()
                    RT.retrain(native, net, ctx, cfg=RT.RetrainConfig(
                        initial_size=128, data_epochs=3, epochs=1 << 20, batch=16, lr=args.retrain_lr,
                        max_steps=retrain_steps, relative_loss=True, warmup_steps=50,
                        seed=media.SEED_DATAGEN + 100 * t))
                    torch.cuda.synchronize(dev)
                    t_retrain += time.perf_counter() - t0
                x = torch.zeros(rhs.shape, dtype=torch.complex128, device=dev)
                _, it, rel, _ = native.helm_solve(ctx, rhs, x, nb, None, TOL, native.HELM_SOLVE_ZERO_X0)
                row[label] = {"mean": float(it.mean()), "max": int(it.max()), "max_rel_residual": float(rel.max())}
            finally:
                native.helm_destroy(ctx)
        rows.append(row)
        print(json.dumps(row), file=sys.stderr, flush=True)
    for net in nets.values():
        native.cnn_destroy(net)
    tot = {k: sum(r[k]["mean"] for r in rows) * nb for k in ("mg", "cnn_no_retraining", "cnn_retrained")}
    line = {"metric": "CNN-FGMRES iterations to 1e-6 along a medium sequence, with and without Alg. 2 retraining",
            "value": tot["cnn_retrained"], "unit": "total FGMRES iterations", "higher_is_better": False,
            "n_gpus": world, "data": "synthetic",
            "config": {"workload": f"retraining_series_{w.nx}x{w.nz}_{nb}rhs_9media", "freq_hz": 8.0,
                       "media": "m_t = (1 - t/8) G_10(m_true) + (t/8) m_true, t = 0..8 (seeded 12-layer m_true)",
                       "retrain_steps_per_medium": retrain_steps, "retrain_lr": args.retrain_lr,
                       "initial_weights": os.path.relpath(args.checkpoint, ROOT)},
            "totals": tot, "retrain_seconds": t_retrain, "per_medium": rows}
    if rank == 0:
        print(json.dumps(line), flush=True)


def run_train(args, native, dev, stream, world, rank, sampler):
    """Alg. 2 training steps per second (cnn_retrain_step: a batch of 16 Eq. 4.3 pairs through
    the network's forward and backward pass and Adam) on the 1024x512, 8 Hz medium, after
    the 128-pair dataset is built; the roofline of the tensor-core weight gradient beside it."""
    import torch
    w = media.workload_cnn(16)
    kap = torch.from_numpy(w.kappa).to(dev)
    gam = torch.from_numpy(w.gamma).to(dev)
    om = torch.tensor(w.omegas, dtype=torch.float32, device=dev)
    net = native.cnn_create(4, (16, 32, 64, 128), seed=media.SEED_CNN)
    ctx = native.helm_setup(kap, gam, w.nx, w.nz, w.h, w.h, om, net=net, opts=native.helm_default_opts(
        mg_levels=3, max_rhs=16, precond=native.HELM_PC_CNN, stream=stream.cuda_stream))
    native.cnn_set_loss(net, 1)
    # 64 steps per epoch once the dataset holds 1024 pairs: warm up into the full dataset first
    native.cnn_retrain_begin(ctx, initial_size=128, data_epochs=3, epochs=1 << 20, seed=media.SEED_DATAGEN)
    for _ in range(56 + max(args.warmup, 3)):
        native.cnn_retrain_step(net, ctx, 16, 1e-4)
    torch.cuda.synchronize(dev)
    steps = args.steps
    st0 = native.cnn_retrain_state(ctx)
    sampler.start()
    time.sleep(0.3)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    launches0 = native.helm_launch_count()
    t0 = time.perf_counter()
    ev0.record(stream)
    for _ in range(steps):
        native.cnn_retrain_step(net, ctx, 16, 1e-4)
    ev1.record(stream)
    torch.cuda.synchronize(dev)
    wall = time.perf_counter() - t0
    clocks = sampler.stop()
    ms = ev0.elapsed_time(ev1)
    launches = native.helm_launch_count() - launches0
    line = {"metric": "Alg. 2 training steps per second (batch 16, 1024x512, 8 Hz)", "value": steps / (ms / 1e3),
            "unit": "steps/s", "n_gpus": world, "steps": steps, "warmup": args.warmup, "ms_per_step": ms / steps,
            "wall_ms_per_step": 1e3 * wall / steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "bf16 network (fp32 accumulate, fp32 master weights)", "data": "synthetic",
            "config": {"workload": "retrain_step_1024x512_batch16", "widths": [16, 32, 64, 128],
                       "dataset_pairs": st0["size"], "loss": "Eq. 4.2 with each pair weighted by 1 / ||e||^2"},
            "gpu_launches": int(launches), "clocks": clocks}
    if not args.no_extras:
        native.helm_profile_enable(ctx, True)
        native.cnn_retrain_step(net, ctx, 16, 1e-4)
        prof = native.helm_profile_read(ctx)
        flops = native.helm_profile_flops(ctx)
        native.helm_profile_enable(ctx, False)
        line["kernels"] = kernel_table(prof, flops)
        hbm, bf16, kind = peaks(sustained=True)
        if "wgrad" in prof and prof["wgrad"][0] > 0:
            kms, kl, kb = prof["wgrad"]
            secs = kms / 1e3
            line["wgrad_roofline"] = {"bound": "tensor", "achieved": flops.get("wgrad", 0.0) / secs / 1e12,
                                      "peak": bf16, "unit": "TFLOP/s", "peak_source": kind,
                                      "frac": flops.get("wgrad", 0.0) / secs / 1e12 / bf16,
                                      "hbm_GBps": kb / secs / 1e9, "hbm_frac": kb / secs / 1e9 / hbm,
                                      "launches": kl, "avg_launch_us": 1e3 * kms / max(kl, 1)}
    native.helm_destroy(ctx)
    native.cnn_destroy(net)
    if rank == 0:
        print(json.dumps(line), flush=True)


def run_fwi_c5(args, native, dev, stream, world, rank):
    """FWI misfit and adjoint-state gradient (Eq. 3.5, Sec. 4.3) on the 2048 x 1024 (h = 10 m)
    fault-and-salt model: 256 sources and 512 receivers on row 2, 8 frequencies in
    [2.5, 10] Hz, each on its own grid of about ten points per 1.5 km/s wavelength (sizes
    multiples of 16).  Set-up (untimed): observed data from the true model on every grid.
    Timed: misfit and gradient at the Gaussian-smoothed starting model, the eight
    frequency contexts solved concurrently (one host thread each, own streams)."""
    import threading
    import torch
    from paper_2405_17696_gb300 import fwi as FWI
    nx0, nz0, h0 = 2048, 1024, 10.0
    c_true = media.fault_salt_velocity(nx0, nz0, seed=media.SEED_MODEL)
    c_init = media.gaussian_smooth(c_true, 10.0)
    k_true0 = torch.from_numpy(media.kappa_of(c_true)).to(dev)
    k_init0 = torch.from_numpy(media.kappa_of(c_init)).to(dev)
    freqs = [float(f) for f in np.linspace(2.5, 10.0, 8)]
    lx, lz = nx0 * h0, nz0 * h0
    ctxs, items = [], []
    t_setup = time.perf_counter()
    for f in freqs:
        nx, nz, hx, hz = FWI.window_grid_size(lx, lz, f)
        kt = torch.empty((nz, nx), dtype=torch.float32, device=dev)
        ki = torch.empty((nz, nx), dtype=torch.float32, device=dev)
        native.helm_resample(k_true0, nx0, nz0, kt, nx, nz)
        native.helm_resample(k_init0, nx0, nz0, ki, nx, nz)
        gam = torch.from_numpy(media.abl_gamma(nx, nz, max(8, int(round(320.0 / hx))))).to(dev)
        src = [2 * nx + int(round((s + 0.5) * nx / 256)) for s in range(256)]
        rcv = [2 * nx + int(round((r + 0.5) * nx / 512)) for r in range(512)]
        st = torch.cuda.Stream(dev)
        om = torch.tensor([2 * math.pi * f], dtype=torch.float32, device=dev)
        ctx = native.helm_setup(kt, gam, nx, nz, hx, hz, om, opts=native.helm_default_opts(
            mg_levels=3, max_iter=2000, max_rhs=128, stream=st.cuda_stream))
        ctxs.append(ctx)
        sv = native.Survey(src, rcv)
        d = torch.zeros((1, len(src), len(rcv)), dtype=torch.complex64, device=dev)
        native.fwi_forward_data(ctx, sv, d, tol=TOL)
        native.helm_set_medium(ctx, ki, gam, om)
        items.append({"f": f, "grid": [nx, nz], "h": [hx, hz], "ctx": ctx, "sv": sv, "d": d,
                      "g": torch.zeros((nz, nx), dtype=torch.float32, device=dev), "om": om, "gam": gam})
    torch.cuda.synchronize(dev)
    t_setup = time.perf_counter() - t_setup
    results = [None] * len(items)
    errors = [None] * len(items)

    def work(i):
        it = items[i]
        torch.cuda.set_device(dev)
        try:
            results[i] = native.fwi_misfit_grad(it["ctx"], it["sv"].src, it["sv"].rcv, it["d"], it["g"], tol=TOL)
        except Exception as e:      # re-raised on the main thread
            errors[i] = e

    for _ in range(max(0, min(args.warmup, 1))):
        for i in range(len(items)):
            work(i)
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    threads = [threading.Thread(target=work, args=(i,)) for i in range(len(items))]
    for th in threads:
        th.start()
    for th in threads:
        th.join()
    torch.cuda.synchronize(dev)
    secs = time.perf_counter() - t0
    for e in errors:
        if e is not None:
            raise e
    # the gradient against the oracle on a 64 x 32 crop of the model (3 and 5 Hz, 8 sources)
    from oracle import fwi as OF
    crop_c = c_true[:32, 1000:1064]
    crop_c0 = media.gaussian_smooth(crop_c, 4.0)
    gam_c = media.abl_gamma(64, 32, 8)
    src_c = [(2, 4 + 8 * s) for s in range(8)]
    rcv_c = [2 * 64 + ix for ix in range(1, 64, 2)]
    om_c = [float(np.float32(2 * math.pi * f)) for f in (3.0, 5.0)]
    gc = media.point_source_rhs(64, 32, src_c, h0, h0)
    k_c = media.kappa_of(crop_c).astype(np.float64)
    k_c0 = media.kappa_of(crop_c0)
    d_c, _ = OF.forward_data(k_c, gam_c.astype(np.float64), om_c, h0, h0, gc, np.array(rcv_c))
    _, g_ref = OF.misfit_and_gradient(k_c0.astype(np.float64), gam_c.astype(np.float64), om_c, h0, h0, gc,
                                      np.array(rcv_c), d_c)
    ctx_c = native.helm_setup(torch.from_numpy(k_c0).to(dev), torch.from_numpy(gam_c).to(dev), 64, 32, h0, h0,
                              torch.tensor(om_c, dtype=torch.float32, device=dev),
                              opts=native.helm_default_opts(mg_levels=3))
    g_gpu = np.zeros((32, 64), np.float32)
    native.fwi_misfit_grad(ctx_c, [iz * 64 + ix for iz, ix in src_c], rcv_c,
                           np.ascontiguousarray(d_c, np.complex64), g_gpu, tol=1e-8)
    native.helm_destroy(ctx_c)
    crop_err = float(np.linalg.norm(g_gpu - g_ref) / np.linalg.norm(g_ref))
    for c in ctxs:
        native.helm_destroy(c)
    line = {"metric": "FWI misfit + adjoint-state gradient, 8 frequencies x 256 sources, seconds", "value": secs,
            "unit": "s", "higher_is_better": False, "n_gpus": world, "data": "synthetic", "dtype": "c64/f64",
            "config": {"workload": "fwi_misfit_grad_2048x1024_256src_512rcv_8freq",
                       "model": "seeded 12-layer model, 3 fault offsets, 4.5 km/s salt ellipse; start: Gaussian "
                                "smoothing (10 cells)",
                       "grids": [{"f_hz": round(it["f"], 3), "grid": it["grid"], "h_m": [round(v, 2) for v in it["h"]]}
                                 for it in items],
                       "solver": "MG-FGMRES to 1e-6 (forward and conjugated adjoint solves), contexts concurrent",
                       "tol": TOL},
            "misfit": float(sum(results)), "setup_seconds": t_setup,
            "rhs_solved": 2 * 256 * len(items),
            "gradient_rel_error_vs_oracle_64x32_crop": crop_err}
    if rank == 0:
        print(json.dumps(line), flush=True)


def run_ours(args, rank, world):
    import torch
    from paper_2405_17696_gb300 import native, retrain as RT

    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    native.cnn_set_conv_path(args.conv_path)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)
    sampler = ClockSampler(local)

    if args.workload == "train":
        run_train(args, native, dev, stream, world, rank, sampler)
        return
    if args.workload == "retrain":
        run_retrain_series(args, native, dev, stream, world, rank)
        return
    if args.workload == "fwi":
        run_fwi_c5(args, native, dev, stream, world, rank)
        return

    if args.workload == "net":
        # the encoder-solver network alone: one forward pass (solver U-Net, contexts
        # cached) of every RHS per step, with He-initialised weights
        w = media.workload_cnn(args.sources_cnn)
        prob = Problem(native, w, dev)
        widths = (16, 32, 64, 128)
        net = native.cnn_create(len(widths), widths)
        native.cnn_init_params(net, media.SEED_CNN, 0.5)
        ctx = native.helm_setup(prob.kappa, prob.gamma, w.nx, w.nz, w.h, w.h, prob.omegas, net=net,
                                opts=native.helm_default_opts(mg_levels=3, max_rhs=prob.nb,
                                                              precond=native.HELM_PC_CNN, stream=stream.cuda_stream))
        tune = autotune_of(native, ctx, prob.nb, args.autotune)
        r = prob.rhs.to(torch.complex64) if prob.rhs.dtype != torch.complex64 else prob.rhs
        e = torch.empty_like(r)
        for _ in range(max(args.warmup, 0)):
            native.cnn_precond_apply(ctx, r, e, prob.nb, prob.fi, 0)
        torch.cuda.synchronize(dev)
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        for _ in range(args.steps):
            native.cnn_precond_apply(ctx, r, e, prob.nb, prob.fi, 0)
        ev1.record(stream)
        torch.cuda.synchronize(dev)
        ms = ev0.elapsed_time(ev1)
        line = {"metric": "encoder-solver network forward passes per second (RHS/s)", "value":
                world * prob.nb * args.steps / (ms / 1e3), "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "bf16 (fp32 accumulate)", "data": "synthetic",
                "config": {"workload": f"network_forward_{w.nx}x{w.nz}_{prob.nb}rhs", "widths": list(widths),
                           "conv_path": args.conv_path}, "autotune": tune}
        if not args.no_extras:
            native.helm_profile_enable(ctx, True)
            native.cnn_precond_apply(ctx, r, e, prob.nb, prob.fi, 0)
            prof = native.helm_profile_read(ctx)
            flops = native.helm_profile_flops(ctx)
            native.helm_profile_enable(ctx, False)
            line["roofline"] = roofline_of(prof, flops)
            line["kernels"] = kernel_table(prof, flops)
        native.helm_destroy(ctx)
        native.cnn_destroy(net)
        if rank == 0:
            print(json.dumps(line), flush=True)
        return

    if args.workload == "mg":
        w = media.workload_batched(args.sources)
        prob = Problem(native, w, dev)
        ctx = native.helm_setup(prob.kappa, prob.gamma, w.nx, w.nz, w.h, w.h, prob.omegas,
                                opts=native.helm_default_opts(mg_levels=3, max_rhs=prob.nb,
                                                              stream=stream.cuda_stream))
        native.helm_set_graphs(ctx, bool(args.graphs))
        ms, its, relmax, launches, clocks = timed(prob, ctx, args.steps, args.warmup, dev, world, stream, sampler)
        value = timed.solved / (ms / 1e3)
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "c64/f64", "data": "synthetic",
                "config": config_of(w, "mg"), "impl": "ours", "precond": "mg",
                "iterations": {"mean": float(its.mean()), "max": int(its.max()), "min": int(its.min())},
                "max_rel_residual": relmax, "unsolved_rhs": world * prob.nb * args.steps - timed.solved,
                "gpu_launches": int(launches), "clocks": clocks}
        if not args.no_extras:
            prof, flops = profile_step(native, prob, ctx)
            line["roofline"] = roofline_of(prof, flops)
            line["kernels"] = kernel_table(prof, flops)
            line["e2e"] = e2e_of(prob, ctx, max(1, min(args.steps, 3)), dev)
            if world == 1:
                line["cpu_baseline"] = cpu_baseline_of(oracle_workload("mg"))
        native.helm_destroy(ctx)
        if rank == 0:
            print(json.dumps(line), flush=True)
        return

    # ---- CNN-FGMRES vs MG-FGMRES, 1024x512, 8 Hz, 128 RHS ----
    w = media.workload_cnn(args.sources_cnn)
    prob = Problem(native, w, dev)
    widths = (16, 32, 64, 128)
    use_ckpt = args.checkpoint and os.path.exists(args.checkpoint) and args.train_steps is None
    if use_ckpt:
        # initial weights trained offline by the library's own Alg. 2 training on other media of
        # the family (paper_2405_17696_gb300.train_checkpoint), as the paper trains its initial
        # weights offline (Sec. 5.2); light Alg. 2 retraining on this medium follows (set-up)
        net = native.cnn_load(args.checkpoint)
        with open(os.path.splitext(args.checkpoint)[0] + ".json") as fh:
            prov = json.load(fh)
    else:
        net = native.cnn_create(len(widths), widths, seed=media.SEED_CNN)
        prov = None
    opts = dict(mg_levels=3, max_rhs=prob.nb, max_iter=1000, stream=stream.cuda_stream)
    ctx_cnn = native.helm_setup(prob.kappa, prob.gamma, w.nx, w.nz, w.h, w.h, prob.omegas, net=net,
                                opts=native.helm_default_opts(precond=native.HELM_PC_CNN, **opts))
    ctx_mg = native.helm_setup(prob.kappa, prob.gamma, w.nx, w.nz, w.h, w.h, prob.omegas,
                               opts=native.helm_default_opts(**opts))
    native.helm_set_graphs(ctx_mg, bool(args.graphs))
    tune = autotune_of(native, ctx_cnn, prob.nb, args.autotune)
    # set-up (not timed): Alg. 2 on this medium
    steps = args.retrain_steps if use_ckpt else (400 if args.train_steps is None else args.train_steps)
    epochs = 3 + max(1, -(-(steps - 56) // 64))
    cfg = RT.RetrainConfig(initial_size=128, data_epochs=3, epochs=epochs, batch=16,
                           lr=1e-4 if use_ckpt else 1e-3, lr_final=1e-4, max_steps=steps,
                           seed=media.SEED_DATAGEN + rank, relative_loss=True, warmup_steps=0 if use_ckpt else 100)
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    hist = RT.retrain(native, net, ctx_cnn, cfg=cfg) if steps > 0 else RT.RetrainHistory()
    torch.cuda.synchronize(dev)
    train_s = time.perf_counter() - t0
    training = {"steps": hist.steps, "seconds": train_s, "batch": 16, "lr": [cfg.lr, cfg.lr_final],
                "loss": "Eq. 4.2 with each pair weighted by 1 / ||e||^2",
                "loss_first_epoch": hist.epoch_loss[0] if hist.epoch_loss else None,
                "loss_last_epoch": hist.epoch_loss[-1] if hist.epoch_loss else None}
    if prov is not None:
        training["initial_weights"] = {"checkpoint": os.path.relpath(args.checkpoint, ROOT),
                                       "offline_steps": prov.get("steps"), "offline_seconds": prov.get("seconds"),
                                       "train_media_seeds": prov.get("train_media_seeds"),
                                       "offline_loss_last_200": prov.get("loss_last_200"),
                                       "benchmark_medium_in_offline_training":
                                           media.SEED_MODEL in (prov.get("train_media_seeds") or [])}

    ms, its, relmax, launches, clocks = timed(prob, ctx_cnn, args.steps, args.warmup, dev, world, stream, sampler)
    solved = timed.solved
    mg_ms, mg_its, mg_rel, _, _ = timed(prob, ctx_mg, args.steps, min(args.warmup, 1), dev, world, stream)
    mg_solved = timed.solved
    value = solved / (ms / 1e3)
    mg_value = mg_solved / (mg_ms / 1e3)
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "c64/f64 solve, bf16 network (fp32 accumulate)", "data": "synthetic",
            "config": config_of(w, "cnn"), "impl": "ours", "precond": "cnn",
            "iterations": {"mean": float(its.mean()), "max": int(its.max()), "min": int(its.min())},
            "max_rel_residual": relmax, "unsolved_rhs": world * prob.nb * args.steps - solved,
            "mg_fgmres": {"value": mg_value, "unit": UNIT, "ms_per_step": mg_ms / args.steps,
                          "unsolved_rhs": world * prob.nb * args.steps - mg_solved,
                          "iterations": {"mean": float(mg_its.mean()), "max": int(mg_its.max()),
                                         "min": int(mg_its.min())}, "max_rel_residual": mg_rel},
            "training": training,
            "autotune": tune, "gpu_launches": int(launches), "clocks": clocks}
    if not args.no_extras:
        prof, flops = profile_step(native, prob, ctx_cnn)
        line["roofline"] = roofline_of(prof, flops)
        line["kernels"] = kernel_table(prof, flops)
        line["e2e"] = e2e_of(prob, ctx_cnn, 1, dev)
        if world == 1:
            line["cpu_baseline"] = cpu_baseline_of(oracle_workload("cnn"))
    native.helm_destroy(ctx_cnn)
    native.helm_destroy(ctx_mg)
    native.cnn_destroy(net)
    if rank == 0:
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
    ap.add_argument("--workload", choices=["cnn", "mg", "net", "train", "retrain", "fwi"], default="cnn",
                    help="cnn: CNN-FGMRES vs MG-FGMRES at 1024x512 (default); mg: MG-FGMRES at 512x256; "
                         "net: the network's forward pass alone at 1024x512; train: Alg. 2 training steps; "
                         "retrain: CNN-FGMRES iterations "
                         "along a medium sequence with and without Alg. 2 retraining; fwi: FWI misfit and "
                         "gradient at 2048x1024 on per-frequency grids")
    ap.add_argument("--train-steps", type=int, default=None,
                    help="train the network from seeded weights for this many Alg. 2 steps instead of loading "
                         "the checkpoint (default: the checkpoint when it exists, else 400 steps)")
    ap.add_argument("--checkpoint", default=CHECKPOINT,
                    help="initial weights (cnn_load) for the cnn workload")
    ap.add_argument("--retrain-lr", type=float, default=1e-5,
                    help="retrain workload: Adam learning rate of the Alg. 2 steps on each medium")
    ap.add_argument("--retrain-steps", type=int, default=0,
                    help="Alg. 2 steps on the benchmark medium after loading the checkpoint (set-up, untimed); "
                         "the retraining series (--workload retrain) uses it per medium (default there: 200)")
    ap.add_argument("--sources", type=int, default=64,
                    help="mg workload: sources per frequency (64 = the benchmark workload)")
    ap.add_argument("--sources-cnn", type=int, default=128,
                    help="cnn workload: sources (128 = the benchmark workload; fewer only for profiling runs)")
    ap.add_argument("--autotune", type=int, default=1, choices=[0, 1],
                    help="time the candidate tilings of every convolution shape before the run (set-up, untimed)")
    ap.add_argument("--graphs", type=int, default=1, choices=[0, 1],
                    help="replay the restart cycles of MG-FGMRES from a CUDA graph (1, default) or launch them one by one")
    ap.add_argument("--conv-path", type=int, default=0, choices=[0, 1, 2, 3],
                    help="convolution kernel: 0 TMA halo tiles (default), 1 gather, 2 TMA with the column "
                         "taps in N for 16-channel layers, 3 TMA with the tap rows in N for "
                         "16- and 32-channel same-grid layers")
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
