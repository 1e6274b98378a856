"""Frequency-domain FWI by Gauss-Newton with frequency continuation (Alg. 1,
Sec. 3.2-3.3) and light-weight retraining of the encoder-solver network between
iterations (Alg. 2, Sec. 4.2).

A thin driver over the C ABI: every arithmetic step (the forward, adjoint and
sensitivity solves, the conjugate-gradient iterations of a Gauss-Newton step, the
line search, the retraining) runs in libhelm.  This module sequences the calls:
for each frequency window (low to high) a context with the window's frequencies is
set up on the current model, ``gn_iters`` Gauss-Newton iterations run with a fresh
set of ``sim_sources`` Rademacher-encoded simultaneous sources each (Sec. 3.2;
the random signs are drawn here, seeded, and passed in), and with the network
preconditioner ``retrain_steps`` steps of Alg. 2 follow each iteration on the new
medium.  The paper's figure of merit is the total number of Helmholtz solver
iterations of the whole inversion, with and without retraining (Sec. 5.4).
"""
from __future__ import annotations

import math
import time
from dataclasses import dataclass, field

import numpy as np

from . import media
from . import retrain as RT


@dataclass
class FwiConfig:
    windows: list                   # frequency windows in Hz, low to high (Alg. 1)
    gn_iters: int = 3               # Gauss-Newton iterations per window
    cg_iters: int = 5               # CG steps per Gauss-Newton iteration
    tol: float = 1e-6               # forward / adjoint solves
    tol_sens: float = 1e-4          # sensitivity solves
    sim_sources: int = 16           # Rademacher-encoded sources per iteration (0: every point source)
    retrain_steps: int = 0          # Alg. 2 steps after each iteration (0: no retraining)
    retrain_lr: float = 1e-4
    retrain_initial: int = 32       # pairs of the Eq. 4.3 dataset built on each new medium
    v_min: float = 1400.0           # m/s bounds of the model (m = 1 / v^2)
    v_max: float = 5000.0
    mg_levels: int = 3
    max_rhs: int = 64
    seed: int = media.SEED_SOURCES
    reg_kind: object = 0            # regulariser of Sec. 5.1: 0 none, 1 R_diff, 2 R_high; or one per
                                    # window (e.g. R_high on the first sweeps, then R_diff, Sec. 5.3)
    reg_alpha: object = 0.0         # its weight (or one per window); the reference model is the model
                                    # the run starts from, kept fixed


@dataclass
class FwiHistory:
    rows: list = field(default_factory=list)   # one dict per Gauss-Newton iteration

    @property
    def total_iterations(self) -> int:
        return int(sum(r["iters_forward"] + r["iters_adjoint"] + r["iters_sensitivity"] + r["iters_line_search"]
                       for r in self.rows))


def rademacher(p: int, nsrc: int, rng: np.random.Generator) -> np.ndarray:
    """p x nsrc weights of +-1 (simultaneous sources, Sec. 3.2)."""
    return np.where(rng.random((p, nsrc)) < 0.5, -1.0, 1.0).astype(np.float32)


def observed_data(native, kappa_true, gamma, nx, nz, hx, hz, freqs_hz, survey, mg_levels=3, max_rhs=64, tol=1e-8):
    """Synthetic observed data [nfreq][nsrc][nrcv] of the true model (Eq. 3.3) and the
    Helmholtz iterations it took."""
    import torch
    om = torch.tensor([2 * math.pi * f for f in freqs_hz], dtype=torch.float32, device="cuda")
    ctx = native.helm_setup(torch.as_tensor(kappa_true, dtype=torch.float32, device="cuda").contiguous(),
                            torch.as_tensor(gamma, dtype=torch.float32, device="cuda").contiguous(), nx, nz, hx, hz,
                            om, opts=native.helm_default_opts(mg_levels=mg_levels, max_rhs=max_rhs, max_iter=2000))
    try:
        d = torch.zeros((len(freqs_hz), survey.src.size, survey.rcv.size), dtype=torch.complex64, device="cuda")
        it = native.fwi_forward_data(ctx, survey, d, tol=tol)
    finally:
        native.helm_destroy(ctx)
    return d, it


@dataclass
class WindowGrid:
    """The grid of one frequency window (about ten points per wavelength): its size and
    spacings over the fine grid's rectangle, absorbing layer, source and receiver nodes
    and observed data [nfreq][nsrc][nrcv] (CUDA tensors / arrays on that grid)."""
    freqs: list
    nx: int
    nz: int
    hx: float
    hz: float
    gamma: object
    src_idx: list
    rcv_idx: list
    d_obs: object


def window_grid_size(lx: float, lz: float, fmax_hz: float, c_min: float = 1500.0, ppw: float = 10.0,
                     multiple: int = 16):
    """(nx, nz, hx, hz) of a grid of about ppw points per shortest wavelength c_min / fmax over
    an lx x lz rectangle, sizes rounded to multiples of `multiple` (multigrid and network)."""
    h = c_min / (ppw * fmax_hz)
    nx = max(multiple, int(round(lx / h / multiple)) * multiple)
    nz = max(multiple, int(round(lz / h / multiple)) * multiple)
    return nx, nz, lx / nx, lz / nz


def run_windows(native, m, nx0, nz0, windows, cfg: FwiConfig, net=None, log=None) -> FwiHistory:
    """Alg. 1 with a grid per frequency window: the fine model m (CUDA tensor [nz0][nx0],
    updated in place) is resampled to each window's grid, the window's Gauss-Newton
    iterations update that copy, and the update is resampled back and added to m."""
    import torch
    hist = FwiHistory()
    pick = lambda v, i: v[i] if isinstance(v, (list, tuple)) else v
    m_init = m.clone()   # the regulariser's reference model: the initial guess, on every window's grid
    for wi, win in enumerate(windows):
        same = (win.nx, win.nz) == (nx0, nz0)
        if same:
            mw, m_ref = m, m_init
        else:
            mw = torch.empty((win.nz, win.nx), dtype=torch.float32, device="cuda")
            native.helm_resample(m, nx0, nz0, mw, win.nx, win.nz)
            mw0 = mw.clone()
            m_ref = torch.empty_like(mw)
            native.helm_resample(m_init, nx0, nz0, m_ref, win.nx, win.nz)
        c = FwiConfig(**{**cfg.__dict__, "windows": [win.freqs], "reg_kind": pick(cfg.reg_kind, wi),
                         "reg_alpha": pick(cfg.reg_alpha, wi)})
        h = run(native, mw, win.gamma, win.nx, win.nz, win.hx, win.hz, win.src_idx, win.rcv_idx, win.d_obs,
                win.freqs, c, net=net, log=log, window_offset=wi, m_ref=m_ref)
        hist.rows += h.rows
        if not same:
            native.helm_resample(mw, win.nx, win.nz, m, nx0, nz0, 1.0, 1.0)     # m += R(m_w) - R(m_w0)
            native.helm_resample(mw0, win.nx, win.nz, m, nx0, nz0, -1.0, 1.0)
    return hist


def regulariser_schedule(cfg: FwiConfig):
    """(kinds, weights), one per frequency window, from cfg.reg_kind / cfg.reg_alpha (a value
    for every window, or a list with one per window).  Kinds are 0 (none), 1 (R_diff) or 2
    (R_high) of Sec. 5.1; weights are >= 0.  ValueError otherwise."""
    nwin = len(cfg.windows)
    per_window = lambda v: list(v) if isinstance(v, (list, tuple)) else [v] * nwin
    kinds, alphas = per_window(cfg.reg_kind), per_window(cfg.reg_alpha)
    if len(kinds) != nwin or len(alphas) != nwin:
        raise ValueError("reg_kind / reg_alpha: one value, or one per window")
    if any(int(k) != k or k not in (0, 1, 2) for k in kinds) or any(not (a >= 0) for a in alphas):
        raise ValueError("reg_kind must be 0, 1 or 2 and reg_alpha >= 0")
    return [int(k) for k in kinds], [float(a) for a in alphas]


def run(native, m, gamma, nx, nz, hx, hz, src_idx, rcv_idx, d_obs, freqs_hz, cfg: FwiConfig, net=None,
        log=None, window_offset: int = 0, m_ref=None) -> FwiHistory:
    """Alg. 1 on the model m (float32 CUDA tensor [nz][nx] of m = 1 / v^2, updated in
    place).  d_obs: observed data [nfreq][nsrc][nrcv] (CUDA tensor) at freqs_hz, ordered as
    the windows' frequencies are drawn from.  net: the encoder-solver network (CNN-FGMRES
    with retraining when cfg.retrain_steps > 0), or None for MG-FGMRES.  m_ref: the
    regulariser's reference model on this grid (default: m as the run starts)."""
    kinds, alphas = regulariser_schedule(cfg)
    import torch
    hist = FwiHistory()
    rng = media.rng(cfg.seed)
    gam = torch.as_tensor(gamma, dtype=torch.float32, device="cuda").contiguous()
    fidx = {f: i for i, f in enumerate(freqs_hz)}
    if not any(k and a > 0 for k, a in zip(kinds, alphas)):
        m_ref = None
    elif m_ref is None:
        m_ref = m.clone()
    for wi, window in enumerate(cfg.windows):
        opts = native.fwi_default_gn_opts(tol=cfg.tol, tol_sens=cfg.tol_sens, cg_iters=cfg.cg_iters,
                                          m_min=1.0 / cfg.v_max ** 2, m_max=1.0 / cfg.v_min ** 2,
                                          reg_kind=int(kinds[wi]), alpha=float(alphas[wi]))
        om = torch.tensor([2 * math.pi * f for f in window], dtype=torch.float32, device="cuda")
        dw = torch.stack([d_obs[fidx[f]] for f in window]).contiguous()
        kappa = torch.empty_like(m)
        native.fwi_model_to_kappa(m, kappa)   # the medium the context starts from
        pc = native.HELM_PC_CNN if net is not None else native.HELM_PC_MG
        ctx = native.helm_setup(kappa, gam, nx, nz, hx, hz, om, net=net,
                                opts=native.helm_default_opts(mg_levels=cfg.mg_levels, max_rhs=cfg.max_rhs,
                                                              precond=pc, max_iter=2000))
        try:
            for it in range(cfg.gn_iters):
                nsrc = len(src_idx)
                w = rademacher(cfg.sim_sources, nsrc, rng) if cfg.sim_sources > 0 else None
                survey = native.Survey(src_idx, rcv_idx, w)
                t0 = time.perf_counter()
                info = native.fwi_gn_iteration(ctx, survey, dw, m, opts, m_ref=m_ref)
                row = dict(info, window=wi + window_offset, freqs=list(window), iteration=it,
                           seconds=time.perf_counter() - t0, grid=[nx, nz])
                if net is not None and cfg.retrain_steps > 0:
                    # Alg. 2 on the new medium: a fresh Eq. 4.3 dataset, then Adam steps
                    t1 = time.perf_counter()
                    rcfg = RT.RetrainConfig(initial_size=cfg.retrain_initial, data_epochs=3, epochs=1000,
                                            batch=min(16, cfg.max_rhs), lr=cfg.retrain_lr,
                                            max_steps=cfg.retrain_steps, relative_loss=True, warmup_steps=0,
                                            seed=int(rng.integers(1 << 31)))
                    h = RT.retrain(native, net, ctx, cfg=rcfg)
                    row["retrain_loss"] = h.epoch_loss
                    row["retrain_seconds"] = time.perf_counter() - t1
                hist.rows.append(row)
                if log:
                    log(row)
        finally:
            native.helm_destroy(ctx)
    return hist
