"""Light-weight retraining of the encoder-solver network (Alg. 2, Sec. 4.2).

A thin driver over the C ABI: every arithmetic step (data generation by
V-cycle-preconditioned FGMRES, the network forward/backward and Adam) runs
in libhelm's kernels; this module only schedules the calls and owns the
dataset tensors.

Alg. 2 (with the paper's budget, Sec. 4.2): build an initial dataset of
``initial_size`` pairs by Eq. 4.3 (x ~ CN(0, 1), a random number of
V-cycle-preconditioned GMRES steps in {1..10}); then for every epoch train
once over the dataset in batches (Adam, learning rate decayed geometrically
per epoch from ``lr`` to ``lr_final``), and during the first ``data_epochs`` epochs
append one refined pair per existing pair (the network's estimate followed by
one preconditioned GMRES step, `cnn_refine_samples`).  128 pairs and 3 data
epochs give the final 1024 pairs; 30 epochs in total.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from . import media


@dataclass
class RetrainConfig:
    initial_size: int = 128
    data_epochs: int = 3
    epochs: int = 30
    batch: int = 16
    lr: float = 1e-4
    lr_final: float | None = None  # learning rate of the last epoch (geometric decay per epoch); None = constant
    max_gmres_steps: int = 10
    literal: bool = False          # Alg. 2 as printed instead of the residual-correction pair
    seed: int = media.SEED_DATAGEN
    max_steps: int | None = None   # optional cap on the number of Adam steps (short sessions)
    relative_loss: bool = False    # weigh each pair by 1 / ||e||^2 instead of Eq. 4.2's plain sum
    warmup_steps: int = 100        # linear learning-rate ramp over the first Adam steps


@dataclass
class RetrainHistory:
    dataset_sizes: list = field(default_factory=list)   # size of the dataset trained on, per epoch
    epoch_loss: list = field(default_factory=list)      # mean batch loss per epoch
    steps: int = 0


def schedule(cfg: RetrainConfig):
    """(dataset size trained on, number of Adam steps) per epoch of Alg. 2."""
    size, out = cfg.initial_size, []
    for i in range(1, cfg.epochs + 1):
        out.append((size, -(-size // cfg.batch)))
        if i <= cfg.data_epochs:
            size *= 2
    return out


def retrain(native, net, ctx, nx: int, nz: int, freq_of_sample=None, cfg: RetrainConfig | None = None,
            device: str = "cuda", chunk: int = 16) -> RetrainHistory:
    """Run Alg. 2 on the medium (and frequencies) of ``ctx``.

    ``freq_of_sample(i)`` gives the frequency index of sample i (default 0);
    ``chunk`` bounds the number of pairs per data-generation call (max_rhs).
    """
    import torch

    cfg = cfg or RetrainConfig()
    native.cnn_set_loss(net, 1 if cfg.relative_loss else 0)
    g = media.rng(cfg.seed)
    fsel = freq_of_sample or (lambda i: 0)
    cap = cfg.initial_size * 2 ** cfg.data_epochs
    R = torch.zeros((cap, nz, nx), dtype=torch.complex64, device=device)
    E = torch.zeros_like(R)
    F = np.array([fsel(i) for i in range(cap)], dtype=np.int32)
    # initial dataset, Eq. 4.3
    for s0 in range(0, cfg.initial_size, chunk):
        nb = min(chunk, cfg.initial_size - s0)
        x = media.complex_normal((nb, nz, nx), seed=int(g.integers(1 << 31)))
        iters = g.integers(1, cfg.max_gmres_steps + 1, size=nb)
        native.cnn_make_samples(ctx, torch.from_numpy(x).to(device), iters, R[s0:s0 + nb], E[s0:s0 + nb], nb,
                                F[s0:s0 + nb])
    size = cfg.initial_size
    hist = RetrainHistory()
    decay = 1.0 if cfg.lr_final is None or cfg.epochs < 2 else (cfg.lr_final / cfg.lr) ** (1.0 / (cfg.epochs - 1))
    for epoch in range(1, cfg.epochs + 1):
        lr = cfg.lr * decay ** (epoch - 1)
        order = g.permutation(size)
        losses = []
        for b0 in range(0, size, cfg.batch):
            idx = order[b0:b0 + cfg.batch]
            ti = torch.from_numpy(idx).to(device)
            r = R.index_select(0, ti).contiguous()
            e = E.index_select(0, ti).contiguous()
            ramp = min(1.0, (hist.steps + 1) / cfg.warmup_steps) if cfg.warmup_steps > 0 else 1.0
            losses.append(native.cnn_train_step(net, ctx, r, e, len(idx), lr * ramp, F[idx]))
            hist.steps += 1
            if cfg.max_steps is not None and hist.steps >= cfg.max_steps:
                break
        hist.dataset_sizes.append(size)
        hist.epoch_loss.append(float(np.mean(losses)))
        if cfg.max_steps is not None and hist.steps >= cfg.max_steps:
            break
        if epoch <= cfg.data_epochs:
            # one refined pair per existing pair (Alg. 2, data epochs)
            for s0 in range(0, size, chunk):
                nb = min(chunk, size - s0)
                native.cnn_refine_samples(ctx, R[s0:s0 + nb], E[s0:s0 + nb], R[size + s0:size + s0 + nb],
                                          E[size + s0:size + s0 + nb], nb, F[s0:s0 + nb], int(cfg.literal))
                F[size + s0:size + s0 + nb] = F[s0:s0 + nb]
            size *= 2
    return hist
