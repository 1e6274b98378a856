"""Light-weight retraining of the encoder-solver network (Alg. 2, Sec. 4.2).

The schedule, the dataset and every arithmetic step (data generation by
V-cycle-preconditioned FGMRES, the network forward/backward and Adam) live in
libhelm behind ``cnn_retrain_step``; this module only chooses the learning
rate of each step and records the losses.

Alg. 2 with the paper's budget (Sec. 4.2): an initial dataset of
``initial_size`` pairs by Eq. 4.3 (x ~ CN(0, 1), a random number of
V-cycle-preconditioned GMRES steps in {1..10}); every epoch trains once over
the dataset in batches (Adam), and the first ``data_epochs`` epochs end with one
refined pair per existing pair (the network's estimate followed by one
preconditioned GMRES step).  128 pairs and 3 data epochs give the final 1024
pairs; 30 epochs in total.  The learning rate decays geometrically per epoch
from ``lr`` to ``lr_final`` after a linear warm-up over the first steps.
"""
from __future__ import annotations

from dataclasses import dataclass, field

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
    max_steps: int | None = None   # Adam steps to take (default: the whole schedule)
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


def learning_rate(cfg: RetrainConfig, epoch: int, step: int) -> float:
    """Learning rate of Adam step `step` (0-based) taken in epoch `epoch` (0-based)."""
    decay = 1.0 if cfg.lr_final is None or cfg.epochs < 2 else (cfg.lr_final / cfg.lr) ** (1.0 / (cfg.epochs - 1))
    ramp = min(1.0, (step + 1) / cfg.warmup_steps) if cfg.warmup_steps > 0 else 1.0
    return cfg.lr * decay ** min(epoch, cfg.epochs - 1) * ramp


def retrain(native, net, ctx, cfg: RetrainConfig | None = None, begin: bool = True) -> RetrainHistory:
    """Run Alg. 2 on the medium (and frequencies) of ``ctx`` through cnn_retrain_step.

    begin=False continues the schedule (and dataset) the context already holds."""
    cfg = cfg or RetrainConfig()
    native.cnn_set_loss(net, 1 if cfg.relative_loss else 0)
    if begin:
        native.cnn_retrain_begin(ctx, initial_size=cfg.initial_size, data_epochs=cfg.data_epochs,
                                 epochs=cfg.epochs, max_gmres_steps=cfg.max_gmres_steps, literal=int(cfg.literal),
                                 seed=cfg.seed)
    total = sum(n for _, n in schedule(cfg)) if cfg.max_steps is None else cfg.max_steps
    hist = RetrainHistory()
    losses, epoch, size = [], None, None
    for step in range(total):
        st = native.cnn_retrain_state(ctx)
        if epoch is not None and st["epoch"] != epoch:
            hist.dataset_sizes.append(size)
            hist.epoch_loss.append(sum(losses) / len(losses))
            losses = []
        epoch = st["epoch"]
        losses.append(native.cnn_retrain_step(net, ctx, cfg.batch, learning_rate(cfg, epoch, step)))
        size = st["size"] or cfg.initial_size     # the first step builds the initial dataset
        hist.steps += 1
    if losses:
        hist.dataset_sizes.append(size)
        hist.epoch_loss.append(sum(losses) / len(losses))
    return hist
