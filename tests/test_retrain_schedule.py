"""Alg. 2 schedule of the retraining driver, checked on the CPU with a fake
backend that records the calls (no GPU): 128 initial pairs and 3 data epochs
end with 1024 pairs (Sec. 4.2); 30 epochs of batch 16 make 1784 Adam steps."""
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2405_17696_gb300 import retrain as RT  # noqa: E402


class FakeNative:
    """The schedule cnn_retrain_step documents (include/helm.h), on the host: the
    first step builds the initial pairs, each step trains on the next batch of the
    epoch, and the first data_epochs epochs end by doubling the dataset."""

    def __init__(self):
        self.steps = []
        self.lrs = []
        self.begun = None

    def cnn_set_loss(self, net, kind):
        self.loss_kind = kind

    def cnn_retrain_begin(self, ctx, **opts):
        self.begun = opts
        self.size, self.epoch, self.pos, self.nsteps = 0, 0, 0, 0

    def cnn_retrain_state(self, ctx):
        return {"epoch": self.epoch, "pos": self.pos, "size": self.size, "steps": self.nsteps,
                "done": int(self.epoch >= self.begun["epochs"]), "capacity": 0}

    def cnn_retrain_step(self, net, ctx, batch, lr):
        if self.size == 0:
            self.size = self.begun["initial_size"]
        nb = min(batch, self.size - self.pos)
        self.steps.append(nb)
        self.lrs.append(lr)
        self.pos += nb
        self.nsteps += 1
        if self.pos >= self.size:
            self.pos = 0
            self.epoch += 1
            if self.epoch <= self.begun["data_epochs"]:
                self.size *= 2
        return 1.0 / len(self.steps)


def _golden():
    path = os.path.join(os.path.dirname(__file__), "golden", "alg2_schedule.txt")
    vals = {}
    for line in open(path):
        line = line.strip()
        if line and not line.startswith("#"):
            k, v = line.split()
            vals[k] = int(v)
    return vals


def test_schedule_matches_the_paper_budget():
    gold = _golden()   # Sec. 4.2, Alg. 2
    cfg = RT.RetrainConfig()
    assert (cfg.initial_size, cfg.data_epochs, cfg.epochs, cfg.batch) == (
        gold["initial_pairs"], gold["data_epochs"], gold["epochs"], gold["batch"])
    sched = RT.schedule(cfg)
    sizes = [gold["initial_pairs"] * 2 ** i for i in range(gold["data_epochs"] + 1)]
    assert [s for s, _ in sched[:4]] == sizes and sizes[-1] == gold["final_pairs"]
    assert sched[-1][0] == gold["final_pairs"] and len(sched) == gold["epochs"]
    # Adam steps: ceil(pairs / batch) per epoch
    assert sum(n for _, n in sched) == sum(-(-s // gold["batch"]) for s, _ in sched) == 1784


def test_driver_follows_the_schedule():
    cfg = RT.RetrainConfig(initial_size=8, data_epochs=3, epochs=5, batch=4, lr=1e-3, lr_final=1e-4,
                           warmup_steps=4)
    fake = FakeNative()
    hist = RT.retrain(fake, None, None, cfg=cfg)
    assert fake.begun["initial_size"] == 8 and fake.begun["data_epochs"] == 3 and fake.begun["epochs"] == 5
    assert hist.dataset_sizes == [8, 16, 32, 64, 64]
    assert hist.steps == sum(n for _, n in RT.schedule(cfg)) == len(fake.steps)
    assert fake.steps == [4] * hist.steps
    # warm-up ramp over the first 4 steps, then the geometric decay per epoch down to lr_final
    decay = (1e-4 / 1e-3) ** (1 / 4)
    assert fake.lrs[0] == pytest.approx(1e-3 / 4) and fake.lrs[1] == pytest.approx(1e-3 / 2)   # epoch 0
    assert fake.lrs[4] == pytest.approx(1e-3 * decay)                                         # epoch 1
    assert fake.lrs[-1] == pytest.approx(1e-4)
    assert len(hist.epoch_loss) == 5
