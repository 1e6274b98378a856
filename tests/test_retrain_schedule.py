"""Alg. 2 schedule of the retraining driver, checked on the CPU with a fake
backend that records the calls (no GPU): 128 initial pairs and 3 data epochs
end with 1024 pairs (Sec. 4.2); 30 epochs of batch 16 make 1784 Adam steps."""
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2405_17696_gb300 import retrain as RT  # noqa: E402


class FakeNative:
    def __init__(self):
        self.made = 0
        self.refined = 0
        self.steps = []

    def cnn_make_samples(self, ctx, x, iters, r, e, nb, fidx):
        assert x.shape[0] == nb and r.shape[0] == nb and all(1 <= int(i) <= 10 for i in iters)
        r.fill_(1.0)
        e.fill_(2.0)
        self.made += nb

    def cnn_refine_samples(self, ctx, r, e, r2, e2, nb, fidx, literal):
        assert torch.all(r == 1.0)          # refines existing pairs only
        r2.copy_(r)
        e2.copy_(e)
        self.refined += nb

    def cnn_set_loss(self, net, kind):
        self.loss_kind = kind

    def cnn_train_step(self, net, ctx, r, e, nb, lr, fidx):
        assert torch.all(r == 1.0) and torch.all(e == 2.0)
        self.steps.append(nb)
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
    cfg = RT.RetrainConfig(initial_size=8, data_epochs=3, epochs=5, batch=4)
    fake = FakeNative()
    hist = RT.retrain(fake, None, None, nx=4, nz=2, cfg=cfg, device="cpu", chunk=3)
    assert fake.made == 8
    assert fake.refined == 8 + 16 + 32
    assert hist.dataset_sizes == [8, 16, 32, 64, 64]
    assert hist.steps == sum(n for _, n in RT.schedule(cfg)) == len(fake.steps)
