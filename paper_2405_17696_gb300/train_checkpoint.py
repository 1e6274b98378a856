"""Offline training of the encoder-solver network's initial weights (Sec. 4.1-4.2,
Sec. 5.2: the paper trains its initial weights offline, then retrains lightly on
the current medium between FWI iterations), through the library's own Alg. 2
training (cnn_retrain_step), and a checkpoint of the result (cnn_save).

The network is trained on one or several seeded media of the layered family at
the given grid and frequency, one Alg. 2 dataset per medium (Eq. 4.3 pairs from
Gaussian x, refined by the network's own estimates), steps taken round-robin
over the media; it is evaluated (CNN-FGMRES iterations on point sources against
MG-FGMRES) on an evaluation medium every --eval-every steps.  A JSON file beside
the checkpoint records how it was made.

    python -m paper_2405_17696_gb300.train_checkpoint --out weights/net.ckpt \\
        [--nx 1024 --nz 512 --h 12.5 --freq 8 --steps 6000 --media 10,11,12,13 --eval-seed 0]
"""
from __future__ import annotations

import argparse
import json
import math
import os
import sys
import time

import numpy as np

from . import media
from . import retrain as RT

WIDTHS = (16, 32, 64, 128)


def _medium(nx, nz, h, freq, seed, torch):
    c = media.layered_velocity(nx, nz, seed=seed)
    kap = torch.from_numpy(media.kappa_of(c)).cuda()
    gam = torch.from_numpy(media.abl_gamma(nx, nz, 32)).cuda()
    om = torch.tensor([2 * math.pi * freq], dtype=torch.float32, device="cuda")
    return kap, gam, om


def evaluate(native, net, nx, nz, h, freq, seed, n_rhs=32, torch=None):
    """(CNN-FGMRES, MG-FGMRES) iterations (mean, max) on n_rhs point sources of the medium."""
    kap, gam, om = _medium(nx, nz, h, freq, seed, torch)
    pos = media.top_row_positions(nx, 128)[::max(1, 128 // n_rhs)][:n_rhs]
    rhs = torch.from_numpy(media.point_source_rhs(nx, nz, pos, h, h)).cuda()
    out = {}
    for label, nn in (("cnn", net), ("mg", None)):
        ctx = native.helm_setup(kap, gam, nx, nz, h, h, om, net=nn, opts=native.helm_default_opts(
            mg_levels=3, max_iter=1000, max_rhs=n_rhs, precond=native.HELM_PC_CNN if nn else native.HELM_PC_MG))
        try:
            x = torch.zeros(rhs.shape, dtype=torch.complex128, device="cuda")
            _, it, rel, _ = native.helm_solve(ctx, rhs, x, n_rhs, None, 1e-6, native.HELM_SOLVE_ZERO_X0)
        finally:
            native.helm_destroy(ctx)
        out[label] = [float(it.mean()), int(it.max())]
    return out


def save(native, net, path):
    """The parameters only (no Adam moments): a fresh network with them, saved."""
    params = np.zeros(native.cnn_num_params(net), np.float32)
    native.cnn_get_params(net, params)
    out = native.cnn_create(len(WIDTHS), WIDTHS)
    native.cnn_set_params(out, params)
    native.cnn_set_loss(out, 1)
    os.makedirs(os.path.dirname(os.path.abspath(path)), exist_ok=True)
    native.cnn_save(out, path)
    native.cnn_destroy(out)


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--out", required=True)
    ap.add_argument("--nx", type=int, default=1024)
    ap.add_argument("--nz", type=int, default=512)
    ap.add_argument("--h", type=float, default=12.5)
    ap.add_argument("--freq", type=float, default=8.0)
    ap.add_argument("--steps", type=int, default=6000)
    ap.add_argument("--media", default="10,11,12,13")
    ap.add_argument("--eval-seed", type=int, default=media.SEED_MODEL)
    ap.add_argument("--eval-every", type=int, default=2000)
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--lr-final", type=float, default=1e-4)
    ap.add_argument("--lr-epochs", type=int, default=None,
                    help="epochs over which the learning rate decays geometrically from --lr to --lr-final, "
                         "then holds (default: steps / 64 + 4); with one medium an epoch is one pass of Alg. 2 "
                         "over its dataset, with several 64 steps")
    ap.add_argument("--save-every-eval", action="store_true",
                    help="also write a checkpoint (suffix _<steps>) at every evaluation")
    ap.add_argument("--init", default=None, help="continue from this checkpoint instead of seeded weights")
    ap.add_argument("--retrain-steps", type=int, default=0,
                    help="Alg. 2 steps on the evaluation medium after the offline training (reported, not saved)")
    args = ap.parse_args(argv)
    import torch
    from . import native
    seeds = [int(s) for s in args.media.split(",")]
    nx, nz, h, f = args.nx, args.nz, args.h, args.freq
    net = native.cnn_load(args.init) if args.init else native.cnn_create(len(WIDTHS), WIDTHS, seed=media.SEED_CNN)
    native.cnn_set_loss(net, 1)
    ctxs = []
    for s in seeds:
        kap, gam, om = _medium(nx, nz, h, f, s, torch)
        ctx = native.helm_setup(kap, gam, nx, nz, h, h, om, net=net, opts=native.helm_default_opts(
            mg_levels=3, max_rhs=32, precond=native.HELM_PC_CNN))
        native.cnn_retrain_begin(ctx, initial_size=128, data_epochs=3, epochs=1 << 20, seed=media.SEED_DATAGEN + s)
        ctxs.append(ctx)
    lr_epochs = args.lr_epochs if args.lr_epochs else args.steps // 64 + 4
    cfg = RT.RetrainConfig(epochs=max(2, lr_epochs), lr=args.lr, lr_final=args.lr_final, warmup_steps=100)
    log = {"command": " ".join([os.path.basename(sys.executable), "-m", "paper_2405_17696_gb300.train_checkpoint"] +
                               (argv if argv is not None else sys.argv[1:])),
           "grid": [nx, nz], "h_m": h, "freq_hz": f, "widths": list(WIDTHS), "train_media_seeds": seeds,
           "loss": "Eq. 4.2 with each pair weighted by 1 / ||e||^2", "batch": 16,
           "lr": [args.lr, args.lr_final], "lr_epochs": lr_epochs, "init": args.init, "evals": []}
    t0 = time.perf_counter()
    losses = []
    for step in range(args.steps):
        ctx = ctxs[step % len(ctxs)]
        # one medium: the epochs of its Alg. 2 schedule; several: 64-step epochs of all media together
        epoch = native.cnn_retrain_state(ctx)["epoch"] if len(ctxs) == 1 else step // 64
        losses.append(native.cnn_retrain_step(net, ctx, 16, RT.learning_rate(cfg, epoch, step)))
        if (step + 1) % args.eval_every == 0 or step + 1 == args.steps:
            torch.cuda.synchronize()
            ev = evaluate(native, net, nx, nz, h, f, args.eval_seed, torch=torch)
            row = {"steps": step + 1, "seconds": time.perf_counter() - t0,
                   "loss_last_200": float(np.mean(losses[-200:])), "eval": ev}
            log["evals"].append(row)
            print(json.dumps(row), flush=True)
            if args.save_every_eval:
                save(native, net, f"{os.path.splitext(args.out)[0]}_{step + 1}.ckpt")
    log["steps"] = args.steps
    log["seconds"] = time.perf_counter() - t0
    log["loss_first_200"] = float(np.mean(losses[:200]))
    log["loss_last_200"] = float(np.mean(losses[-200:]))
    for ctx in ctxs:
        native.helm_destroy(ctx)
    save(native, net, args.out)
    if args.retrain_steps > 0:
        # light retraining on the evaluation medium (Alg. 2), as between FWI iterations
        kap, gam, om = _medium(nx, nz, h, f, args.eval_seed, torch)
        ctx = native.helm_setup(kap, gam, nx, nz, h, h, om, net=net, opts=native.helm_default_opts(
            mg_levels=3, max_rhs=32, precond=native.HELM_PC_CNN))
        t1 = time.perf_counter()
        hist = RT.retrain(native, net, ctx, cfg=RT.RetrainConfig(max_steps=args.retrain_steps, epochs=1 << 20,
                                                                 lr=args.lr_final, relative_loss=True,
                                                                 warmup_steps=0))
        native.helm_destroy(ctx)
        log["retrain_on_eval_medium"] = {"steps": args.retrain_steps, "seconds": time.perf_counter() - t1,
                                         "loss": hist.epoch_loss[-1],
                                         "eval": evaluate(native, net, nx, nz, h, f, args.eval_seed, torch=torch)}
        print(json.dumps(log["retrain_on_eval_medium"]), flush=True)
    native.cnn_destroy(net)
    with open(os.path.splitext(args.out)[0] + ".json", "w") as fh:
        json.dump(log, fh, indent=1)


if __name__ == "__main__":
    main()
