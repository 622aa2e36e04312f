"""Train the learned initial guess of the symmetron solve and measure what it gains.

    python -m paper_1307_6748_gb300.train_guess --pairs 2000 --N 128 --epochs 4 --out guess.npz

1. Training pairs: seeded lognormal densities (sigma 1.5, cell size 1 Mpc/h) at
   N^3, half at a = 0.8 and half at a = 1.0, solved by isis_scalar_solve
   (FP32 cycles + FP64 refinement, relative residual 1e-8).  Target chi - chi_bg(a).
2. Training: Adam on the squared error, one pair per step, every kernel the
   library's own (forward, backward, optimiser).
3. Evaluation on held-out seeds at the evaluation grid (default 256^3, 256
   Mpc/h): V-cycles and wall time to 1e-8 from the background field and from
   the net's guess (the net's inference time included).
Prints one JSON summary line.
"""
from __future__ import annotations

import argparse
import json
import math
import time

import numpy as np
import torch

from . import isis, synth, unet

A_SSB = 0.5
SIGMA = 1.5


def solve(eta, a, phi, tol, init):
    opts = isis.Opts(prec=isis.ISIS_F32_REFINE64, inner_cycles=3, n_coarsest=2, init=init)
    return isis.isis_scalar_solve(isis.ISIS_SYMMETRON, isis.Params(a_ssb=A_SSB), isis.Grid(eta.shape[0], float(eta.shape[0])),
                                  a, eta, phi, tol=tol, opts=opts)


def make_pairs(n_pairs, N, seed0=1000):
    lg = int(round(math.log2(N)))
    etas, targets, avals = [], [], []
    phi = torch.empty((N,) * 3, dtype=torch.float64, device="cuda")
    t0 = time.time()
    for s in range(n_pairs):
        a = 0.8 if s % 2 == 0 else 1.0
        eta = synth.lognormal_eta(N, float(N), SIGMA, seed0 + s, device="cuda")
        solve(eta, a, phi, 1e-8, isis.ISIS_INIT_BACKGROUND)
        etas.append(eta)
        targets.append((phi - isis.isis_background_field(isis.ISIS_SYMMETRON, isis.Params(a_ssb=A_SSB), a)).float().reshape(-1))
        avals.append(a)
    torch.cuda.synchronize()
    return etas, targets, avals, lg, time.time() - t0


def train(net, etas, targets, avals, lg, epochs, lr0=1e-3, lr1=1e-4, seed=7):
    rng = np.random.Generator(np.random.PCG64(seed))
    n = len(etas)
    total = epochs * n
    history = []
    step = 0
    t0 = time.time()
    for ep in range(epochs):
        order = rng.permutation(n)
        acc = torch.zeros(1, dtype=torch.float64, device="cuda")
        for q in order:
            lr = lr1 + 0.5 * (lr0 - lr1) * (1 + math.cos(math.pi * step / max(1, total - 1)))
            loss = net.train_step(etas[q], avals[q], targets[q], lg, lr=lr)
            acc += loss
            step += 1
        torch.cuda.synchronize()
        history.append(float(acc.item()) / n)
    torch.cuda.synchronize()
    return history, time.time() - t0


def evaluate(net, N, seeds, avals, tol=1e-8):
    out = []
    phi = torch.empty((N,) * 3, dtype=torch.float64, device="cuda")
    ref = torch.empty_like(phi)

    def rms(x):
        return float(torch.sqrt(torch.mean(x * x)).item())

    def run(mode, eta, a):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record()
        if mode == "net":
            net.guess(eta, a, A_SSB, phi)  # inference is part of the timed solve
            info = solve(eta, a, phi, tol, isis.ISIS_INIT_INPUT)
        else:
            info = solve(eta, a, phi, tol, isis.ISIS_INIT_BACKGROUND)
        e1.record()
        torch.cuda.synchronize()
        return info, e0.elapsed_time(e1)

    for seed in seeds:
        eta = synth.lognormal_eta(N, float(N), SIGMA, seed, device="cuda")
        for a in avals:
            solve(eta, a, ref, 1e-10, isis.ISIS_INIT_BACKGROUND)  # converged reference (not timed)
            row = {"seed": seed, "a": a}
            for mode in ("background", "net"):
                run(mode, eta, a)  # warm-up
                info, ms = run(mode, eta, a)
                row[mode] = {"cycles": info.cycles, "outer": info.outer, "ms": ms,
                             "rel_l2_vs_converged": rms(phi - ref) / rms(ref)}
            net.guess(eta, a, A_SSB, phi)
            row["net"]["guess_rms_error"] = rms(phi - ref)
            row["background"]["guess_rms_error"] = rms(ref - isis.isis_background_field(isis.ISIS_SYMMETRON, isis.Params(a_ssb=A_SSB), a))
            out.append(row)
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--pairs", type=int, default=2000)
    ap.add_argument("--N", type=int, default=128)
    ap.add_argument("--epochs", type=int, default=4)
    ap.add_argument("--eval-N", type=int, default=256)
    ap.add_argument("--eval-seeds", type=int, default=4)
    ap.add_argument("--out", default="guess.npz")
    args = ap.parse_args()
    isis.load()
    etas, targets, avals, lg, t_data = make_pairs(args.pairs, args.N)
    net = unet.UNet(seed=0, mu=-0.5 * SIGMA * SIGMA, sd=SIGMA)
    hist, t_train = train(net, etas, targets, avals, lg, args.epochs)
    assert int(net.err.item()) == 0
    net.save(args.out, model="symmetron", h=1.0, a_ssb=A_SSB, lambda0=1.0, beta=1.0, sigma=SIGMA,
             pairs=args.pairs, N=args.N, epochs=args.epochs)
    del etas, targets
    torch.cuda.empty_cache()
    ev = evaluate(net, args.eval_N, [9000 + s for s in range(args.eval_seeds)], [0.8, 1.0])
    summary = {"pairs": args.pairs, "N": args.N, "epochs": args.epochs, "data_s": t_data, "train_s": t_train,
               "steps_per_s": args.pairs * args.epochs / t_train, "loss_per_epoch": hist, "eval_N": args.eval_N,
               "eval": ev,
               "mean_cycles": {m: float(np.mean([r[m]["cycles"] for r in ev])) for m in ("background", "net")},
               "mean_ms": {m: float(np.mean([r[m]["ms"] for r in ev])) for m in ("background", "net")}}
    print(json.dumps(summary), flush=True)


if __name__ == "__main__":
    main()
