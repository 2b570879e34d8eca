"""Learned closure pipeline: data from fine RR runs, training, evaluation.

Everything the method computes runs in the library's kernels (RR steps,
coarsening, features, targets, the network's forward/backward and Adam, the
closure step). This module only orchestrates: it picks snapshot times and cell
samples, forms minibatches (index selection) and reduces statistics with
torch.

Recipe (a priori training on filtered fine data):
  * fine D3Q27 RR runs of the Taylor-Green vortex at n_f^3 (Ma, Re), one per
    seeded phase shift;
  * at each snapshot the fine populations are box-filtered 2x2x2 onto the
    coarse grid (n_f/2)^3; features are the coarse cells' 3^3-neighbourhood
    moments, targets the order 3..6 off-equilibrium coefficients that the
    recursion does not reproduce;
  * standardisation: mean / std per moment kind (features) and root mean
    square per coefficient (targets), from the training data;
  * Adam on minibatches;
  * evaluation on a held-out phase: the coarse run (tau_c = 1/2 + (tau_f - 1/2)/2,
    one coarse step per two fine steps) with and without the closure, both
    started from the filtered fine state, against the filtered fine run.
"""
from __future__ import annotations

import math

import numpy as np

from . import binding as B
from . import workloads as W


def coarse_tau(tau_f: float) -> float:
    return 0.5 + (tau_f - 0.5) / 2.0


def phase_of(seed: int):
    rng = np.random.default_rng(seed)
    return tuple(rng.uniform(0.0, 2.0 * math.pi, 3))


def tgv_solver(n: int, mach: float, re: float, seed: int, stream=None):
    import torch
    tau = W.taylor_green_3d_tau(n, mach, re)
    rho, u = W.taylor_green_3d(n, mach, phase=phase_of(seed))
    s = B.Solver(B.D3Q27, (n, n, n), tau, stream=stream)
    s.init_fields(torch.from_numpy(rho.astype(np.float32)).cuda(),
                  torch.from_numpy(u.astype(np.float32)).cuda())
    return s


def _snapshots(n_fine, mach, re, seeds, snapshots):
    """Yield (seed index, snapshot index, coarse solver) holding the filtered
    fine state at each snapshot of each seeded run."""
    nc = n_fine // 2
    for si, seed in enumerate(seeds):
        fine = tgv_solver(n_fine, mach, re, seed)
        coarse = B.Solver(B.D3Q27, (nc, nc, nc), coarse_tau(fine.tau))
        done = 0
        for ki, snap in enumerate(snapshots):
            assert snap % 2 == 0 and snap >= done
            fine.step(snap - done)
            done = snap
            coarse.coarsen_from(fine)
            yield si, ki, coarse
        fine.close()
        coarse.close()


def generate_dataset(n_fine: int, mach: float, re: float, seeds, snapshots, fraction: float,
                     sample_seed: int = 0):
    """Standardised training data (X [S][288] BF16, T [S][32] FP32) of a random
    fraction of the coarse cells at the snapshot fine steps of each seeded run,
    and the standardisation (in_mean, in_inv_std, out_scale).

    Two passes over the (deterministic) fine runs: the first takes the
    statistics from the coarse moment fields and the raw targets, the second
    computes the features with the final standardisation."""
    import torch
    raw = B.MLP()  # identity standardisation
    gen = torch.Generator(device="cuda").manual_seed(sample_seed)
    picks, targs = {}, []
    s1 = torch.zeros(10, dtype=torch.float64, device="cuda")
    s2 = torch.zeros(10, dtype=torch.float64, device="cuda")
    cnt = 0
    for si, ki, coarse in _snapshots(n_fine, mach, re, seeds, snapshots):
        rho, u, pi = coarse.moments()
        mom = torch.cat([(rho - 1.0).reshape(1, -1), u.reshape(3, -1), pi.reshape(6, -1)])
        mom = mom.double()
        s1 += mom.sum(1)
        s2 += (mom * mom).sum(1)
        cnt += mom.shape[1]
        idx = torch.nonzero(torch.rand(coarse.n, device="cuda", generator=gen) < fraction)[:, 0]
        picks[(si, ki)] = idx
        targs.append(coarse.closure_targets(raw).index_select(0, idx))
    mean = s1 / cnt
    std = torch.sqrt(torch.clamp(s2 / cnt - mean * mean, min=0.0))
    # a moment kind that barely varies (e.g. a velocity component that stays
    # zero) must not turn round-off into large standardised features
    std = torch.maximum(std, 1e-3 * std.max())
    T = torch.cat(targs)
    out_scale = T[:, :17].double().pow(2).mean(0).sqrt().clamp_min(1e-30)
    T[:, :17] = (T[:, :17].double() / out_scale).float()
    mean_np = mean.cpu().numpy().astype(np.float32)
    inv_np = (1.0 / std).cpu().numpy().astype(np.float32)
    out_np = out_scale.cpu().numpy().astype(np.float32)
    scaled = B.MLP()
    scaled.set_scaling(mean_np, inv_np, out_np)
    feats = []
    for si, ki, coarse in _snapshots(n_fine, mach, re, seeds, snapshots):
        feats.append(coarse.closure_features(scaled).index_select(0, picks[(si, ki)]))
    return torch.cat(feats).contiguous(), T.contiguous(), (mean_np, inv_np, out_np)


def init_params(seed: int) -> np.ndarray:
    """Small random weights (Glorot-like), zero biases, zero padded rows/cols,
    and a zero output layer so that the untrained network is exactly RR."""
    rng = np.random.default_rng(seed)
    W1 = rng.standard_normal((64, 288)) * math.sqrt(1.0 / 270)
    W1[:, 270:] = 0.0
    W2 = rng.standard_normal((64, 64)) * math.sqrt(1.0 / 64)
    W3 = np.zeros((32, 64))
    return np.concatenate([W1.ravel(), np.zeros(64), W2.ravel(), np.zeros(64), W3.ravel(),
                           np.zeros(32)]).astype(np.float32)


def train(net: B.MLP, X, T, steps: int, batch: int, lr: float, seed: int = 0):
    import torch
    gen = torch.Generator(device="cuda").manual_seed(seed)
    losses = []
    n = X.shape[0]
    for k in range(steps):
        idx = torch.randint(0, n, (batch,), device="cuda", generator=gen)
        loss = net.train_step(X.index_select(0, idx), T.index_select(0, idx), lr,
                              want_loss=(k % 50 == 0 or k == steps - 1))
        if loss is not None:
            losses.append((k, loss))
    return losses


def velocity_error(a, b) -> float:
    import torch
    return float(torch.linalg.vector_norm(a - b) / torch.linalg.vector_norm(b))


def evaluate(net, n_fine: int, mach: float, re: float, seed: int, coarse_steps: int,
             bound: float = 8.0):
    """Relative L2 errors of u of the coarse RR run and of the coarse run with
    the closure against the filtered fine run, after coarse_steps coarse steps."""
    import torch
    nc = n_fine // 2
    fine = tgv_solver(n_fine, mach, re, seed)
    tc = coarse_tau(fine.tau)
    ref = B.Solver(B.D3Q27, (nc, nc, nc), tc)
    rr = B.Solver(B.D3Q27, (nc, nc, nc), tc)
    ml = B.Solver(B.D3Q27, (nc, nc, nc), tc)
    rr.coarsen_from(fine)
    ml.coarsen_from(fine)
    ml.set_closure(net, bound)
    fine.step(2 * coarse_steps)
    rr.step(coarse_steps)
    ml.step(coarse_steps)
    ref.coarsen_from(fine)
    _, u_ref, _ = ref.moments()
    _, u_rr, _ = rr.moments()
    _, u_ml, _ = ml.moments()
    out = {"err_rr": velocity_error(u_rr, u_ref), "err_closure": velocity_error(u_ml, u_ref),
           "fallbacks": ml.closure_fallbacks(), "cells": nc ** 3, "coarse_steps": coarse_steps}
    for s in (fine, ref, rr, ml):
        s.close()
    torch.cuda.synchronize()
    return out


def held_out_loss(net, n_fine: int, mach: float, re: float, seed: int, snapshots) -> dict:
    """A priori check on a phase the network was not trained on: the mean
    square of the standardised targets (orders 3..6 that the recursion leaves
    out) over every coarse cell of the filtered snapshots, left as they are
    (the zero network, i.e. plain RR) and after subtracting the network's
    prediction."""
    import torch
    raw = B.MLP()  # identity standardisation: raw targets
    out_scale = torch.from_numpy(net.scaling[2].astype(np.float64)).cuda()
    s_zero = s_net = 0.0
    count = 0
    for _, _, coarse in _snapshots(n_fine, mach, re, [seed], snapshots):
        T = coarse.closure_targets(raw)[:, :17].double() / out_scale
        Y = net.forward(coarse.closure_features(net))[:, :17].double()
        s_zero += float((T * T).sum())
        s_net += float(((Y - T) ** 2).sum())
        count += T.numel()
    raw.close()
    return {"zero": s_zero / count, "trained": s_net / count, "values": count}


def study(n_fine=64, mach=0.3, re=1600.0, train_seeds=range(1, 9), eval_seed=9,
          snapshots=(100, 200, 300, 400), fraction=0.25, steps=1500, batch=8192, lr=2e-3,
          coarse_steps=200):
    """The whole recipe at one size; returns the trained network and a report."""
    X, T, (mean, inv, out_scale) = generate_dataset(n_fine, mach, re, list(train_seeds),
                                                     snapshots, fraction)
    net = B.MLP(init_params(0))
    net.set_scaling(mean, inv, out_scale)
    losses = train(net, X, T, steps, batch, lr)
    report = {"samples": int(X.shape[0]), "loss_first": losses[0][1], "loss_last": losses[-1][1],
              "n_fine": n_fine, "mach": mach, "re": re}
    report.update(evaluate(net, n_fine, mach, re, eval_seed, coarse_steps))
    return net, report


def main():
    """The recipe at a chosen size, printed as one JSON line: the training
    statistics, the held-out phase's a priori check and the velocity errors
    of coarse RR with and without the closure against the filtered fine run.

        python -m paper_1505_06900_gb300.closure --n-fine 512 --fraction 0.02
    """
    import argparse
    import json
    import time

    ap = argparse.ArgumentParser()
    ap.add_argument("--n-fine", type=int, default=128)
    ap.add_argument("--fraction", type=float, default=0.25)
    ap.add_argument("--steps", type=int, default=1500)
    ap.add_argument("--coarse-steps", type=int, default=400)
    ap.add_argument("--snapshots", type=int, nargs="+", default=[200, 400, 600, 800])
    args = ap.parse_args()
    t0 = time.perf_counter()
    net, rep = study(n_fine=args.n_fine, fraction=args.fraction, steps=args.steps,
                     coarse_steps=args.coarse_steps, snapshots=tuple(args.snapshots))
    rep["seconds_study"] = time.perf_counter() - t0
    rep["held_out_a_priori"] = held_out_loss(net, args.n_fine, rep["mach"], rep["re"], 9,
                                             tuple(args.snapshots))
    rep["fraction"] = args.fraction
    rep["adam_steps"] = args.steps
    net.close()
    print(json.dumps(rep), flush=True)


if __name__ == "__main__":
    main()

