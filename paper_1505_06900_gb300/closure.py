"""Learned closure pipeline: data from fine RR runs, training, evaluation.

Everything the method computes runs in the library's kernels (RR steps,
coarsening, features, targets, the network's forward/backward and Adam, the
closure step). This module only orchestrates: it picks snapshot times and cell
samples, forms minibatches (index selection), schedules the learning rate and
reduces statistics with torch.

Recipe (step-matching targets on filtered fine data):
  * fine D3Q27 RR runs of the Taylor-Green vortex at n_f^3 (Ma, Re), one per
    seeded phase shift;
  * the coarse grid (n_f/2)^3 takes acoustic scaling (tau_c = 1/2 +
    (tau_f - 1/2)/2, one coarse update per two fine updates); fine states are
    box-filtered 2x2x2 onto it with the off-equilibrium part rescaled by
    2 tau_c / tau_f (lb_coarsen_neq), which makes them states the coarse
    dynamics itself would carry (the plain average holds about half the
    off-equilibrium part a coarse run builds, and a coarse run started from
    it rings for its first updates);
  * at each snapshot fine step t: A = the filtered state at t, B = the one at
    t + 2; features are A's 3^3-neighbourhood moments, targets the order 3..6
    correction that makes the RR update of A reproduce those coefficients of B
    (lb_closure_step_targets);
  * standardisation: mean / std per moment kind (features) and root mean
    square per coefficient (targets), from the training data;
  * Adam on minibatches with a cosine-decaying learning rate;
  * the coarse run adds GAIN times the predicted correction: the orders 0 and
    1 of B are out of a local collision's reach, and correcting orders 3..6 in
    full against them overshoots; each standardised prediction is shrunk by
    the dead zone DEAD_ZONE first (sign(y) max(|y| - DEAD_ZONE, 0)), so that
    where the coarse grid still resolves the flow and the correction is below
    the network's own error, the cell keeps plain RR;
  * evaluation on a held-out phase: the coarse run (tau_c, one coarse step
    per two fine steps) with and without the closure, both started from the
    filtered fine state, against the filtered fine run.
"""
from __future__ import annotations

import math

import numpy as np

from . import binding as B
from . import workloads as W


GAIN = 0.5  # share of the predicted correction the coarse run applies
DEAD_ZONE = 0.25  # shrinkage of the standardised predictions (lb_set_closure_ex)


def coarse_tau(tau_f: float) -> float:
    return 0.5 + (tau_f - 0.5) / 2.0


def neq_scale(tau_f: float) -> float:
    """Off-equilibrium rescaling of the filtered fine state, 2 tau_c / tau_f."""
    return 2.0 * coarse_tau(tau_f) / tau_f


def dense_snapshots(last: int, spacing: int = 24):
    """Even fine steps 0, spacing, 2 spacing, ... up to `last`."""
    return tuple(range(0, last + 1, spacing))


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
    """Yield (seed index, snapshot index, A, B): coarse solvers holding the
    filtered fine state at each snapshot step t of each seeded run and the
    one at t + 2 (off-equilibrium part rescaled)."""
    nc = n_fine // 2
    for si, seed in enumerate(seeds):
        fine = tgv_solver(n_fine, mach, re, seed)
        tc, scale = coarse_tau(fine.tau), neq_scale(fine.tau)
        a = B.Solver(B.D3Q27, (nc, nc, nc), tc)
        b = B.Solver(B.D3Q27, (nc, nc, nc), tc)
        done = 0
        for ki, snap in enumerate(snapshots):
            assert snap % 2 == 0 and snap >= done
            fine.step(snap - done)
            a.coarsen_from(fine, scale)
            fine.step(2)
            done = snap + 2
            b.coarsen_from(fine, scale)
            yield si, ki, a, b
        for x in (fine, a, b):
            x.close()


def generate_dataset(n_fine: int, mach: float, re: float, seeds, snapshots, fraction: float,
                     sample_seed: int = 0):
    """Standardised training data (X [S][288] BF16, T [S][32] FP32) of a random
    fraction of the coarse cells at the snapshot fine steps of each seeded run,
    and the standardisation (in_mean, in_inv_std, out_scale).

    The feature standardisation comes from the first run's snapshots (a
    phase shift only translates the periodic flow, so every run has the same
    moment statistics); one pass over all runs then gathers features and raw
    targets, and the targets are standardised at the end."""
    import torch
    s1 = torch.zeros(10, dtype=torch.float64, device="cuda")
    s2 = torch.zeros(10, dtype=torch.float64, device="cuda")
    cnt = 0
    for _, _, a, _ in _snapshots(n_fine, mach, re, list(seeds)[:1], snapshots):
        rho, u, pi = a.moments()
        mom = torch.cat([(rho - 1.0).reshape(1, -1), u.reshape(3, -1), pi.reshape(6, -1)])
        mom = mom.double()
        s1 += mom.sum(1)
        s2 += (mom * mom).sum(1)
        cnt += mom.shape[1]
        del rho, u, pi, mom
    mean = s1 / cnt
    std = torch.sqrt(torch.clamp(s2 / cnt - mean * mean, min=0.0))
    # a moment kind that barely varies (e.g. a velocity component that stays
    # zero) must not turn round-off into large standardised features
    std = torch.maximum(std, 1e-3 * std.max())
    mean_np = mean.cpu().numpy().astype(np.float32)
    inv_np = (1.0 / std).cpu().numpy().astype(np.float32)
    scaled = B.MLP()  # feature standardisation, raw targets (out_scale 1)
    scaled.set_scaling(mean_np, inv_np, np.ones(17, np.float32))
    gen = torch.Generator(device="cuda").manual_seed(sample_seed)
    feats, targs = [], []
    for _, _, a, b in _snapshots(n_fine, mach, re, seeds, snapshots):
        idx = torch.nonzero(torch.rand(a.n, device="cuda", generator=gen) < fraction)[:, 0]
        feats.append(a.closure_features(scaled).index_select(0, idx))
        targs.append(a.closure_step_targets(b, scaled).index_select(0, idx))
    scaled.close()
    T = torch.cat(targs)
    out_scale = T[:, :17].double().pow(2).mean(0).sqrt().clamp_min(1e-30)
    T[:, :17] = (T[:, :17].double() / out_scale).float()
    out_np = out_scale.cpu().numpy().astype(np.float32)
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
    """Adam steps on random minibatches, the learning rate decaying from lr
    to 0 along a half cosine."""
    import torch
    gen = torch.Generator(device="cuda").manual_seed(seed)
    losses = []
    n = X.shape[0]
    for k in range(steps):
        idx = torch.randint(0, n, (batch,), device="cuda", generator=gen)
        lr_k = 0.5 * lr * (1.0 + math.cos(math.pi * k / steps))
        loss = net.train_step(X.index_select(0, idx), T.index_select(0, idx), lr_k,
                              want_loss=(k % 50 == 0 or k == steps - 1))
        if loss is not None:
            losses.append((k, loss))
    return losses


def velocity_error(a, b) -> float:
    import torch
    return float(torch.linalg.vector_norm(a - b) / torch.linalg.vector_norm(b))


def inference_net(params, scaling, gain: float = GAIN) -> B.MLP:
    """A network for the coarse run: the trained parameters with the output
    scale multiplied by the gain."""
    mean, inv, out_scale = scaling
    net = B.MLP(params)
    net.set_scaling(mean, inv, np.asarray(out_scale, np.float32) * np.float32(gain))
    return net


def evaluate(net, n_fine: int, mach: float, re: float, seed: int, coarse_steps: int,
             bound: float = 8.0, every: int | None = None, dead_zone: float = DEAD_ZONE):
    """Relative L2 errors of u of the coarse RR run and of the coarse run with
    the closure against the filtered fine run, after coarse_steps coarse steps
    (and every `every` coarse steps on the way, in "history")."""
    import torch
    nc = n_fine // 2
    fine = tgv_solver(n_fine, mach, re, seed)
    tc, scale = coarse_tau(fine.tau), neq_scale(fine.tau)
    ref = B.Solver(B.D3Q27, (nc, nc, nc), tc)
    rr = B.Solver(B.D3Q27, (nc, nc, nc), tc)
    ml = B.Solver(B.D3Q27, (nc, nc, nc), tc)
    rr.coarsen_from(fine, scale)
    ml.coarsen_from(fine, scale)
    ml.set_closure(net, bound, dead_zone)
    hist = []
    done = 0
    every = every or coarse_steps
    while done < coarse_steps:
        k = min(every, coarse_steps - done)
        fine.step(2 * k)
        rr.step(k)
        ml.step(k)
        done += k
        ref.coarsen_from(fine)
        _, u_ref, _ = ref.moments()
        _, u_rr, _ = rr.moments()
        _, u_ml, _ = ml.moments()
        hist.append((done, velocity_error(u_rr, u_ref), velocity_error(u_ml, u_ref)))
    out = {"err_rr": hist[-1][1], "err_closure": hist[-1][2], "history": hist,
           "fallbacks": ml.closure_fallbacks(), "cells": nc ** 3, "coarse_steps": coarse_steps}
    for s in (fine, ref, rr, ml):
        s.close()
    torch.cuda.synchronize()
    return out


def held_out_loss(net, n_fine: int, mach: float, re: float, seed: int, snapshots,
                  scaling) -> dict:
    """A priori check on a phase the network was not trained on: the mean
    square of the standardised targets (the step-matching correction of
    orders 3..6) over every coarse cell of the filtered snapshots, left as they
    are (the zero network, i.e. plain RR) and after subtracting the network's
    prediction. `scaling` is the training standardisation."""
    mean, inv, out_scale = scaling
    std_net = B.MLP(net.get_params())
    std_net.set_scaling(mean, inv, out_scale)
    s_zero = s_net = 0.0
    count = 0
    for _, _, a, b in _snapshots(n_fine, mach, re, [seed], snapshots):
        T = a.closure_step_targets(b, std_net)[:, :17].double()
        Y = std_net.forward(a.closure_features(std_net))[:, :17].double()
        s_zero += float((T * T).sum())
        s_net += float(((Y - T) ** 2).sum())
        count += T.numel()
    std_net.close()
    return {"zero": s_zero / count, "trained": s_net / count, "values": count}


def study(n_fine=64, mach=0.3, re=1600.0, train_seeds=range(1, 9), eval_seed=9,
          snapshots=None, fraction=0.25, steps=3000, batch=8192, lr=2e-3, coarse_steps=200,
          gain=GAIN, every=None, dead_zone=DEAD_ZONE):
    """The whole recipe at one size; returns the network the coarse run uses
    (output scale times the gain), the training standardisation and a report.
    Snapshots default to every 24 fine steps over the evaluated interval."""
    if snapshots is None:
        snapshots = dense_snapshots(2 * coarse_steps)
    X, T, scaling = generate_dataset(n_fine, mach, re, list(train_seeds), snapshots, fraction)
    samples = int(X.shape[0])
    trainer = B.MLP(init_params(0))
    losses = train(trainer, X, T, steps, batch, lr)
    del X, T
    net = inference_net(trainer.get_params(), scaling, gain)
    trainer.close()
    report = {"samples": samples, "loss_first": losses[0][1],
              "loss_last": losses[-1][1], "n_fine": n_fine, "mach": mach, "re": re,
              "gain": gain, "dead_zone": dead_zone,
              "snapshots": [snapshots[0], snapshots[-1], len(snapshots)]}
    report.update(evaluate(net, n_fine, mach, re, eval_seed, coarse_steps, every=every,
                           dead_zone=dead_zone))
    return net, scaling, report


def main():
    """The recipe at a chosen size, printed as one JSON line: the training
    statistics, the held-out phase's a priori check and the velocity errors
    of coarse RR with and without the closure against the filtered fine run.

        python -m paper_1505_06900_gb300.closure --n-fine 512 --fraction 0.01
    """
    import argparse
    import json
    import time

    ap = argparse.ArgumentParser()
    ap.add_argument("--n-fine", type=int, default=128)
    ap.add_argument("--fraction", type=float, default=0.05)
    ap.add_argument("--steps", type=int, default=3000)
    ap.add_argument("--coarse-steps", type=int, default=400)
    ap.add_argument("--every", type=int, default=100, help="coarse steps between error samples")
    ap.add_argument("--snapshots", type=int, nargs="+",
                    help="fine steps of the training snapshots (default: every 24 over the run)")
    ap.add_argument("--gain", type=float, default=GAIN)
    ap.add_argument("--dead-zone", type=float, default=DEAD_ZONE)
    args = ap.parse_args()
    t0 = time.perf_counter()
    net, scaling, rep = study(n_fine=args.n_fine, fraction=args.fraction, steps=args.steps,
                              coarse_steps=args.coarse_steps, every=args.every,
                              snapshots=tuple(args.snapshots) if args.snapshots else None,
                              gain=args.gain, dead_zone=args.dead_zone)
    rep["seconds_study"] = time.perf_counter() - t0
    snaps = tuple(args.snapshots) if args.snapshots else dense_snapshots(2 * args.coarse_steps, 96)
    rep["held_out_a_priori"] = held_out_loss(net, args.n_fine, rep["mach"], rep["re"], 9, snaps,
                                             scaling)
    rep["fraction"] = args.fraction
    rep["adam_steps"] = args.steps
    net.close()
    print(json.dumps(rep), flush=True)


if __name__ == "__main__":
    main()
