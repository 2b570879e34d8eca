"""Small, self-contained run of the step kernel for profilers (ncu).

    python -m paper_1505_06900_gb300.profile_step [--n 256] [--storage f32|f16|bf16]
                                                  [--lattice 27|19|9] [--steps 6]
                                                  [--collision rr|reg2|bgk]
                                                  [--closure | --train BATCH]

Initialises a Taylor-Green vortex on an n^3 (D3Q27, D3Q19) or n^2 (D2Q9) periodic
grid, runs `steps` updates through the C ABI and prints the elapsed time. At
n = 256 the D3Q27 FP32 store is 1.8 GB: larger than L2, small enough for a
multi-pass profiler capture.
"""
from __future__ import annotations

import argparse
import time

import numpy as np


def main():
    import torch

    from . import binding as B
    from . import build as build_mod
    from . import workloads as W

    ap = argparse.ArgumentParser()
    ap.add_argument("--n", type=int, default=256)
    ap.add_argument("--lattice", type=int, default=27, choices=[9, 19, 27])
    ap.add_argument("--storage", default="f32", choices=["f32", "f16", "bf16"])
    ap.add_argument("--steps", type=int, default=6)
    ap.add_argument("--collision", default="rr", choices=["rr", "reg2", "bgk"])
    ap.add_argument("--closure", action="store_true",
                    help="run the learned-closure update (D3Q27, FP32) with small random weights")
    ap.add_argument("--train", type=int, default=0, metavar="BATCH",
                    help="instead: `steps` Adam steps of the closure network on a random "
                         "batch of BATCH rows")
    args = ap.parse_args()
    build_mod.build()
    if args.train:
        rng = np.random.default_rng(0)
        X = torch.from_numpy(rng.standard_normal((args.train, 288)).astype(np.float32)).cuda()
        X[:, 270:] = 0
        X = X.to(torch.bfloat16)
        T = torch.from_numpy(rng.standard_normal((args.train, 32)).astype(np.float32)).cuda()
        net = B.MLP((0.05 * rng.standard_normal(B.MLP_PARAMS)).astype(np.float32))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            net.train_step(X, T, 1e-3, want_loss=False)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        print(f"closure network, batch {args.train}: {args.steps} Adam steps in {dt * 1e3:.2f} ms "
              f"(loss {net.train_step(X, T, 1e-3):.6f})")
        net.close()
        return
    storage = {"f32": B.STORE_F32, "f16": B.STORE_F16, "bf16": B.STORE_BF16}[args.storage]
    n = args.n
    if args.lattice != 9:
        shape = (n, n, n)
        rho, u = W.taylor_green_3d(n, 0.1)
        tau = W.taylor_green_3d_tau(n, 0.1)
    else:
        shape = (n, n, 1)
        rho, u = W.taylor_green_2d(n, 0.05)
        tau = W.taylor_green_2d_tau(n, 0.05)
    net = None
    collision = {"rr": B.COLLIDE_RR, "reg2": B.COLLIDE_REG2, "bgk": B.COLLIDE_BGK}[args.collision]
    with B.Solver(args.lattice, shape, tau, storage=storage, collision=collision) as s:
        s.init_fields(torch.from_numpy(rho.astype(np.float32)).cuda(),
                      torch.from_numpy(u.astype(np.float32)).cuda())
        if args.closure:
            rng = np.random.default_rng(0)
            params = (0.02 * rng.standard_normal(B.MLP_PARAMS)).astype(np.float32)
            net = B.MLP(params)
            net.set_scaling(np.zeros(10), np.full(10, 10.0), np.full(17, 1e-6))
            s.set_closure(net, bound=1e6)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        s.step(args.steps)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        d = s.diagnostics()
    if net is not None:
        net.close()
    cells = int(np.prod(shape))
    print(f"lattice D{2 if args.lattice == 9 else 3}Q{args.lattice} {shape} {args.storage} "
          f"{args.collision}: "
          f"{args.steps} steps in {dt * 1e3:.2f} ms ({cells * args.steps / dt / 1e9:.2f} GLUPS), "
          f"mass {d[0]:.6f}")


if __name__ == "__main__":
    main()
