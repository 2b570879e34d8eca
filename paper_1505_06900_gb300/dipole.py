"""Dipole-wall collision benchmark (Sec. 4.1) on the library's walled D2Q9
grids.

    python -m paper_1505_06900_gb300.dipole [--N 125 250 500 1000] [--t-end 0.75]

A dipole (eq_dipole1 / eq_dipole2) in the box [-1, 1]^2 bounded by no-slip
walls, Re = L U / nu = 2500 with L = 1. Lattice: N intervals per unit length
(2N + 1 nodes across, the wall nodes on x, y = +-1), U_lb = 0.01 * 125 / N so
that nu stays fixed while N grows (the paper's convergence series), one time
unit = N / U_lb updates. The enstrophy 0.5 int omega^2 and the kinetic energy
0.5 int |u|^2 are sampled every `sample_dt`; the two local maxima after the
first and second collisions with the right wall are compared with the
reference values 3313 and 1418 printed in the paper (from a spectral
solution). Everything the method computes runs in the library's kernels; this
module only steps, samples and picks maxima.
"""
from __future__ import annotations

import argparse
import json
import time

import numpy as np

from . import binding as B
from . import workloads as W

REFERENCE_PEAKS = (3313.0, 1418.0)
# time windows of the two collisions (dimensionless time)
PEAK_WINDOWS = ((0.2, 0.45), (0.45, 0.8))


def run(N: int, t_end: float = 0.75, sample_dt: float = 0.0025, storage: int = B.STORE_F32,
        collision: int = B.COLLIDE_RR, u_lb: float | None = None):
    import torch
    u_lb = W.dipole_u_lb(N) if u_lb is None else u_lb
    tau = W.dipole_tau(N, u_lb)
    rho, u = W.dipole_2d(N, u_lb)
    n = 2 * N + 1
    steps_per_t = N / u_lb
    total = int(round(t_end * steps_per_t))
    every = max(1, int(round(sample_dt * steps_per_t)))
    hist = []
    with B.Solver(B.D2Q9, (n, n, 1), tau, storage=storage, collision=collision,
                  walls=B.WALL_X | B.WALL_Y) as s:
        s.init_fields(torch.from_numpy(rho.astype(np.float32)).cuda(),
                      torch.from_numpy(u.astype(np.float32)).cuda())
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        done = 0
        while True:
            ens = s.enstrophy() / u_lb ** 2
            ke = s.diagnostics()[-1] / u_lb ** 2 / N ** 2
            hist.append((done / steps_per_t, ens, ke))
            if done >= total:
                break
            k = min(every, total - done)
            s.step(k)
            done += k
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
    t = np.array([h[0] for h in hist])
    om = np.array([h[1] for h in hist])
    peaks = []
    for lo, hi in PEAK_WINDOWS:
        sel = (t >= lo) & (t <= hi)
        k = int(np.argmax(np.where(sel, om, -np.inf)))
        peaks.append((float(t[k]), float(om[k])))
    return {
        "N": N, "nodes": n * n, "u_lb": u_lb, "tau": tau, "steps": total,
        "seconds": wall, "glups": n * n * total / wall / 1e9,
        "omega0": float(om[0]), "energy0": float(hist[0][2]),
        "peaks": [{"t": pt, "enstrophy": pv, "reference": ref, "error": abs(pv - ref) / ref}
                  for (pt, pv), ref in zip(peaks, REFERENCE_PEAKS)],
        "history": [[float(a), float(b), float(c)] for a, b, c in hist],
    }


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--N", type=int, nargs="+", default=[125, 250, 500, 1000])
    ap.add_argument("--t-end", type=float, default=0.75)
    ap.add_argument("--sample-dt", type=float, default=0.0025)
    ap.add_argument("--history", action="store_true", help="include the sampled time series")
    args = ap.parse_args()
    from . import build as build_mod
    build_mod.build()
    for N in args.N:
        r = run(N, args.t_end, args.sample_dt)
        if not args.history:
            r.pop("history")
        print(json.dumps(r), flush=True)


if __name__ == "__main__":
    main()
