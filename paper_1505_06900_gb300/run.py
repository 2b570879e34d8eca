"""Run a workload configuration (configs.py) through the library and write
its diagnostics history as JSON lines.

    python -m paper_1505_06900_gb300.run tgv3d --sizes 256 --machs 0.1 --steps 5000 \
        [--every 50] [--storage f16] [--out history.jsonl]
    python -m paper_1505_06900_gb300.run tgv3d_lowprec --compare f32,f16,bf16 [--sizes 512]
    python -m paper_1505_06900_gb300.run --list

One line per sample: step, convective time, mass, momentum, kinetic energy
and enstrophy (all FP64 reductions on the device); then one summary line per
run with the rate of the updates (CUDA events around each lb_step call,
samples excluded) and, for the 2-D Taylor-Green vortex, the viscosity fitted
to the kinetic-energy decay exp(-4 nu k^2 t) against c_s^2 (tau - 1/2).
"""
from __future__ import annotations

import argparse
import json
import math
import sys

import numpy as np

from . import binding as B
from . import configs as C


def convective_time(r: C.Run, step: int) -> float:
    """Time in the flow's own unit: 1 / (U0 k) (tgv2d), L / U0 (shear2d), (N / 2 pi) / U0 (tgv3d)."""
    if r.flow == "tgv2d":
        return step * r.u0 * 2.0 * math.pi / r.n
    if r.flow == "shear2d":
        return step * r.u0 / r.n
    return step * r.u0 / (r.n / (2.0 * math.pi))


def run_one(r: C.Run, emit) -> dict:
    import torch
    tau = r.tau()
    rho, u = r.fields()
    hist = []
    with B.Solver(r.lattice, r.shape, tau, storage=C.STORAGE[r.storage]) as s:
        s.init_fields(torch.from_numpy(rho.astype(np.float32)).cuda(),
                      torch.from_numpy(u.astype(np.float32)).cuda())
        stream = s.stream
        ms, done = 0.0, 0
        while True:
            d = s.diagnostics()
            line = {"config": r.config, "n": r.n, "mach": r.mach, "step": done,
                    "t": convective_time(r, done), "mass": d[0], "momentum": d[1:-1].tolist(),
                    "kinetic_energy": d[-1], "enstrophy": s.enstrophy()}
            hist.append(line)
            emit(line)
            if done >= r.steps:
                break
            k = min(r.every, r.steps - done)
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            s.step(k)
            b.record(stream)
            b.synchronize()
            ms += a.elapsed_time(b)
            done += k
    cells = int(np.prod(r.shape))
    summary = {"config": r.config, "summary": True, "lattice": r.lattice, "n": r.n,
               "mach": r.mach, "re": r.re, "tau": tau, "storage": r.storage, "steps": r.steps,
               "glups": cells * r.steps / (ms * 1e-3) / 1e9 if ms > 0 else None,
               "ke_end_over_start": hist[-1]["kinetic_energy"] / hist[0]["kinetic_energy"]}
    if r.flow == "tgv2d" and len(hist) > 2:
        k = 2.0 * math.pi / r.n
        steps = np.array([h["step"] for h in hist], dtype=np.float64)
        ke = np.array([h["kinetic_energy"] for h in hist], dtype=np.float64)
        slope = np.polyfit(steps, np.log(ke), 1)[0]
        nu_fit, nu = -slope / (4.0 * k * k), (tau - 0.5) / 3.0
        summary.update({"nu_fit": nu_fit, "nu": nu, "nu_rel_error": nu_fit / nu - 1.0})
    emit(summary)
    return summary


def compare_storages(r: C.Run, storages, emit) -> dict:
    """The same run in several storage precisions side by side, in lock step:
    every `every` updates one line per sample with each store's kinetic energy
    and enstrophy and, for every store after the first (the reference, FP32
    normally), the relative L2 difference of its velocity field from the
    reference's; then a summary with the largest differences over the run."""
    import torch
    tau = r.tau()
    rho, u = r.fields()
    rho_d = torch.from_numpy(rho.astype(np.float32)).cuda()
    u_d = torch.from_numpy(u.astype(np.float32)).cuda()
    solvers = [B.Solver(r.lattice, r.shape, tau, storage=C.STORAGE[st]) for st in storages]
    worst = {st: {"u_rel_l2": 0.0, "ke_rel": 0.0, "enstrophy_rel": 0.0} for st in storages[1:]}
    try:
        for s in solvers:
            s.init_fields(rho_d, u_d)
        del rho_d, u_d
        done = 0
        while True:
            line = {"config": r.config, "n": r.n, "mach": r.mach, "step": done,
                    "t": convective_time(r, done)}
            ref_u = None
            ref = {}
            for st, s in zip(storages, solvers):
                d = s.diagnostics()
                ens = s.enstrophy()
                _, uu, _ = s.moments()
                line[st] = {"kinetic_energy": d[-1], "enstrophy": ens, "mass": d[0]}
                if ref_u is None:
                    ref_u, ref = uu, line[st]
                    continue
                du = float(torch.linalg.vector_norm(uu - ref_u) / torch.linalg.vector_norm(ref_u))
                dke = d[-1] / ref["kinetic_energy"] - 1.0
                dens = ens / ref["enstrophy"] - 1.0
                line[st].update({"u_rel_l2_vs_" + storages[0]: du, "ke_rel_vs_" + storages[0]: dke,
                                 "enstrophy_rel_vs_" + storages[0]: dens})
                w = worst[st]
                w["u_rel_l2"] = max(w["u_rel_l2"], du)
                w["ke_rel"] = max(w["ke_rel"], abs(dke))
                w["enstrophy_rel"] = max(w["enstrophy_rel"], abs(dens))
                del uu
            del ref_u
            emit(line)
            if done >= r.steps:
                break
            k = min(r.every, r.steps - done)
            for s in solvers:
                s.step(k)
            done += k
    finally:
        for s in solvers:
            s.close()
    summary = {"config": r.config, "summary": True, "n": r.n, "mach": r.mach, "re": r.re,
               "tau": tau, "steps": r.steps, "reference": storages[0], "max_over_run": worst,
               "final": {st: line[st] for st in storages}}
    emit(summary)
    return summary


def main(argv=None) -> int:
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("config", nargs="?")
    ap.add_argument("--list", action="store_true", help="print the configurations and exit")
    ap.add_argument("--sizes", type=int, nargs="+")
    ap.add_argument("--machs", type=float, nargs="+")
    ap.add_argument("--steps", type=int)
    ap.add_argument("--every", type=int)
    ap.add_argument("--storage", choices=sorted(C.STORAGE))
    ap.add_argument("--compare", help="comma-separated storages run side by side, the first "
                                      "the reference (e.g. f32,f16,bf16)")
    ap.add_argument("--out", help="JSON-lines file (default: stdout)")
    args = ap.parse_args(argv)
    if args.list or not args.config:
        for c in C.CONFIGS.values():
            print(f"{c.name:15s} sizes {c.sizes} machs {c.machs} Re {c.re:g} steps {c.steps} "
                  f"{c.storage}: {c.note}")
        return 0
    runs = C.runs(args.config, sizes=args.sizes, machs=args.machs, steps=args.steps,
                  storage=args.storage, every=args.every)
    fh = open(args.out, "w") if args.out else sys.stdout
    try:
        def emit(obj):
            fh.write(json.dumps(obj) + "\n")
            fh.flush()
        for r in runs:
            if args.compare:
                compare_storages(r, args.compare.split(","), emit)
            else:
                run_one(r, emit)
    finally:
        if args.out:
            fh.close()
    return 0


if __name__ == "__main__":
    sys.exit(main())
