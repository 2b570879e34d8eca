"""Throughput of the recursive-regularized BGK collide-and-stream step on GB300.

Default workload (N=1): D3Q27 recursive-regularized BGK, FP32 storage, fully
periodic 512^3 Taylor-Green vortex (Ma = 0.1, Re = 1600), AA-pattern store in
HBM (14.5 GB, far larger than L2). One timed "step" is one full update of the
grid (gather, moments, recursive reconstruction, collision, scatter), with the
FP64 mass/momentum/energy reduction every 50 steps. Prints one JSON line:
GLUPS (10^9 cell updates per second), the HBM roofline of the step kernel, an
end-to-end figure through host buffers, FP16/BF16 storage variants, and the
FP64 CPU oracle timed on the host cores on a bounded sample.

Multi-GPU: replicas only. Each rank runs its own 512^3 domain (the path has no
data exchange between replicas), so the figure is weak scaling.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--n 512] [--impl reference]
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "GLUPS & %HBM roofline, D3Q27 RR: FP32 vs FP16-store vs learned at fixed error"
UNIT = "GLUPS"
DIAG_EVERY = 50
MACH, RE = 0.1, 1600.0
U_ERROR_UPDATES = 1000   # updates after which the 16-bit forms' u error is taken
RATED_HBM_GBS = 7900.0   # nominal GB300 HBM3e bandwidth, beside the measured copy peak

# DRAM traffic of one step-kernel launch from an ncu capture (dram__bytes_read.sum
# + dram__bytes_write.sum), keyed by the sha256 of the kernel sources it was
# taken on; reported as null when the sources have changed since.
# The 512^3 launch is too large for a multi-pass capture; the value is the
# capture of the same kernel at 256^3 (mean of the even and odd launches,
# 3,564,379,136 B, 212.45 B per cell) scaled by the cell count, since the
# traffic per cell does not depend on the grid size for this streaming kernel.
TRAFFIC = {
    "d3q27_f32_512": {"kernel_sha": "a3ad16e41d5d7862", "bytes_per_launch": 28515033088,
                      "source": "ncu capture at 256^3 (mean of the even and odd launches) x 8"},
}

KERNEL_SOURCES = ["paper_1505_06900_gb300/csrc/lbrr_step.cu",
                  "paper_1505_06900_gb300/csrc/lbrr_device.cuh"]


def kernel_sha() -> str:
    h = hashlib.sha256()
    for p in KERNEL_SOURCES:
        with open(os.path.join(ROOT, p), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def log(*a):
    print(*a, file=sys.stderr, flush=True)


# ------------------------------------------------------------------ clocks --
class ClockSampler:
    """nvidia-smi sampling of SM clock and throttle reasons, every 50 ms, over the
    whole GPU arm; each sample carries its host time, so a summary can be taken
    over the timed region alone (mark() brackets it) and over the arm."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
    PERIOD_MS = 50

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.samples = []  # (host time, line)
        self.regions = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", str(self.PERIOD_MS)],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self._t = threading.Thread(target=self._read, daemon=True)
            self._t.start()
        except (OSError, ValueError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.samples.append((time.monotonic(), line.strip()))

    def mark(self, t0: float, t1: float):
        """Record a timed region [t0, t1] (host monotonic seconds)."""
        self.regions.append((t0, t1))

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    @staticmethod
    def _summarise(lines):
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax = float(parts[2])
            except ValueError:
                continue
            for name, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        loaded = [s for s in sm if smax and s > 0.5 * smax] or sm
        return {"sm_mhz": statistics.median(loaded), "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}

    def summary(self):
        """Summary over the marked timed regions (samples taken while one was
        running, widened by half a period at each end), plus the whole arm."""
        half = 0.5 * self.PERIOD_MS / 1e3
        inside = [ln for t, ln in self.samples
                  if any(a - half <= t <= b + half for a, b in self.regions)]
        out = self._summarise(inside)
        out["period_ms"] = self.PERIOD_MS
        out["arm"] = self._summarise([ln for _, ln in self.samples])
        return out


# --------------------------------------------------------------- distributed --
def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def init_dist(ws, backend):
    import torch.distributed as dist
    if ws > 1 and not dist.is_initialized():
        dist.init_process_group(backend=backend)
    return dist if ws > 1 else None


def max_over_ranks(dist, values, device):
    """Element-wise maximum of a list of floats over all ranks (the slowest
    rank sets the job's time); the values themselves with no process group."""
    import torch
    t = torch.tensor(values, dtype=torch.float64, device=device)
    if dist:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return t.tolist()


def job_glups(world_size, cells_per_rank, steps, total_ms):
    """Whole-job rate: the cell updates of all ranks over the slowest rank's time."""
    return world_size * cells_per_rank * steps / (total_ms * 1e-3) / 1e9


# -------------------------------------------------------------- reference --
def oracle_sample(steps: int, warmup: int, n_sample: int, threads: int | None = None):
    """Time the FP64 CPU oracle on a D3Q27 Taylor-Green vortex of n_sample^3
    cells (a bounded sample of the 512^3 workload, same Ma and Re scaling)."""
    import oracle as O
    from paper_1505_06900_gb300 import workloads as W
    O.build()
    if threads:
        O.set_num_threads(threads)
    shape = (n_sample,) * 3
    tau = W.taylor_green_3d_tau(n_sample, MACH, RE)
    rho, u = W.as_f32(*W.taylor_green_3d(n_sample, MACH))
    f = O.init(O.D3Q27, shape, tau, rho, u)
    if warmup:
        f = O.step(O.D3Q27, shape, tau, f, warmup)
    t0 = time.perf_counter()
    O.step(O.D3Q27, shape, tau, f, steps)
    dt = time.perf_counter() - t0
    cells = n_sample ** 3
    return {"value": cells * steps / dt / 1e9, "unit": UNIT, "cores": O.num_threads(),
            "kind": "oracle", "seconds": dt,
            "sample": f"D3Q27 Taylor-Green {n_sample}^3 (Ma {MACH}, Re {RE:g}), {steps} "
                      f"oracle updates, FP64, OpenMP over cells"}


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    # the same sample grid as the GPU arm's cpu_baseline (a 1/64 sample of 512^3)
    n_sample = args.cpu_sample
    res = oracle_sample(args.steps, args.warmup, n_sample)
    line = {
        "impl": "reference", "metric": METRIC, "value": res["value"], "unit": UNIT,
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * res["seconds"] / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": f"D3Q27 RR Taylor-Green {n_sample}^3 sample of the 512^3 "
                               f"workload (FP64 CPU oracle)", "lattice": "D3Q27",
                   "grid": [n_sample] * 3, "parallelism": "replicas"},
        "cpu_baseline": {k: res[k] for k in ("value", "unit", "cores", "kind", "sample")},
        "e2e": {"value": res["value"], "unit": UNIT, "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------------- GPU arm --
def time_variant(B, torch, n, storage, steps, warmup, tau, rho_d, u_d, diag_every, stream,
                 sync_all, sampler=None, u_at=None, closure=None, lattice=None,
                 dead_zone=0.0):
    """Warm up, then time `steps` updates with the diagnostics reduction every
    `diag_every` updates inside the timed region; returns timing and per-launch
    data. With u_at, the run then continues (untimed) to u_at updates in all
    and returns the velocity field there. Lattice D3Q27 unless given."""
    lattice = B.D3Q27 if lattice is None else lattice
    s = B.Solver(lattice, (n, n, n), tau, storage=storage, stream=stream)
    try:
        s.init_fields(rho_d, u_d)
        diag0 = s.diagnostics()
        if closure is not None:
            s.set_closure(closure, dead_zone=dead_zone)
        s.step(warmup)
        for _ in range(max(1, warmup // diag_every)):
            s.diagnostics()
        torch.cuda.synchronize()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(steps)]
        t_start = torch.cuda.Event(enable_timing=True)
        t_end = torch.cuda.Event(enable_timing=True)
        sync_all()
        torch.cuda.synchronize()
        launches = 0
        diag_calls = 0
        h0 = time.monotonic()
        with torch.cuda.stream(stream):
            t_start.record(stream)
            for k in range(steps):
                ev[k][0].record(stream)
                s.step(1)
                ev[k][1].record(stream)
                launches += 1
                if (k + 1) % diag_every == 0:
                    s.diagnostics()
                    launches += 2
                    diag_calls += 1
            t_end.record(stream)
        torch.cuda.synchronize()
        if sampler is not None:
            sampler.mark(h0, time.monotonic())
        sync_all()
        total_ms = t_start.elapsed_time(t_end)
        kern_ms = [a.elapsed_time(b) for a, b in ev]
        diag = s.diagnostics()
        out = {"total_ms": total_ms, "kernel_ms": statistics.mean(kern_ms),
               "kernel_ms_median": statistics.median(kern_ms), "launches": launches,
               "diag_calls": diag_calls, "diag": diag.tolist(), "diag0": diag0.tolist(),
               "bytes_per_update": s.info()["bytes_per_update"]}
        if u_at is not None:
            s.step(max(0, u_at - warmup - steps))
            out["u"] = s.moments()[1]
            out["diag_u_at"] = s.diagnostics().tolist()
        if closure is not None:
            out["fallbacks"] = s.closure_fallbacks()
        return out
    finally:
        s.close()


def ke_decay_vs(r, ref, key="diag") -> float:
    """Kinetic energy lost over the run (start minus end) relative to that of
    the reference run, minus one."""
    return (r["diag0"][-1] - r[key][-1]) / (ref["diag0"][-1] - ref[key][-1]) - 1.0


def rel_l2(torch, a, b) -> float:
    return float(torch.linalg.vector_norm(a - b) / torch.linalg.vector_norm(b))


# Algorithmic cost of one closure update per coarse cell: the populations read
# and written (216 B) plus a BF16 moment field of 10 channels written once and
# read once for the 3^3 gather (40 B); the network's padded BF16 products
# 2 (288 x 64 + 64 x 64 + 64 x 32) flops.
CLOSURE_BYTES_PER_CELL = 256
CLOSURE_FLOP_PER_CELL = 2 * (288 * 64 + 64 * 64 + 64 * 32)


def learned_variant(B, torch, n_coarse, steps, warmup, stream, sync_all, fine_ms_per_step,
                    sampler=None):
    """The learned-closure recipe at the configuration's sizes: fine
    (2 n_coarse)^3 Taylor-Green runs (Ma 0.3, Re 1600) of four seeded phases,
    17 snapshots each up to t = 6.8, give the training data, the network is
    trained by the library's kernels, and the coarse runs with and without it
    start from the held-out phase's filtered state and are judged against its
    filtered fine run over 1600 coarse steps (t = 6.8: the 256^3 grid
    resolves the vortex at first and under-resolves it from t ~ 4 on). Then
    the closure step is timed on the n_coarse^3 grid (one coarse step stands
    for two fine steps) next to plain RR on the same grid."""
    from paper_1505_06900_gb300 import closure as CL
    from paper_1505_06900_gb300 import workloads as W
    n_fine, coarse_steps, seeds = 2 * n_coarse, 1600, range(1, 5)
    t0 = time.perf_counter()
    net, scaling, rep = CL.study(n_fine=n_fine, steps=1500, coarse_steps=coarse_steps,
                                 train_seeds=seeds,
                                 snapshots=CL.dense_snapshots(2 * coarse_steps, 192),
                                 fraction=min(0.25, 2.5e6 / (n_coarse ** 3 * 17 * len(seeds))),
                                 every=200)
    train_s = time.perf_counter() - t0
    tau_c = CL.coarse_tau(W.taylor_green_3d_tau(n_fine, MACH, RE))
    rho, u = W.taylor_green_3d(n_coarse, MACH)
    rho_d = torch.from_numpy(rho.astype(np.float32)).cuda()
    u_d = torch.from_numpy(u.astype(np.float32)).cuda()
    diag_every = min(DIAG_EVERY, steps)
    ml = time_variant(B, torch, n_coarse, B.STORE_F32, steps, warmup, tau_c, rho_d, u_d,
                      diag_every, stream, sync_all, sampler, closure=net,
                      dead_zone=CL.DEAD_ZONE)
    rr = time_variant(B, torch, n_coarse, B.STORE_F32, steps, warmup, tau_c, rho_d, u_d,
                      diag_every, stream, sync_all, sampler)
    cells = n_coarse ** 3
    ms_ml = ml["total_ms"] / steps
    ms_rr = rr["total_ms"] / steps
    net.close()
    peaks = _peaks()
    gbs = CLOSURE_BYTES_PER_CELL * cells / (ms_ml * 1e-3) / 1e9
    tfs = CLOSURE_FLOP_PER_CELL * cells / (ms_ml * 1e-3) / 1e12
    return {
        "value": cells * steps / (ml["total_ms"] * 1e-3) / 1e9, "unit": "GLUPS (coarse cells)",
        "grid": [n_coarse] * 3, "ms_per_coarse_step": ms_ml,
        "kernels_per_step": 2,
        "kernels": "feature source (moments, BF16, padded), TMA-fed tcgen05 network fused with "
                   "the corrected RR update",
        "roofline_frac": gbs / float(peaks.get("hbm_gbs", 6800.0)),
        "tensor_frac": tfs / float(peaks.get("bf16_tflops_sustained", 1700.0)),
        "speedup_vs_fine_f32_equal_time": 2.0 * fine_ms_per_step / ms_ml,
        "coarse_rr": {"ms_per_coarse_step": ms_rr,
                      "speedup_vs_fine_f32_equal_time": 2.0 * fine_ms_per_step / ms_rr},
        "fallback_cell_updates": ml["fallbacks"],
        "u_error_vs_filtered_fine": rep["err_closure"],
        "coarse_rr_u_error_vs_filtered_fine": rep["err_rr"],
        "u_error_history": rep["history"],
        "error_sizes": f"D3Q27 Taylor-Green Ma {rep['mach']} Re {rep['re']:g}, fine "
                       f"{n_fine}^3 -> coarse {n_coarse}^3, held-out phase (seed 9), "
                       f"{coarse_steps} coarse steps; history: (coarse steps, coarse RR, "
                       f"closure) relative L2 of u",
        "training": {"samples": rep["samples"], "loss_first": rep["loss_first"],
                     "loss_last": rep["loss_last"], "seconds": train_s,
                     "gain": rep["gain"], "dead_zone": rep["dead_zone"],
                     "fallbacks_in_evaluation": rep["fallbacks"]},
    }


def shear_variant(B, torch, stream, peak_gbs, n: int = 2048, steps: int = 20000,
                  machs=(0.1, 0.3, 0.5)):
    """The periodic D2Q9 double shear layer at n^2 (Re 1000 on L = n), FP32 store: the
    updates of a whole run timed with CUDA events on the solver's stream (lb_step
    replays captured graphs of 8 updates), for each Mach number; the kinetic energy
    at the end against the start (finite: the run stayed stable)."""
    from paper_1505_06900_gb300 import workloads as W
    out = {"grid": [n, n], "steps": steps, "re": 1000.0, "bytes_per_update": 72, "runs": {}}
    for mach in machs:
        rho, u = W.double_shear_2d(n, mach)
        tau = W.double_shear_2d_tau(n, mach)
        with B.Solver(B.D2Q9, (n, n, 1), tau, stream=stream) as s:
            s.init_fields(torch.from_numpy(rho.astype(np.float32)).cuda(),
                          torch.from_numpy(u.astype(np.float32)).cuda())
            e0 = s.diagnostics()[-1]
            s.step(24)
            torch.cuda.synchronize()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            s.step(steps)
            b.record(stream)
            torch.cuda.synchronize()
            ms = a.elapsed_time(b)
            e1 = s.diagnostics()[-1]
        gbs = 72.0 * n * n * steps / (ms * 1e-3) / 1e9
        out["runs"][f"ma{mach}"] = {"tau": tau, "glups": n * n * steps / (ms * 1e-3) / 1e9,
                                    "kernel_gbs": gbs, "roofline_frac": gbs / peak_gbs,
                                    "ms": ms, "ke_end_over_start": e1 / e0}
    return out


def dipole_variant(B, N: int = 500):
    """The dipole-wall collision (walls, D2Q9, Re 2500) at N = 500 with each
    storage precision: the two enstrophy maxima against the reference values
    the paper prints, i.e. the error each store reaches on a physical
    benchmark, and the update rate (enstrophy sampling included)."""
    from paper_1505_06900_gb300 import dipole
    out = {"N": N, "nodes": (2 * N + 1) ** 2, "reference": list(dipole.REFERENCE_PEAKS)}
    for name, st in (("f32", B.STORE_F32), ("f16", B.STORE_F16), ("bf16", B.STORE_BF16)):
        r = dipole.run(N, t_end=0.75, storage=st)
        out[name] = {"glups": r["glups"], "steps": r["steps"],
                     "peaks": [p["enstrophy"] for p in r["peaks"]],
                     "errors": [p["error"] for p in r["peaks"]]}
    return out


def _peaks() -> dict:
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return json.load(fh)
    except OSError:
        return {}


class _Null:
    def __enter__(self):
        return self

    def __exit__(self, *a):
        return False


def run_gpu(args):
    import torch

    from paper_1505_06900_gb300 import binding as B
    from paper_1505_06900_gb300 import build as build_mod
    from paper_1505_06900_gb300 import workloads as W

    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    dist = init_dist(ws, "nccl")

    def sync_all():
        if dist:
            dist.barrier()

    if rank == 0:
        build_mod.build()
    sync_all()
    B.load()

    n = args.n
    tau = W.taylor_green_3d_tau(n, MACH, RE)
    rho, u = W.taylor_green_3d(n, MACH)
    rho32 = np.ascontiguousarray(rho, dtype=np.float32)
    u32 = np.ascontiguousarray(u, dtype=np.float32)
    rho_d = torch.from_numpy(rho32).cuda()
    u_d = torch.from_numpy(u32).cuda()
    stream = torch.cuda.Stream()
    cells = n ** 3

    # the diagnostics reduction runs inside every timed region, at least once
    diag_every = min(DIAG_EVERY, args.steps)
    # the 16-bit and D3Q19 forms are compared with the FP32 run after the same
    # number of updates, at least 1000 whatever --steps is
    n_cmp = max(U_ERROR_UPDATES, args.warmup + args.steps)
    single = ws == 1
    sampler = ClockSampler(local)
    with sampler:
        main = time_variant(B, torch, n, B.STORE_F32, args.steps, args.warmup, tau, rho_d, u_d,
                            diag_every, stream, sync_all, sampler,
                            u_at=n_cmp if single else None)
        u_f32 = main.pop("u", None)
        # end to end through host buffers (pinned), one lb_run_host call of K steps,
        # right after the device-timed run it is compared with
        rho_h = torch.from_numpy(rho32).pin_memory()
        u_h = torch.from_numpy(u32).pin_memory()
        rho_o = torch.empty_like(rho_h).pin_memory()
        u_o = torch.empty_like(u_h).pin_memory()
        diag_h = np.zeros(5)
        with B.Solver(B.D3Q27, (n, n, n), tau, stream=stream) as s:
            s.run_host(rho_h, u_h, 2, rho_out=rho_o, u_out=u_o, diag_out=diag_h)  # warm-up
            sync_all()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            s.run_host(rho_h, u_h, args.steps, rho_out=rho_o, u_out=u_o, diag_out=diag_h)
            e2e_s = time.perf_counter() - t0
            sync_all()
        h2d = (rho32.nbytes + u32.nbytes)
        d2h = (rho32.nbytes + u32.nbytes) + diag_h.nbytes
        del rho_h, u_h, rho_o, u_o

        # the storage, lattice and closure variants and the other workloads belong to
        # the single-GPU line; a multi-GPU run times the headline workload only
        variants = {}
        if single:
            peak_gbs = float(_peaks().get("hbm_gbs", 6800.0))
            for name, st in (("f16", B.STORE_F16), ("bf16", B.STORE_BF16)):
                r = time_variant(B, torch, n, st, args.steps, args.warmup, tau, rho_d, u_d,
                                 diag_every, stream, sync_all, sampler, u_at=n_cmp)
                kgbs = r["bytes_per_update"] * cells / (r["kernel_ms"] * 1e-3) / 1e9
                variants[name] = {
                    "value": cells * args.steps / (r["total_ms"] * 1e-3) / 1e9, "unit": UNIT,
                    "bytes_per_update": r["bytes_per_update"], "kernel_gbs": kgbs,
                    "roofline_frac": kgbs / peak_gbs,
                    "roofline_frac_rated": kgbs / RATED_HBM_GBS,
                    "speedup_vs_f32": main["total_ms"] / r["total_ms"],
                    "u_error_vs_f32": rel_l2(torch, r.pop("u"), u_f32),
                    "u_error_updates": n_cmp,
                    "ke_decay_vs_f32": ke_decay_vs(r, main, "diag_u_at"),
                    "u_error_note": f"relative L2 of u against the FP32 store after {n_cmp} "
                                    "updates from the same initial state",
                }
            # D3Q19 (Sec. 5): 19 populations per cell, the same flow and tau
            for name, st in (("d3q19_f32", B.STORE_F32), ("d3q19_f16", B.STORE_F16)):
                r = time_variant(B, torch, n, st, args.steps, args.warmup, tau, rho_d, u_d,
                                 diag_every, stream, sync_all, sampler, u_at=n_cmp,
                                 lattice=B.D3Q19)
                kgbs = r["bytes_per_update"] * cells / (r["kernel_ms"] * 1e-3) / 1e9
                variants[name] = {
                    "value": cells * args.steps / (r["total_ms"] * 1e-3) / 1e9, "unit": UNIT,
                    "bytes_per_update": r["bytes_per_update"], "kernel_gbs": kgbs,
                    "roofline_frac": kgbs / peak_gbs,
                    "speedup_vs_d3q27_f32": main["total_ms"] / r["total_ms"],
                    "u_diff_vs_d3q27_f32": rel_l2(torch, r.pop("u"), u_f32),
                    "u_diff_updates": n_cmp,
                    "ke_decay_vs_d3q27_f32": ke_decay_vs(r, main, "diag_u_at"),
                    "u_diff_note": f"relative L2 of u against the D3Q27 FP32 run after {n_cmp} "
                                   "updates, same init (lattice + storage difference)",
                }
            del u_f32
            # context for the decay ratios: the share of its kinetic energy the FP32 run
            # loses over the compared updates (the 512^3 Taylor-Green vortex decays slowly)
            ke0, ke1 = main["diag0"][-1], main["diag_u_at"][-1]
            variants["ke_loss_fraction_f32"] = (ke0 - ke1) / ke0
            variants["learned"] = learned_variant(B, torch, n // 2, args.steps, args.warmup,
                                                  stream, sync_all, main["total_ms"] / args.steps,
                                                  sampler)
            variants["dipole_wall"] = dipole_variant(B)
            variants["d2q9_shear_2048"] = shear_variant(B, torch, stream, peak_gbs)

    total_ms, kernel_ms, e2e_s = max_over_ranks(dist, [main["total_ms"], main["kernel_ms"], e2e_s],
                                                "cuda")

    if rank != 0:
        return 0

    peaks = _peaks()
    if "hbm_gbs" in peaks:
        peak, peak_src = float(peaks["hbm_gbs"]), "measured"
    else:
        peak, peak_src = 6800.0, "fallback"
    bpu = main["bytes_per_update"]
    achieved = bpu * cells / (kernel_ms * 1e-3) / 1e9
    sha = kernel_sha()
    tr = TRAFFIC.get(f"d3q27_f32_{n}")
    traffic = tr["bytes_per_launch"] if tr and tr.get("kernel_sha") == sha else None

    # the CPU oracle is timed beside the single-GPU run only: on all host cores
    # and on one core, on the same sample grid
    cpu = None
    if single:
        cpu = oracle_sample(steps=args.cpu_steps, warmup=0, n_sample=args.cpu_sample)
        one = oracle_sample(steps=args.cpu_steps_single, warmup=0, n_sample=args.cpu_sample,
                            threads=1)
        cpu = {k: cpu[k] for k in ("value", "unit", "cores", "kind", "sample")}
        cpu["single_thread"] = {k: one[k] for k in ("value", "unit", "cores", "sample")}
    clocks = sampler.summary()
    value = job_glups(ws, cells, args.steps, total_ms)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {
            "workload": f"D3Q27 recursive-regularized BGK, FP32 AA store, periodic {n}^3 "
                        f"Taylor-Green vortex Ma={MACH} Re={RE:g}",
            "lattice": "D3Q27", "grid": [n, n, n], "storage": "f32", "tau": tau,
            "diag_every": diag_every, "diag_calls_timed": main["diag_calls"],
            "bytes_per_update": bpu,
            "l2": f"inputs larger than L2 ({bpu // 2 * cells / 1e9:.1f} GB store)",
            "parallelism": "replicas" if ws > 1 else "single",
        },
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": traffic,
                     "traffic_source": tr["source"] if traffic else None,
                     "kernel": "rr_step_kernel<27,f32,RR>", "peak_source": peak_src,
                     "frac_rated": achieved / RATED_HBM_GBS, "peak_rated": RATED_HBM_GBS,
                     "peak_rated_source": "nominal GB300 HBM3e bandwidth",
                     "kernel_ms": kernel_ms, "algorithmic_bytes_per_launch": bpu * cells},
        "variants": variants,
        "e2e": {"value": job_glups(ws, cells, args.steps, e2e_s * 1e3), "unit": UNIT,
                "h2d_bytes_per_step": h2d / args.steps, "d2h_bytes_per_step": d2h / args.steps,
                "scope": "lb_run_host: pinned upload of rho,u, init, K updates, download of "
                         "rho,u and diagnostics"},
        "cpu_baseline": cpu,
        "gpu_launches": main["launches"],
        "clocks": clocks,
        "kernel_sha": sha,
        "diagnostics_end": main["diag"],
    }
    # the three forms of the metric, where the driver's parser sees them
    for name in ("f16", "bf16", "learned"):
        if name in variants:
            line[name] = summary_of(name, variants[name])
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()
    return 0


def summary_of(name, v):
    """The compact record of one form of the metric (FP16 / BF16 store, learned
    closure): its rate, its velocity error and its roofline fraction."""
    if name == "learned":
        return {k: v.get(k) for k in ("value", "unit", "u_error_vs_filtered_fine",
                                      "coarse_rr_u_error_vs_filtered_fine",
                                      "speedup_vs_fine_f32_equal_time", "roofline_frac",
                                      "tensor_frac", "ms_per_coarse_step", "error_sizes")}
    return {k: v[k] for k in ("value", "unit", "u_error_vs_f32", "u_error_updates",
                              "roofline_frac", "roofline_frac_rated", "speedup_vs_f32",
                              "bytes_per_update")}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--n", type=int, default=512)
    ap.add_argument("--cpu-sample", type=int, default=128)
    ap.add_argument("--cpu-steps", type=int, default=50)
    ap.add_argument("--cpu-steps-single", type=int, default=4)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.impl == "reference":
        return run_reference(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
