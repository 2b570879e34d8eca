"""The benchmark's workload configurations as data.

Each configuration names a lattice, grid, flow, Mach and Reynolds numbers,
storage and run length; `runs()` expands the Mach and grid sweeps into single
runs that `paper_1505_06900_gb300.run` executes. Flows come from workloads.py
(analytic fields, no dataset):

  tgv2d   2-D Taylor-Green vortex, U0 = 0.05, Re = U0 N / nu
  shear2d periodic double shear layer, U0 = Ma c_s, Re = U0 L / nu, L = N
  tgv3d   3-D Taylor-Green vortex on [0, 2 pi)^3, U0 = Ma c_s, Re = U0 (N / 2 pi) / nu
"""
from __future__ import annotations

import math
from dataclasses import dataclass, replace

from . import binding as B
from . import workloads as W

STORAGE = {"f32": B.STORE_F32, "f16": B.STORE_F16, "bf16": B.STORE_BF16}


@dataclass(frozen=True)
class Config:
    name: str
    lattice: int
    flow: str                      # tgv2d | shear2d | tgv3d
    sizes: tuple                   # grid edge lengths to run (N x N or N^3)
    machs: tuple = (0.1,)          # tgv2d: ignored (U0 = 0.05)
    re: float = 100.0
    steps: int = 1000
    storage: str = "f32"
    every: int = 50                # diagnostics interval (updates)
    note: str = ""


@dataclass(frozen=True)
class Run:
    config: str
    lattice: int
    flow: str
    n: int
    mach: float
    re: float
    steps: int
    storage: str
    every: int

    @property
    def shape(self):
        return (self.n, self.n, 1) if self.flow != "tgv3d" else (self.n,) * 3

    @property
    def u0(self) -> float:
        return 0.05 if self.flow == "tgv2d" else self.mach * math.sqrt(W.CS2)

    def tau(self) -> float:
        if self.flow == "tgv2d":
            return W.taylor_green_2d_tau(self.n, 0.05, self.re)
        if self.flow == "shear2d":
            return W.double_shear_2d_tau(self.n, self.mach, self.re)
        return W.taylor_green_3d_tau(self.n, self.mach, self.re)

    def fields(self):
        """rho [nz, ny, nx] and u [D, nz, ny, nx] of the initial state (float64)."""
        if self.flow == "tgv2d":
            return W.taylor_green_2d(self.n, 0.05)
        if self.flow == "shear2d":
            return W.double_shear_2d(self.n, self.mach)
        return W.taylor_green_3d(self.n, self.mach)


CONFIGS = {
    c.name: c for c in (
        Config("tgv2d_128", B.D2Q9, "tgv2d", (128,), re=100.0, steps=1000,
               note="D2Q9 Taylor-Green vortex, 128^2, Re 100: closed-form decay exp(-2 nu k^2 t)"),
        Config("shear2d_2048", B.D2Q9, "shear2d", (2048,), machs=(0.1, 0.3, 0.5), re=1000.0,
               steps=20000, note="D2Q9 periodic double shear layer, 2048^2, Re 1000"),
        Config("tgv3d", B.D3Q27, "tgv3d", (256, 512), machs=(0.1, 0.5), re=1600.0, steps=5000,
               note="D3Q27 Taylor-Green vortex, Re 1600: kinetic energy and enstrophy history"),
        Config("tgv3d_lowprec", B.D3Q27, "tgv3d", (512,), machs=(0.1,), re=1600.0, steps=5000,
               storage="f16", note="the 512^3 vortex with FP16 (or BF16) shifted storage"),
        Config("tgv3d_d3q19", B.D3Q19, "tgv3d", (512,), machs=(0.1,), re=1600.0, steps=5000,
               note="the 512^3 vortex on D3Q19 (Sec. 5)"),
    )
}


def runs(name: str, *, sizes=None, machs=None, steps=None, storage=None, every=None):
    """The single runs of a configuration, with optional overrides."""
    c = CONFIGS[name]
    if storage is not None:
        c = replace(c, storage=storage)
    out = []
    for n in (sizes or c.sizes):
        for mach in (machs or c.machs):
            out.append(Run(c.name, c.lattice, c.flow, int(n), float(mach), c.re,
                           int(steps if steps is not None else c.steps), c.storage,
                           int(every if every is not None else c.every)))
    return out
