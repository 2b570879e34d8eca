"""Seeded synthetic input fields (density and velocity) for the solver.

This module holds no arithmetic of the lattice Boltzmann method itself: it only
evaluates analytic initial flow fields on a cell grid, in double precision,
and returns them as numpy arrays shaped ``rho [nz, ny, nx]`` and
``u [D, nz, ny, nx]`` (x fastest). Both the CUDA path and the CPU oracle take
their inputs from here, cast to float32 first so that the two start from
identical values.

Workloads (lattice units, c_s^2 = 1/3, nu = c_s^2 (tau - 1/2)):
  * ``taylor_green_2d``   u_x = U0 sin(kx) cos(ky), u_y = -U0 cos(kx) sin(ky),
                          rho = 1 - U0^2/(4 c_s^2) (cos 2kx + cos 2ky).
  * ``double_shear_2d``   u_x = U0 tanh(80 (y/L - 1/4)) for y <= L/2, else
                          U0 tanh(80 (3/4 - y/L)); u_y = 0.05 U0 sin(2 pi (x/L + 1/4)); rho = 1.
  * ``taylor_green_3d``   u = U0 (sin x cos y cos z, -cos x sin y cos z, 0) on
                          [0, 2 pi)^3 at cell centres, rho = 1 + U0^2/(16 c_s^2)
                          (cos 2x + cos 2y)(cos 2z + 2), optional phase shift.
  * ``dipole_2d``         the dipole of the dipole-wall benchmark (Sec. 4.1,
                          eq_dipole1 / eq_dipole2) on the nodes of [-1, 1]^2
                          (N intervals per unit length, no-slip walls on the
                          boundary nodes), velocities scaled by U_lb.
  * ``channel_wave``      u_x = U sin(pi y / (ny - 1)) between no-slip walls on
                          the first and last y planes, the slowest decaying
                          Stokes mode of the channel.
  * ``random_field``      rho = 1 + a_rho * N(0,1), u = a_u * N(0,1), seeded:
                          a field with every Fourier mode present, for parity
                          tests that must exercise all index paths.
"""
from __future__ import annotations

import math

import numpy as np

CS2 = 1.0 / 3.0


def _grid(nx, ny, nz):
    z, y, x = np.meshgrid(np.arange(nz, dtype=np.float64), np.arange(ny, dtype=np.float64),
                          np.arange(nx, dtype=np.float64), indexing="ij")
    return x, y, z


def taylor_green_2d(n: int, u0: float = 0.05, nx: int | None = None):
    """2D Taylor-Green vortex on an n x n periodic grid, k = 2 pi / n."""
    nx = nx or n
    x, y, _ = _grid(nx, n, 1)
    kx, ky = 2.0 * math.pi / nx, 2.0 * math.pi / n
    ux = u0 * np.sin(kx * x) * np.cos(ky * y)
    uy = -u0 * np.cos(kx * x) * np.sin(ky * y)
    rho = 1.0 - u0 * u0 / (4.0 * CS2) * (np.cos(2 * kx * x) + np.cos(2 * ky * y))
    return rho, np.stack([ux, uy])


def taylor_green_2d_tau(n: int, u0: float = 0.05, re: float = 100.0) -> float:
    """tau for Re = U0 n / nu."""
    return 0.5 + (u0 * n / re) / CS2


def double_shear_2d(n: int, mach: float = 0.1):
    """Periodic double shear layer on an n x n grid with U0 = Ma c_s."""
    u0 = mach * math.sqrt(CS2)
    x, y, _ = _grid(n, n, 1)
    L = float(n)
    ux = np.where(y <= L / 2, u0 * np.tanh(80.0 * (y / L - 0.25)),
                  u0 * np.tanh(80.0 * (0.75 - y / L)))
    uy = 0.05 * u0 * np.sin(2.0 * math.pi * (x / L + 0.25))
    rho = np.ones_like(x)
    return rho, np.stack([ux, uy])


def double_shear_2d_tau(n: int, mach: float = 0.1, re: float = 1000.0) -> float:
    u0 = mach * math.sqrt(CS2)
    return 0.5 + (u0 * n / re) / CS2


def taylor_green_3d(n: int, mach: float = 0.1, phase=(0.0, 0.0, 0.0)):
    """3D Taylor-Green vortex on [0, 2 pi)^3 sampled at cell centres. The
    factors of each axis are evaluated once on a 1-D array and broadcast."""
    u0 = mach * math.sqrt(CS2)
    h = 2.0 * math.pi / n
    c = (np.arange(n, dtype=np.float64) + 0.5) * h
    X = (c + phase[0])[None, None, :]
    Y = (c + phase[1])[None, :, None]
    Z = (c + phase[2])[:, None, None]
    ux = u0 * np.sin(X) * np.cos(Y) * np.cos(Z)
    uy = -u0 * np.cos(X) * np.sin(Y) * np.cos(Z)
    uz = np.zeros_like(ux)
    rho = 1.0 + u0 * u0 / (16.0 * CS2) * (np.cos(2 * X) + np.cos(2 * Y)) * (np.cos(2 * Z) + 2.0)
    return rho, np.stack([ux, uy, uz])


def taylor_green_3d_tau(n: int, mach: float = 0.1, re: float = 1600.0) -> float:
    """tau for Re = U0 L / nu with L = n / (2 pi) cells."""
    u0 = mach * math.sqrt(CS2)
    nu = u0 * (n / (2.0 * math.pi)) / re
    return 0.5 + nu / CS2


# Dipole-wall benchmark (Sec. 4.1): core vorticity, monopole radius and
# centres printed in the paper; Re = L U / nu = 2500 with L = 1 (half width).
DIPOLE_OMEGA_E = 299.5286
DIPOLE_R0 = 0.1
DIPOLE_CENTRES = ((0.0, 0.1), (0.0, -0.1))
DIPOLE_RE = 2500.0


def dipole_velocity(x, y):
    """Dimensionless dipole velocity (u_x, u_y) at points (x, y) (eq_dipole1,
    eq_dipole2): monopole 1 (positive core vorticity) at (0, 0.1), monopole 2
    (negative) at (0, -0.1)."""
    (x1, y1), (x2, y2) = DIPOLE_CENTRES
    we, r0 = DIPOLE_OMEGA_E, DIPOLE_R0
    e1 = np.exp(-((x - x1) ** 2 + (y - y1) ** 2) / r0 ** 2)
    e2 = np.exp(-((x - x2) ** 2 + (y - y2) ** 2) / r0 ** 2)
    ux = -0.5 * we * (y - y1) * e1 + 0.5 * we * (y - y2) * e2
    uy = 0.5 * we * (x - x1) * e1 - 0.5 * we * (x - x2) * e2
    return ux, uy


def dipole_2d(N: int, u_lb: float | None = None):
    """Nodes x_i = -1 + i / N, i = 0 .. 2N, in both directions (the wall nodes
    lie on x, y = +-1); rho = 1 and u = U_lb * (dipole velocity), zero on the
    wall nodes. U_lb defaults to 0.01 * 125 / N (the paper's convergence series
    at constant nu)."""
    u_lb = dipole_u_lb(N) if u_lb is None else u_lb
    n = 2 * N + 1
    X = -1.0 + np.arange(n) / N
    x, y = np.meshgrid(X, X, indexing="xy")
    ux, uy = dipole_velocity(x, y)
    u = np.zeros((2, 1, n, n))
    u[0, 0], u[1, 0] = u_lb * ux, u_lb * uy
    u[:, 0, 0, :] = u[:, 0, -1, :] = u[:, 0, :, 0] = u[:, 0, :, -1] = 0.0
    return np.ones((1, n, n)), u


def dipole_u_lb(N: int) -> float:
    return 0.01 * 125.0 / N


def dipole_tau(N: int, u_lb: float | None = None) -> float:
    u_lb = dipole_u_lb(N) if u_lb is None else u_lb
    return 0.5 + (u_lb * N / DIPOLE_RE) / CS2


def channel_wave(nx: int, ny: int, nz: int, u0: float, dims: int = 2):
    """u_x = u0 sin(pi y / (ny - 1)) on nodes y = 0 .. ny - 1 (zero on both wall
    planes), rho = 1."""
    y = np.arange(ny)
    u = np.zeros((dims, nz, ny, nx))
    u[0] = u0 * np.sin(np.pi * y / (ny - 1))[None, :, None]
    return np.ones((nz, ny, nx)), u


def random_field(shape, dims: int, seed: int, a_rho: float = 0.01, a_u: float = 0.05):
    """Seeded random density/velocity field of shape (nx, ny, nz)."""
    nx, ny, nz = shape
    rng = np.random.default_rng(seed)
    rho = 1.0 + a_rho * rng.standard_normal((nz, ny, nx))
    u = a_u * rng.standard_normal((dims, nz, ny, nx))
    return rho, u


def random_populations(q: int, shape, seed: int, amp: float = 0.02):
    """Seeded random shifted populations df [Q, nz, ny, nx] of relative size amp.

    Each df_i is drawn as amp * N(0,1) scaled by a weight-like factor 6^-(number
    of non-zero velocity components), so that f_i = w_i + df_i stays positive.
    The weights themselves are not needed here (the caller adds them)."""
    nx, ny, nz = shape
    rng = np.random.default_rng(seed)
    df = amp * rng.standard_normal((q, nz, ny, nx))
    d = 2 if q == 9 else 3
    for i in range(q):
        nnz = sum(1 for a in range(d) if (i // 3 ** a) % 3 != 1)
        df[i] *= (2.0 / 3.0) ** (d - nnz) * (1.0 / 6.0) ** nnz
    return df


def as_f32(*arrays):
    """Round to float32 and back to float64, so both sides see identical inputs."""
    out = tuple(np.asarray(a, dtype=np.float32).astype(np.float64) for a in arrays)
    return out if len(out) > 1 else out[0]
