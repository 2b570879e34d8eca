"""Von Neumann linear stability of the oracle's collide-and-stream update (Sec. 3.6).

TEST INFRASTRUCTURE (part of the oracle). The linearised scheme is
f'_i(x + xi_i, t+1) = sum_j Lambda_ij f'_j(x, t) with Lambda the Jacobian of the
post-collision populations Omega_i = f0_i + (1 - 1/tau) f1_i at the uniform
state f = f0(rho, u). For a plane wave of wave vector k the amplification
matrix is A^-1 Lambda with A^-1 = diag(exp(-i k.xi_j)); its eigenvalues lambda
give omega = i log(lambda), whose imaginary part ln|lambda| is the growth rate
per step (a mode is unstable when it is positive).

Lambda is taken by fourth-order central differences of the oracle's C
collision (a rational function of f, so the differences are accurate to about
1e-12); the eigenvalues come from numpy (a library routine).
"""
from __future__ import annotations

import numpy as np

from . import D2Q9, RR, collide_cell, dims_of, feq_cell, lattice_tables


def jacobian(lattice: int, rho: float, u, tau: float, variant: int = RR,
             h: float = 1e-4) -> np.ndarray:
    """d Omega_i / d f_j at f = f0(rho, u)."""
    _, Q = dims_of(lattice)
    f0 = feq_cell(lattice, rho, u)
    J = np.zeros((Q, Q))
    for j in range(Q):
        e = np.zeros(Q)
        e[j] = h
        p1 = collide_cell(lattice, f0 + e, tau, variant)
        m1 = collide_cell(lattice, f0 - e, tau, variant)
        p2 = collide_cell(lattice, f0 + 2 * e, tau, variant)
        m2 = collide_cell(lattice, f0 - 2 * e, tau, variant)
        J[:, j] = (-p2 + 8 * p1 - 8 * m1 + m2) / (12 * h)
    return J


def growth_rates(lattice: int, J: np.ndarray, k) -> np.ndarray:
    """ln|lambda_j| of A^-1 Lambda at wave vector k (length D)."""
    c, _ = lattice_tables(lattice)
    D, _ = dims_of(lattice)
    phase = sum(k[a] * c[:, a] for a in range(D))
    lam = np.linalg.eigvals(np.exp(-1j * phase)[:, None] * J)
    return np.log(np.abs(lam))


def max_growth(lattice: int, u, tau: float, variant: int = RR, nk: int = 97,
               ky_zero: bool = False, rho: float = 1.0):
    """Largest growth rate over a uniform grid of wave vectors in [-pi, pi)^2
    (or over k_y = 0 only); returns (rate, k)."""
    if lattice != D2Q9:
        raise ValueError("the k-map scan is written for D2Q9")
    J = jacobian(lattice, rho, u, tau, variant)
    ks = np.linspace(-np.pi, np.pi, nk, endpoint=False)
    best, arg = -np.inf, None
    for kx in ks:
        for ky in ([0.0] if ky_zero else ks):
            g = growth_rates(lattice, J, (kx, ky)).max()
            if g > best:
                best, arg = g, (kx, ky)
    return best, arg


def growth_map(lattice: int, u, tau: float, variant: int = RR, nk: int = 97,
               rho: float = 1.0) -> np.ndarray:
    """max_j ln|lambda_j| on the uniform nk x nk grid of wave vectors in
    [-pi, pi)^2 (the map of the paper's dissipation figures), shape [nk, nk]."""
    if lattice != D2Q9:
        raise ValueError("the k-map scan is written for D2Q9")
    J = jacobian(lattice, rho, u, tau, variant)
    c, _ = lattice_tables(lattice)
    ks = np.linspace(-np.pi, np.pi, nk, endpoint=False)
    kx, ky = np.meshgrid(ks, ks, indexing="ij")
    phase = kx[..., None] * c[:, 0] + ky[..., None] * c[:, 1]
    M = np.exp(-1j * phase)[..., :, None] * J
    lam = np.linalg.eigvals(M.reshape(-1, J.shape[0], J.shape[0]))
    return np.log(np.abs(lam)).max(axis=-1).reshape(nk, nk)


def onset_velocity(tau: float, nk: int, lo: float = 0.2, hi: float = 0.26,
                   tol: float = 5e-4, threshold: float = 1e-10, variant: int = RR) -> float:
    """Smallest u_x (u_y = 0) at which some wave vector of the nk x nk map has a
    growing mode (max growth rate above `threshold`, which lies above the
    round-off of the numerical Jacobian), by bisection between a stable `lo`
    and an unstable `hi`; returns the upper end of the final bracket."""
    def unstable(ux):
        return growth_map(D2Q9, (ux, 0.0), tau, variant, nk).max() > threshold
    if unstable(lo) or not unstable(hi):
        raise ValueError("the bracket does not contain the onset")
    while hi - lo > tol:
        mid = 0.5 * (lo + hi)
        if unstable(mid):
            hi = mid
        else:
            lo = mid
    return hi
