"""FP64 reference of the learned closure (test infrastructure, part of the oracle).

The paper has no learned component; this module is the plain reference of
the learned-closure extension built around the RR step:

* coarsening: 2 x 2 x 2 box average of fine populations (one coarse cell per
  eight fine cells, Delta x and Delta t doubled: acoustic scaling, the coarse
  relaxation time is 1/2 + (tau_fine - 1/2)/2);
* features of a coarse cell: the ten moments (rho - 1, u, Pi1 in the order
  xx, xy, xz, yy, yz, zz) of the cell and of its 26 periodic neighbours,
  standardised per moment kind, neighbour index (dx+1) + 3(dy+1) + 9(dz+1),
  feature index 10 * neighbour + moment, zero padded to 288;
* target (a priori form): the Hermite coefficients of orders 3..6 of the
  cell's populations minus those of the RR reconstruction f0 + f1 from the
  cell's own moments (the order-2 difference is zero by construction), 17
  values, standardised per coefficient and zero padded to 32;
* target (step-matching form): the correction of orders 3..6 that makes one
  coarse RR update of a coarse state A reproduce a coarse state B two fine
  steps later: the post-collision populations that streaming would carry into
  B are P_i(x) = B_i(x + xi_i); R = the RR post-collision of A; the target is
  the order 3..6 Hermite coefficients of (P - R) divided by (1 - 1/tau), since
  the closure adds its prediction to the off-equilibrium coefficients before
  the relaxation;
* coarsening with a rescaled off-equilibrium part: the box average fbar,
  then f0(rho, u) + s (fbar - f0(rho, u)) with rho, u the moments of fbar.
  With s = 2 tau_c / tau_f the coarse state carries the off-equilibrium part
  a coarse run builds itself: the constitutive relation of Sec. 3.3,
  a1^(2) = -2 c_s^2 rho tau S, holds on each grid in its own lattice units,
  where the strain rate per coarse step and cell is twice the fine one;
* the network: y = W3 tanh(W2 tanh(W1 x + b1) + b2) + b3 with W1 [64 x 288],
  W2 [64 x 64], W3 [32 x 64]; loss = mean over samples and the 17 used outputs
  of (y - t)^2; analytic backward; Adam (beta1 0.9, beta2 0.999, eps 1e-8,
  bias-corrected);
* the corrected collision: the predicted 17 coefficients (unstandardised) are
  added to the recursion's off-equilibrium coefficients before the
  (1 - 1/tau) relaxation (oracle C function ora_collide_cell_closure);
  with a dead zone theta >= 0, each standardised prediction y is first shrunk
  to sign(y) max(|y| - theta, 0), so that predictions at the level of the
  network's own error leave the cell to plain RR.

All arithmetic is numpy float64 except the collisions, which call the C
oracle.
"""
from __future__ import annotations

import numpy as np

from . import D3Q27, collide_cell_closure, feq_cell, fields, fneq_cell, hermite_basis

N_IN, N_IN_USED, N_HID, N_OUT, N_OUT_USED = 288, 270, 64, 32, 17
N_MOM = 10
PARAM_SHAPES = [("W1", (N_HID, N_IN)), ("b1", (N_HID,)), ("W2", (N_HID, N_HID)), ("b2", (N_HID,)),
                ("W3", (N_OUT, N_HID)), ("b3", (N_OUT,))]
N_PARAMS = sum(int(np.prod(s)) for _, s in PARAM_SHAPES)  # 24736


# ------------------------------------------------------------------ params --
def unpack(flat: np.ndarray) -> dict:
    out, o = {}, 0
    for name, shape in PARAM_SHAPES:
        n = int(np.prod(shape))
        out[name] = np.asarray(flat[o:o + n], dtype=np.float64).reshape(shape)
        o += n
    return out


def pack(p: dict) -> np.ndarray:
    return np.concatenate([np.asarray(p[name], np.float64).reshape(-1) for name, _ in PARAM_SHAPES])


# ----------------------------------------------------------------- network --
def forward(X: np.ndarray, p: dict, round_hidden: bool = False):
    """Y [M, 32] and the cache of activations for backward. round_hidden rounds
    the two hidden layers to bfloat16 before they feed the next product (the
    precision of the tensor-core kernels), for tight comparisons."""
    X = np.asarray(X, np.float64)
    H1 = np.tanh(X @ p["W1"].T + p["b1"])
    A1 = bf16_round(H1) if round_hidden else H1
    H2 = np.tanh(A1 @ p["W2"].T + p["b2"])
    A2 = bf16_round(H2) if round_hidden else H2
    Y = A2 @ p["W3"].T + p["b3"]
    return Y, (X, H1, H2)


def loss(Y: np.ndarray, T: np.ndarray) -> float:
    d = (Y - T)[:, :N_OUT_USED]
    return float(np.mean(d * d))


def backward(Y: np.ndarray, T: np.ndarray, cache, p: dict) -> dict:
    """Gradients of loss() with respect to every parameter."""
    X, H1, H2 = cache
    M = Y.shape[0]
    dY = np.zeros_like(Y)
    dY[:, :N_OUT_USED] = 2.0 * (Y - T)[:, :N_OUT_USED] / (M * N_OUT_USED)
    g = {"W3": dY.T @ H2, "b3": dY.sum(0)}
    dA2 = (dY @ p["W3"]) * (1.0 - H2 * H2)
    g["W2"], g["b2"] = dA2.T @ H1, dA2.sum(0)
    dA1 = (dA2 @ p["W2"]) * (1.0 - H1 * H1)
    g["W1"], g["b1"] = dA1.T @ X, dA1.sum(0)
    return g


def adam(p: dict, g: dict, state: dict, lr: float, b1=0.9, b2=0.999, eps=1e-8) -> dict:
    """One Adam update; state holds m, v (dicts) and the step count t."""
    t = state.get("t", 0) + 1
    m = state.setdefault("m", {k: np.zeros_like(v) for k, v in p.items()})
    v = state.setdefault("v", {k: np.zeros_like(x) for k, x in p.items()})
    out = {}
    for k in p:
        m[k] = b1 * m[k] + (1 - b1) * g[k]
        v[k] = b2 * v[k] + (1 - b2) * g[k] * g[k]
        mh = m[k] / (1 - b1 ** t)
        vh = v[k] / (1 - b2 ** t)
        out[k] = p[k] - lr * mh / (np.sqrt(vh) + eps)
    state["t"] = t
    return out


# ------------------------------------------------------------ lattice data --
def coarsen(f: np.ndarray) -> np.ndarray:
    """2x2x2 box average of populations f [Q, nz, ny, nx] (even sizes)."""
    q, nz, ny, nx = f.shape
    return f.reshape(q, nz // 2, 2, ny // 2, 2, nx // 2, 2).mean(axis=(2, 4, 6))


def moment_field(f: np.ndarray) -> np.ndarray:
    """[10, nz, ny, nx]: rho - 1, ux, uy, uz, Pi xx, xy, xz, yy, yz, zz."""
    q, nz, ny, nx = f.shape
    rho, u, pi = fields(D3Q27, (nx, ny, nz), f)
    return np.concatenate([(rho - 1.0)[None], u, pi], axis=0)


def coarsen_neq(f: np.ndarray, scale: float) -> np.ndarray:
    """2x2x2 box average of f [Q, nz, ny, nx] with the off-equilibrium part
    scaled by `scale`: f0(rho, u) + scale (fbar - f0(rho, u))."""
    fb = coarsen(f)
    q, nz, ny, nx = fb.shape
    rho, u, _ = fields(D3Q27, (nx, ny, nz), fb)
    out = np.empty_like(fb).reshape(q, -1)
    fbf, rr, uu = fb.reshape(q, -1), rho.reshape(-1), u.reshape(3, -1)
    for c in range(nx * ny * nz):
        f0 = feq_cell(D3Q27, rr[c], uu[:, c])
        out[:, c] = f0 + scale * (fbf[:, c] - f0)
    return out.reshape(fb.shape)


def step_targets(f_pre: np.ndarray, f_post: np.ndarray, tau: float) -> np.ndarray:
    """Unstandardised step-matching targets [N, 17]: orders 3..6 of
    (P - R) / (1 - 1/tau) per cell, P_i(x) = f_post_i(x + xi_i) the populations
    streaming would carry into f_post, R the RR post-collision of f_pre."""
    from . import collide_cell, lattice_tables
    q, nz, ny, nx = f_pre.shape
    H, _ = hermite_basis(D3Q27)
    Hhi = H[10:27]
    cvel, _ = lattice_tables(D3Q27)
    P = np.empty_like(f_post)
    for i in range(q):
        # value at x of the field shifted back by xi_i: f_post_i(x + xi_i)
        P[i] = np.roll(f_post[i], shift=(-cvel[i, 2], -cvel[i, 1], -cvel[i, 0]), axis=(0, 1, 2))
    pre, P = f_pre.reshape(q, -1), P.reshape(q, -1)
    out = np.zeros((nx * ny * nz, N_OUT_USED))
    om1 = 1.0 - 1.0 / tau
    for c in range(nx * ny * nz):
        R = collide_cell(D3Q27, pre[:, c], tau)
        out[c] = Hhi @ (P[:, c] - R) / om1
    return out


def features(mom: np.ndarray, mean: np.ndarray, inv_std: np.ndarray) -> np.ndarray:
    """X [N, 288] of every cell, cells in x-fastest order."""
    _, nz, ny, nx = mom.shape
    z = (mom - mean[:, None, None, None]) * inv_std[:, None, None, None]
    cols = []
    for dz in (-1, 0, 1):
        for dy in (-1, 0, 1):
            for dx in (-1, 0, 1):
                # value of neighbour (x + dx, y + dy, z + dz) at cell (x, y, z)
                nb = np.roll(z, shift=(-dz, -dy, -dx), axis=(1, 2, 3))
                cols.append(nb.reshape(N_MOM, -1).T)
    X = np.zeros((nx * ny * nz, N_IN))
    X[:, :N_IN_USED] = np.concatenate(cols, axis=1)
    return X


def targets(f: np.ndarray) -> np.ndarray:
    """Unstandardised targets [N, 17]: orders 3..6 of f - f_RR per cell."""
    q, nz, ny, nx = f.shape
    H, _ = hermite_basis(D3Q27)
    Hhi = H[10:27]
    rho, u, pi = fields(D3Q27, (nx, ny, nz), f)
    out = np.zeros((nx * ny * nz, N_OUT_USED))
    ff = f.reshape(q, -1)
    rr, uu, pp = rho.reshape(-1), u.reshape(3, -1), pi.reshape(6, -1)
    for c in range(nx * ny * nz):
        frr = feq_cell(D3Q27, rr[c], uu[:, c]) + fneq_cell(D3Q27, uu[:, c], pp[:, c])
        out[c] = Hhi @ (ff[:, c] - frr)
    return out


def predict_delta(X: np.ndarray, p: dict, out_scale: np.ndarray,
                  bf16: bool = False, dead_zone: float = 0.0) -> np.ndarray:
    """Unstandardised correction [N, 17] predicted by the network (bf16: with
    the features and hidden layers rounded to bfloat16), each standardised
    prediction shrunk by the dead zone first."""
    Y, _ = forward(bf16_round(X) if bf16 else X, p, round_hidden=bf16)
    Y = Y[:, :N_OUT_USED]
    Y = np.sign(Y) * np.maximum(np.abs(Y) - dead_zone, 0.0)
    return Y * out_scale


def step_closure(f: np.ndarray, tau: float, p: dict, mean, inv_std, out_scale,
                 bf16: bool = False, dead_zone: float = 0.0) -> np.ndarray:
    """One update of the D3Q27 RR scheme with the learned correction: features
    from the pre-collision moments, corrected collision of every cell, periodic
    streaming (pull)."""
    delta = predict_delta(features(moment_field(f), mean, inv_std), p, out_scale, bf16,
                          dead_zone)
    return step_with_delta(f, tau, delta)


def step_with_delta(f: np.ndarray, tau: float, delta: np.ndarray) -> np.ndarray:
    """One update with given unstandardised corrections delta [N, 17]: the
    corrected collision of every cell, then periodic streaming (pull)."""
    from . import lattice_tables
    q, nz, ny, nx = f.shape
    post = np.empty_like(f).reshape(q, -1)
    ff = f.reshape(q, -1)
    for c in range(nx * ny * nz):
        post[:, c] = collide_cell_closure(ff[:, c], tau, delta[c])
    post = post.reshape(f.shape)
    cvel, _ = lattice_tables(D3Q27)
    out = np.empty_like(f)
    for i in range(q):
        out[i] = np.roll(post[i], shift=(cvel[i, 2], cvel[i, 1], cvel[i, 0]), axis=(0, 1, 2))
    return out


def bf16_round(a: np.ndarray) -> np.ndarray:
    """Round float values to bfloat16 (nearest even) and back to float64."""
    x = np.asarray(a, np.float32).copy()
    bits = x.view(np.uint32)
    lsb = (bits >> 16) & 1
    bits = (bits + 0x7FFF + lsb) & 0xFFFF0000
    return bits.view(np.float32).astype(np.float64)
