"""Pins of the oracle's D3Q19 lattice, whose recursion the paper leaves open
(Sec. 5: it would need basis vectors other than Hermite polynomials).

The reading pinned here: D3Q19 is the D3Q27 velocity set without the eight
corners; the basis kept is 1, xi, the six order-2 Hermite polynomials and,
for each odd index b with even pair (a, c), the sum and the difference
H_aab +- H_bcc, the largest set of (sums of) Hermite polynomials that the
D3Q19 weights keep mutually orthogonal. f0 and f1 are the members of that
span whose projections on the basis are the Hermite coefficients of Sec. 2
(equilibrium) and of the recursion eq_rel_a1 (off-equilibrium).

Every test builds what it compares with from the velocity set and textbook
formulas, not from the oracle's expansion.
"""
import itertools

import numpy as np
import pytest

import oracle as O
from oracle import stability

CS2 = 1.0 / 3.0
L19 = O.D3Q19


def velocities():
    """D3Q27 order i = (cx+1) + 3(cy+1) + 9(cz+1) without |c|^2 = 3."""
    out = []
    for i in range(27):
        c = (i % 3 - 1, (i // 3) % 3 - 1, i // 9 - 1)
        if sum(v * v for v in c) < 3:
            out.append(c)
    return np.array(out, dtype=float)


def hermite(c, idx):
    """Tensor Hermite polynomial with variance cs2 for an index string such as
    'xxy': per axis, power 0 -> 1, 1 -> xi, 2 -> xi^2 - cs2."""
    v = np.ones(len(c))
    for a in range(3):
        p = idx.count("xyz"[a])
        v = v * (1.0 if p == 0 else (c[:, a] if p == 1 else c[:, a] ** 2 - CS2))
    return v


# odd index b with even pair (a, c), as the three order-3 sums/differences
TRIPLES = [("xyy", "xzz"), ("xxy", "yzz"), ("xxz", "yyz")]


def basis(c):
    """The 16 members: 1, x, y, z, xx, xy, xz, yy, yz, zz, three sums, three
    differences (rows), built from textbook Hermite polynomials."""
    rows = [hermite(c, "")] + [hermite(c, s) for s in ("x", "y", "z")]
    rows += [hermite(c, s) for s in ("xx", "xy", "xz", "yy", "yz", "zz")]
    rows += [hermite(c, p) + hermite(c, q) for p, q in TRIPLES]
    rows += [hermite(c, p) - hermite(c, q) for p, q in TRIPLES]
    return np.array(rows)


def test_lattice_is_d3q27_without_corners():
    c, w = O.lattice_tables(L19)
    assert np.array_equal(c, velocities().astype(int))
    m = np.sum(c * c, axis=1)
    assert np.allclose(w, np.select([m == 0, m == 1, m == 2], [1 / 3, 1 / 18, 1 / 36]), atol=0)
    for i in range(19):
        assert np.all(c[18 - i] == -c[i])  # opposite = Q - 1 - i
    assert np.all(c[9] == 0)


def test_quadrature_is_exact_to_degree_five_only():
    """D3Q19 integrates every monomial of total degree <= 5 against the
    Gaussian of variance cs2, unlike D3Q27 not all of degree 6."""
    c, w = O.lattice_tables(L19)
    gauss = {0: 1.0, 1: 0.0, 2: CS2, 3: 0.0, 4: 3 * CS2 ** 2, 5: 0.0, 6: 15 * CS2 ** 3}
    for p in itertools.product(range(6), repeat=3):
        if sum(p) > 5:
            continue
        lhs = np.sum(w * np.prod([c[:, a].astype(float) ** p[a] for a in range(3)], axis=0))
        assert abs(lhs - np.prod([gauss[k] for k in p])) < 1e-15, p
    # x^2 y^2 z^2: cs^6 for the Gaussian, 0 on D3Q19 (no corner velocity)
    assert abs(np.sum(w * (c[:, 0] * c[:, 1] * c[:, 2]) ** 2)) == 0.0


def test_basis_is_the_orthogonal_hermite_sums_with_their_norms():
    c, w = O.lattice_tables(L19)
    cf = c.astype(float)
    H, pref = O.hermite_basis(L19)
    B = basis(cf)
    assert H.shape == (16, 19)
    assert np.allclose(H, B, atol=1e-15)
    G = (B * w) @ B.T
    assert np.abs(G - np.diag(np.diag(G))).max() < 1e-15
    cs4, cs6 = CS2 ** 2, CS2 ** 3
    norms = [1.0] + [CS2] * 3 + [2 * cs4, cs4, cs4, 2 * cs4, cs4, 2 * cs4] + [2 * cs6] * 3 + [6 * cs6] * 3
    assert np.allclose(np.diag(G), norms, rtol=1e-14, atol=0)
    # the expansion term of member k is w pref_k H_k a_k: pref = 1 / norm
    assert np.allclose(pref * np.array(norms), 1.0, atol=1e-14)
    # why these members: on D3Q19 the single order-3 polynomials are not
    # orthogonal (<H_xxy, H_yzz> = -cs^6), xyz vanishes, and order 4 leans
    # on order 2 (<H_xxyy, H_zz> = -cs^6)
    ip = lambda p, q: np.sum(w * hermite(cf, p) * hermite(cf, q))
    assert abs(ip("xxy", "yzz") + cs6) < 1e-16
    assert np.all(hermite(cf, "xyz") == 0.0)
    assert abs(ip("xxyy", "zz") + cs6) < 1e-16


@pytest.mark.parametrize("seed", range(4))
def test_equilibrium_moments(seed):
    """Sec. 2 on D3Q19: rho, rho u and rho cs2 I + rho u u exactly, and every
    order-3 Hermite moment except xyz equal to rho u_a u_b u_c (the sum and the
    difference are both kept); the xyz moment is zero."""
    rng = np.random.default_rng(seed)
    c, w = O.lattice_tables(L19)
    cf = c.astype(float)
    rho, u = 1 + 0.1 * rng.standard_normal(), 0.15 * rng.standard_normal(3)
    f0 = O.feq_cell(L19, rho, u)
    assert abs(f0.sum() - rho) < 1e-15
    assert np.allclose(cf.T @ f0, rho * u, atol=1e-15)
    assert np.allclose((cf.T * f0) @ cf, rho * (CS2 * np.eye(3) + np.outer(u, u)), atol=1e-15)
    for name in ("xxy", "xxz", "xyy", "xzz", "yzz", "yyz"):
        expect = rho * np.prod([u["xyz".index(ch)] for ch in name])
        assert abs(hermite(cf, name) @ f0 - expect) < 1e-15, name
    assert abs(hermite(cf, "xyz") @ f0) < 1e-16


@pytest.mark.parametrize("seed", range(4))
def test_equilibrium_is_the_moment_matching_member_of_the_span(seed):
    """Solving the 16 moment conditions for f = w * (B^T x) by a dense linear
    solve gives the oracle's f0 (the two share nothing but the velocity set)."""
    rng = np.random.default_rng(10 + seed)
    c, w = O.lattice_tables(L19)
    cf = c.astype(float)
    B = basis(cf)
    rho, u = 1 + 0.1 * rng.standard_normal(), 0.2 * rng.standard_normal(3)
    a3 = {n: rho * np.prod([u["xyz".index(ch)] for ch in n]) for p in TRIPLES for n in p}
    m = [rho] + list(rho * u) + [rho * u[a] * u[b] for a, b in
                                 ((0, 0), (0, 1), (0, 2), (1, 1), (1, 2), (2, 2))]
    m += [a3[p] + a3[q] for p, q in TRIPLES] + [a3[p] - a3[q] for p, q in TRIPLES]
    x = np.linalg.solve((B * w) @ B.T, np.array(m))
    assert np.allclose(w * (B.T @ x), O.feq_cell(L19, rho, u), rtol=0, atol=1e-15)


@pytest.mark.parametrize("seed", range(4))
def test_off_equilibrium_moments_follow_the_recursion(seed):
    """f1 carries no mass or momentum, has Pi1 as its order-2 moment and, on
    every order-3 member but xyz, the pair sum of eq_rel_a1:
    a1_aab = Pi_aa u_b + 2 Pi_ab u_a."""
    rng = np.random.default_rng(20 + seed)
    c, _ = O.lattice_tables(L19)
    cf = c.astype(float)
    u = 0.2 * rng.standard_normal(3)
    p = 0.02 * rng.standard_normal(6)
    P = np.array([[p[0], p[1], p[2]], [p[1], p[3], p[4]], [p[2], p[4], p[5]]])
    f1 = O.fneq_cell(L19, u, p)
    assert abs(f1.sum()) < 1e-16 and np.abs(cf.T @ f1).max() < 1e-16
    assert np.allclose((cf.T * f1) @ cf, P, atol=1e-16)
    for name in ("xxy", "xxz", "xyy", "xzz", "yzz", "yyz"):
        a = "xyz".index(name[0]) if name[0] == name[1] else "xyz".index(name[1])
        b = "xyz".index(name[2]) if name[0] == name[1] else "xyz".index(name[0])
        expect = P[a, a] * u[b] + 2 * P[a, b] * u[a]
        assert abs(hermite(cf, name) @ f1 - expect) < 1e-16, name


def test_shear_wave_decays_at_the_navier_stokes_rate():
    """Whole scheme: a periodic shear wave u_x = U sin(2 pi y / L) decays as
    exp(-nu k^2 t), nu = cs2 (tau - 1/2), on D3Q19 as on the full lattice."""
    L, tau, U = 32, 0.8, 0.01
    shape = (2, L, 3)
    y = np.arange(L)
    ux = U * np.sin(2 * np.pi * y / L)
    u = np.zeros((3, 3, L, 2))
    u[0] = ux[None, :, None]
    f = O.init(L19, shape, tau, np.ones((3, L, 2)), u)
    mode = np.sin(2 * np.pi * y / L)
    steps, amps, done = [100, 200, 300, 400], [], 0
    for s in steps:
        f = O.step(L19, shape, tau, f, s - done)
        done = s
        _, uu, _ = O.fields(L19, shape, f)
        amps.append(np.dot(uu[0, 1, :, 1], mode) / np.dot(mode, mode))
    rate = -np.polyfit(steps, np.log(amps), 1)[0]
    expected = CS2 * (tau - 0.5) * (2 * np.pi / L) ** 2
    assert abs(rate / expected - 1.0) < 2e-3, rate / expected - 1.0


def test_linear_stability_at_rest_and_shear_mode():
    """Linearised D3Q19 update at rest: no mode grows anywhere on a k grid,
    and the shear mode decays at the Navier-Stokes rate -nu k^2 at small k."""
    tau = 0.8
    nu = CS2 * (tau - 0.5)
    J = stability.jacobian(L19, 1.0, (0.0, 0.0, 0.0), tau)
    ks = np.linspace(-np.pi, np.pi, 9, endpoint=False)
    worst = max(stability.growth_rates(L19, J, k).max() for k in itertools.product(ks, repeat=3))
    assert worst < 1e-10
    k = 0.02
    rates = stability.growth_rates(L19, J, (k, 0.0, 0.0))
    assert np.any(np.abs(rates + nu * k * k) < 1e-3 * nu * k * k)
