"""Pins of the FP64 oracle against what the paper and the mathematics fix.

None of these tests compares the oracle with itself: each checks it against a
closed form, an invariant, a textbook special case, a library routine on a tiny
input, or a value printed in the paper (tests/golden/).
"""
import itertools
import json
import math
import os

import numpy as np
import pytest

import oracle as O
from oracle import stability
from paper_1505_06900_gb300 import workloads as W

CS2 = 1.0 / 3.0
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
LATTICES = [O.D2Q9, O.D3Q27]
# pins that hold for any of the three lattices (D3Q19 keeps an incomplete,
# non-tensor basis: its own pins are in test_oracle_d3q19.py)
ALL_LATTICES = [O.D2Q9, O.D3Q27, O.D3Q19]


def rand_u(rng, d, scale=0.15):
    return scale * rng.standard_normal(d)


def rand_pi(rng, d, scale=0.01):
    return scale * rng.standard_normal(3 if d == 2 else 6)


def pi_matrix(d, p):
    if d == 2:
        return np.array([[p[0], p[1]], [p[1], p[2]]])
    return np.array([[p[0], p[1], p[2]], [p[1], p[3], p[4]], [p[2], p[4], p[5]]])


# ---------------------------------------------------------------- lattice ----

@pytest.mark.parametrize("lat", LATTICES)
def test_quadrature_reproduces_gaussian_moments(lat):
    """Sec. 3.2: the quadrature integrates Gaussian-weighted polynomials of
    degree <= 5 per axis exactly (variance c_s^2 = 1/3)."""
    c, w = O.lattice_tables(lat)
    d, q = O.dims_of(lat)
    gauss = {0: 1.0, 1: 0.0, 2: CS2, 3: 0.0, 4: 3 * CS2 ** 2, 5: 0.0}
    for powers in itertools.product(range(6), repeat=d):
        lhs = np.sum(w * np.prod([c[:, a].astype(float) ** powers[a] for a in range(d)], axis=0))
        rhs = np.prod([gauss[p] for p in powers])
        assert abs(lhs - rhs) < 1e-15, powers
    # degree 6 is not exact (E[X^6] = 15 c_s^6): the rule is of degree 5
    assert abs(np.sum(w * c[:, 0] ** 6.0) - 15 * CS2 ** 3) > 1e-3
    # velocity ordering i = (cx+1) + 3(cy+1) + 9(cz+1); opposite = Q-1-i
    for i in range(q):
        assert c[i, 0] == i % 3 - 1 and c[i, 1] == (i // 3) % 3 - 1
        assert np.all(c[q - 1 - i] == -c[i])


@pytest.mark.parametrize("lat", LATTICES)
def test_hermite_basis_orthogonal_and_prefactors_are_inverse_norms(lat):
    """Sec. 3.2: the kept Hermite polynomials form a complete orthogonal basis
    of the Q-dimensional space, and each prefactor printed in the expansion of
    f (1/cs2, 1/(2cs4), 2/(2cs4), ..., 1/(8cs12)) is the inverse of the
    polynomial's squared norm sum_i w_i H_k,i^2."""
    _, w = O.lattice_tables(lat)
    H, pref = O.hermite_basis(lat)
    G = (H * w) @ H.T
    off = G - np.diag(np.diag(G))
    assert np.abs(off).max() < 1e-15
    assert np.allclose(pref * np.diag(G), 1.0, rtol=0, atol=1e-14)
    assert np.linalg.matrix_rank(H) == H.shape[0]


@pytest.mark.parametrize("lat", LATTICES)
def test_expansion_of_f_is_an_identity(lat):
    """Sec. 3.2: any population set equals its Hermite expansion with the
    paper's prefactors, f_i = w_i sum_k pref_k H_k,i a_k, a_k = sum_i H_k,i f_i."""
    _, w = O.lattice_tables(lat)
    H, pref = O.hermite_basis(lat)
    rng = np.random.default_rng(1)
    f = w * (1 + 0.2 * rng.standard_normal(len(w)))
    a = H @ f
    assert np.allclose(w * ((pref * a) @ H), f, rtol=0, atol=1e-15)


# ------------------------------------------------------------ equilibrium ----

@pytest.mark.parametrize("lat", LATTICES)
def test_equilibrium_moments_and_coefficients(lat):
    """Sec. 2: sum f0 = rho, sum xi f0 = rho u, sum xi xi f0 = rho cs2 I + rho u u,
    and every kept Hermite coefficient of f0 is a0 = rho u_x^a u_y^b u_z^c
    (recursion a0^(n) = a0^(n-1) u of Sec. 3.1), computed here by projection."""
    c, w = O.lattice_tables(lat)
    d, q = O.dims_of(lat)
    H, _ = O.hermite_basis(lat)
    rng = np.random.default_rng(2)
    for _ in range(5):
        rho = 1 + 0.1 * rng.standard_normal()
        u = rand_u(rng, d)
        f0 = O.feq_cell(lat, rho, u)
        cc = c[:, :d].astype(float)
        assert abs(f0.sum() - rho) < 1e-15
        assert np.allclose(cc.T @ f0, rho * u, atol=1e-15)
        P = (cc.T * f0) @ cc
        assert np.allclose(P, rho * CS2 * np.eye(d) + rho * np.outer(u, u), atol=1e-15)
        # projection on each basis member: the member H_k is the product of
        # 1-D factors {1, xi, xi^2 - cs2}; its coefficient is rho prod u^(power)
        a_proj = H @ f0
        expected = []
        for k in range(q):
            # power of each axis: fit H_k along the lattice against 1-D factors
            pw = _member_powers(lat, H[k], c)
            expected.append(rho * np.prod([u[a] ** pw[a] for a in range(d)]))
        assert np.allclose(a_proj, expected, atol=1e-15)


def _member_powers(lat, Hrow, c):
    """Powers (0, 1, 2) per axis of a tensor-product Hermite member, found by
    matching its values with products of the 1-D factors 1, x, x^2 - cs2."""
    d, _ = O.dims_of(lat)
    fac = [lambda x: 1.0 + 0 * x, lambda x: x, lambda x: x * x - CS2]
    for pw in itertools.product(range(3), repeat=d):
        vals = np.prod([fac[pw[a]](c[:, a].astype(float)) for a in range(d)], axis=0)
        if np.allclose(vals, Hrow, atol=1e-15):
            return pw
    raise AssertionError("not a tensor-product member")


@pytest.mark.parametrize("lat", LATTICES)
def test_equilibrium_closed_product_form(lat):
    """f0 equals rho prod_d g(xi_d, u_d) with the 1-D equilibrium of the D1Q3
    rule, g(0,u) = 2/3 - u^2, g(+-1,u) = 1/6 +- u/2 + u^2/2 (the tensor-product
    structure of the basis makes the series factorise)."""
    c, _ = O.lattice_tables(lat)
    d, _ = O.dims_of(lat)

    def g(xi, u):
        return 2.0 / 3.0 - u * u if xi == 0 else 1.0 / 6.0 + xi * u / 2.0 + u * u / 2.0

    rng = np.random.default_rng(3)
    for _ in range(5):
        rho = 1 + 0.1 * rng.standard_normal()
        u = rand_u(rng, d, 0.3)
        f0 = O.feq_cell(lat, rho, u)
        ref = np.array([rho * np.prod([g(ci[a], u[a]) for a in range(d)]) for ci in c])
        assert np.allclose(f0, ref, rtol=0, atol=1e-15)


@pytest.mark.parametrize("lat", [O.D3Q27, O.D3Q19])
def test_order2_equilibrium_textbook(lat):
    """eq_feq_2: the order-2 equilibrium is the textbook
    w rho (1 + 3 xi.u + 9/2 (xi.u)^2 - 3/2 u^2)."""
    c, w = O.lattice_tables(lat)
    u = np.array([0.1, -0.07, 0.05])
    f = O.feq_cell(lat, 1.1, u, variant=O.REG2)
    cu = c @ u
    ref = w * 1.1 * (1 + 3 * cu + 4.5 * cu ** 2 - 1.5 * u @ u)
    assert np.allclose(f, ref, atol=1e-15)


# ---------------------------------------------------- non-equilibrium part ----

def _pair_sum(d, idx, u, A):
    """Closed form of the recursion: sum over position pairs j<k of
    a1^(2)[idx_j, idx_k] * prod_{m != j,k} u[idx_m]."""
    s = 0.0
    n = len(idx)
    for j in range(n):
        for k in range(j + 1, n):
            prod = A[idx[j], idx[k]]
            for m in range(n):
                if m not in (j, k):
                    prod *= u[idx[m]]
            s += prod
    return s


NAMES_2D = ["xx", "xy", "yy", "xxy", "xyy", "xxyy"]
NAMES_3D = ["xx", "xy", "xz", "yy", "yz", "zz", "xxy", "xxz", "xyy", "xzz", "yzz", "yyz", "xyz",
            "xxyy", "xxzz", "yyzz", "xyzz", "xyyz", "xxyz", "xxyzz", "xxyyz", "xyyzz", "xxyyzz"]


@pytest.mark.parametrize("lat", ALL_LATTICES)
def test_recursion_equals_pair_sum_closed_form(lat):
    """eq_rel_a1 (Appendix B without the starred terms): a1^(n) equals the sum,
    over unordered pairs of index positions, of a1^(2) on that pair times the
    velocity components of the other positions."""
    d, _ = O.dims_of(lat)
    names = NAMES_2D if d == 2 else NAMES_3D
    rng = np.random.default_rng(4)
    for _ in range(10):
        u = rand_u(rng, d, 0.3)
        p = rand_pi(rng, d, 0.05)
        A = pi_matrix(d, p)
        got = O.a1_coefficients(lat, u, p)
        for name, val in zip(names, got):
            idx = ["xyz".index(ch) for ch in name]
            assert abs(val - _pair_sum(d, idx, u, A)) < 1e-15, name


@pytest.mark.parametrize("lat", ALL_LATTICES)
def test_fneq_is_second_velocity_derivative_of_feq(lat):
    """With a1^(n) given by the recursion, f1 = 1/2 sum_ab a1^(2)_ab
    d^2 (f0/rho) / du_a du_b. f0/rho is a polynomial of degree <= 2 in each
    velocity component, so central differences give the derivatives exactly."""
    d, _ = O.dims_of(lat)
    rng = np.random.default_rng(5)
    h = 0.125
    for _ in range(5):
        u = rand_u(rng, d, 0.2)
        p = rand_pi(rng, d, 0.02)
        A = pi_matrix(d, p)
        e = np.eye(d) * h

        def F(v):
            return O.feq_cell(lat, 1.0, v)

        ref = 0.0
        for a in range(d):
            ref = ref + 0.5 * A[a, a] * (F(u + e[a]) - 2 * F(u) + F(u - e[a])) / h ** 2
            for b in range(a + 1, d):
                mixed = (F(u + e[a] + e[b]) - F(u + e[a] - e[b]) - F(u - e[a] + e[b])
                         + F(u - e[a] - e[b])) / (4 * h * h)
                ref = ref + A[a, b] * mixed
        assert np.allclose(O.fneq_cell(lat, u, p), ref, rtol=0, atol=1e-14)


@pytest.mark.parametrize("lat", ALL_LATTICES)
def test_fneq_at_rest_is_order_two(lat):
    """Sec. 3.7 (boundary conditions): at u = 0 the off-equilibrium part reduces
    to f1 = w/(2 cs4) H2 : Pi1 exactly."""
    c, w = O.lattice_tables(lat)
    d, _ = O.dims_of(lat)
    rng = np.random.default_rng(6)
    p = rand_pi(rng, d)
    A = pi_matrix(d, p)
    cc = c[:, :d].astype(float)
    H2A = np.einsum("ia,ib,ab->i", cc, cc, A) - CS2 * np.trace(A)
    ref = w / (2 * CS2 ** 2) * H2A
    assert np.allclose(O.fneq_cell(lat, np.zeros(d), p), ref, atol=1e-16)


# -------------------------------------------------------------- collision ----

@pytest.mark.parametrize("lat", ALL_LATTICES)
@pytest.mark.parametrize("variant", [O.RR, O.REG2, O.BGK])
def test_collision_moments(lat, variant):
    """eq_discr_bgk_reg: post-collision populations keep rho and rho u and
    relax the non-equilibrium stress, sum xi xi f_post = rho cs2 I + rho u u +
    (1 - 1/tau) Pi1, where Pi1 = sum xi xi f - rho cs2 I - rho u u."""
    c, w = O.lattice_tables(lat)
    d, q = O.dims_of(lat)
    cc = c[:, :d].astype(float)
    rng = np.random.default_rng(7)
    for tau in (0.5001, 0.7, 1.3):
        f = w * (1 + 0.1 * rng.standard_normal(q)) + 0.01 * w * (cc @ rng.standard_normal(d))
        rho = f.sum()
        u = cc.T @ f / rho
        Pi = (cc.T * f) @ cc - rho * CS2 * np.eye(d) - rho * np.outer(u, u)
        fp = O.collide_cell(lat, f, tau, variant)
        assert abs(fp.sum() - rho) < 1e-15
        assert np.allclose(cc.T @ fp, rho * u, atol=1e-15)
        P = (cc.T * fp) @ cc
        assert np.allclose(P, rho * CS2 * np.eye(d) + rho * np.outer(u, u) + (1 - 1 / tau) * Pi,
                           atol=1e-15)
        # the cell's own moment routine agrees with the plain definition
        r2, u2, p2 = O.moments_cell(lat, f, variant)
        assert abs(r2 - rho) < 1e-15 and np.allclose(u2, u, atol=1e-15)
        iu = np.triu_indices(d)
        assert np.allclose(p2, Pi[iu], atol=1e-15)


@pytest.mark.parametrize("lat", ALL_LATTICES)
def test_bgk_relaxes_every_hermite_coefficient(lat):
    """eq_full_discr_bgk: plain BGK scales every Hermite coefficient of
    f - f0 by (1 - 1/tau), the ones of order > 2 included (which RR replaces by
    the recursion)."""
    _, w = O.lattice_tables(lat)
    d, q = O.dims_of(lat)
    H, _ = O.hermite_basis(lat)
    rng = np.random.default_rng(12)
    f = w * (1 + 0.1 * rng.standard_normal(q))
    rho, u, _ = O.moments_cell(lat, f)
    f0 = O.feq_cell(lat, rho, u)
    for tau in (0.6, 1.7):
        post = O.collide_cell(lat, f, tau, O.BGK)
        assert np.allclose(H @ (post - f0), (1 - 1 / tau) * (H @ (f - f0)), atol=1e-15)
        rr = O.collide_cell(lat, f, tau, O.RR)
        assert np.abs(H[1 + d + d * (d + 1) // 2:] @ (rr - post)).max() > 1e-6


@pytest.mark.parametrize("lat", ALL_LATTICES)
def test_collision_fixed_points(lat):
    """f = f0 is a fixed point; tau = 1 gives f_post = f0 for any f."""
    c, w = O.lattice_tables(lat)
    d, q = O.dims_of(lat)
    rng = np.random.default_rng(8)
    u = rand_u(rng, d)
    f0 = O.feq_cell(lat, 1.05, u)
    assert np.allclose(O.collide_cell(lat, f0, 0.6), f0, atol=1e-16)
    f = w * (1 + 0.1 * rng.standard_normal(q))
    rho, uu, _ = O.moments_cell(lat, f)
    assert np.allclose(O.collide_cell(lat, f, 1.0), O.feq_cell(lat, rho, uu), atol=1e-16)


@pytest.mark.parametrize("lat", ALL_LATTICES)
def test_regularization_is_a_projection(lat):
    """eq_reg: regularizing twice equals regularizing once (tau -> infinity is
    f_post = f0 + f1), and the regularized f keeps rho, rho u and Pi1."""
    _, w = O.lattice_tables(lat)
    d, q = O.dims_of(lat)
    rng = np.random.default_rng(9)
    f = w * (1 + 0.1 * rng.standard_normal(q))
    big = 1e15
    r1 = O.collide_cell(lat, f, big)
    r2 = O.collide_cell(lat, r1, big)
    assert np.allclose(r1, r2, atol=1e-15)
    m0, m1 = O.moments_cell(lat, f), O.moments_cell(lat, r1)
    assert abs(m0[0] - m1[0]) < 1e-15
    assert np.allclose(m0[1], m1[1], atol=1e-15) and np.allclose(m0[2], m1[2], atol=1e-14)


# ------------------------------------------------------ streaming, periodic ----

def _brute_step(lat, shape, tau, f):
    """One update by independent means: the oracle's single-cell collision on
    every cell, then numpy.roll for the periodic streaming."""
    c, _ = O.lattice_tables(lat)
    q = f.shape[0]
    nx, ny, nz = shape
    post = np.zeros_like(f)
    for z in range(nz):
        for y in range(ny):
            for x in range(nx):
                post[:, z, y, x] = O.collide_cell(lat, f[:, z, y, x], tau)
    out = np.empty_like(f)
    for i in range(q):
        out[i] = np.roll(post[i], shift=(c[i, 2], c[i, 1], c[i, 0]), axis=(0, 1, 2))
    return out


@pytest.mark.parametrize("lat,shape", [(O.D2Q9, (5, 4, 1)), (O.D3Q27, (4, 5, 3)),
                                       (O.D3Q19, (3, 4, 5))])
def test_step_matches_collide_then_roll(lat, shape):
    """eq_discr_bgk_reg with periodic wrap: f_i(x + xi_i, t+1) = f_post_i(x, t),
    checked by brute force on a tiny non-cubic grid."""
    _, w = O.lattice_tables(lat)
    q = len(w)
    rng = np.random.default_rng(10)
    f = w[:, None, None, None] * (1 + 0.1 * rng.standard_normal((q, shape[2], shape[1], shape[0])))
    got = O.step(lat, shape, 0.8, f, 2)
    ref = _brute_step(lat, shape, 0.8, _brute_step(lat, shape, 0.8, f))
    assert np.allclose(got, ref, rtol=0, atol=1e-16)


@pytest.mark.parametrize("lat,shape", [(O.D2Q9, (8, 6, 1)), (O.D3Q27, (6, 5, 4)),
                                       (O.D3Q19, (5, 4, 6))])
def test_conservation_and_uniform_flow(lat, shape):
    """Mass and momentum are conserved to round-off on a periodic grid
    (Sec. 2 conservation), and a uniform flow stays uniform at f0."""
    d, q = O.dims_of(lat)
    rho, u = W.random_field(shape, d, seed=11)
    f = O.init(lat, shape, 0.6, rho, u, O.INIT_EQ_NEQ_FD)
    d0 = O.diagnostics(lat, shape, f)
    f2 = O.step(lat, shape, 0.6, f, 50)
    d1 = O.diagnostics(lat, shape, f2)
    assert abs(d1[0] - d0[0]) < 1e-12 * d0[0]
    assert np.allclose(d1[1:1 + d], d0[1:1 + d], atol=1e-13)
    nx, ny, nz = shape
    uu = np.zeros((d, nz, ny, nx)) + np.array([0.1, -0.05, 0.03][:d])[:, None, None, None]
    f = O.init(lat, shape, 0.6, np.ones((nz, ny, nx)), uu, O.INIT_EQ_NEQ_FD)
    f2 = O.step(lat, shape, 0.6, f, 5)
    f0 = O.feq_cell(lat, 1.0, uu[:, 0, 0, 0])
    assert np.allclose(f2, f0[:, None, None, None], atol=1e-15)


@pytest.mark.parametrize("lat", [O.D3Q27, O.D3Q19])
def test_single_population_moves_one_cell_per_step(lat):
    """Streaming: with tau = 1 the post-collision state is f0 of the cell, so a
    one-cell density bump at rest spreads as w_i * bump to exactly the cells
    x + xi_i after one step (brute force on 3^3)."""
    shape = (3, 3, 3)
    c, w = O.lattice_tables(lat)
    rho = np.ones((3, 3, 3))
    rho[1, 1, 1] = 1.5
    u = np.zeros((3, 3, 3, 3))
    f = O.init(lat, shape, 1.0, rho, u, O.INIT_EQ)
    f1 = O.step(lat, shape, 1.0, f, 1)
    for i in range(len(w)):
        expect = np.full((3, 3, 3), w[i])
        expect[1 + c[i, 2], 1 + c[i, 1], 1 + c[i, 0]] = 1.5 * w[i]
        assert np.allclose(f1[i], expect, atol=1e-16)


# ------------------------------------------------------------------ init ----

def test_init_stress_matches_central_difference_closed_form():
    """Initial a1^(2) = -2 cs2 rho tau S with S from periodic central
    differences: for u_x = U sin(kx) cos(ky), the difference of sin(kx) is
    cos(kx) sin(k), so S_xx = U sin(k) cos(kx) cos(ky) exactly, etc."""
    n, U, tau = 16, 0.05, 0.7
    rho, u = W.taylor_green_2d(n, U)
    f = O.init(O.D2Q9, (n, n, 1), tau, rho, u, O.INIT_EQ_NEQ_FD)
    r, uu, p = O.fields(O.D2Q9, (n, n, 1), f)
    assert np.allclose(r, rho, atol=1e-15) and np.allclose(uu, u, atol=1e-15)
    k = 2 * math.pi / n
    x = np.arange(n)[None, :]
    y = np.arange(n)[:, None]
    Sxx = U * math.sin(k) * np.cos(k * x) * np.cos(k * y)
    Syy = -U * math.sin(k) * np.cos(k * x) * np.cos(k * y)
    Sxy = 0.5 * (-U * math.sin(k) * np.sin(k * x) * np.sin(k * y)
                 + U * math.sin(k) * np.sin(k * x) * np.sin(k * y))
    fac = -2 * CS2 * rho[0] * tau
    assert np.allclose(p[0, 0], fac * Sxx, atol=1e-15)
    assert np.allclose(p[1, 0], fac * Sxy, atol=1e-15)
    assert np.allclose(p[2, 0], fac * Syy, atol=1e-15)


# ----------------------------------------------------------- diagnostics ----

def test_diagnostics_and_enstrophy_closed_forms():
    """Mass, momentum and kinetic energy of an initialised field equal the plain
    sums over the input fields; the enstrophy of the 2D Taylor-Green field with
    central differences is U^2 sin(k)^2 n^2 / 2."""
    n, U = 32, 0.05
    rho, u = W.taylor_green_2d(n, U)
    f = O.init(O.D2Q9, (n, n, 1), 0.7, rho, u, O.INIT_EQ_NEQ_FD)
    dg = O.diagnostics(O.D2Q9, (n, n, 1), f)
    assert abs(dg[0] - rho.sum()) < 1e-10
    assert np.allclose(dg[1:3], (rho[None] * u).sum(axis=(1, 2, 3)), atol=1e-13)
    assert abs(dg[3] - 0.5 * (rho * (u ** 2).sum(0)).sum()) < 1e-13
    k = 2 * math.pi / n
    assert abs(O.enstrophy(O.D2Q9, (n, n, 1), f) - U * U * math.sin(k) ** 2 * n * n / 2) < 1e-13


def test_enstrophy_3d_closed_form():
    """3D Taylor-Green field: with central differences, omega_x = -U s c_x s_y... the
    sum of |omega|^2 / 2 over an n^3 grid has the closed form below."""
    n, mach = 12, 0.1
    rho, u = W.taylor_green_3d(n, mach)
    U = mach * math.sqrt(CS2)
    f = O.init(O.D3Q27, (n, n, n), 0.6, rho, u, O.INIT_EQ)
    h = 2 * math.pi / n
    s = math.sin(h)
    X = (np.arange(n) + 0.5) * h
    # omega_x = -d_z u_y = -U cos x sin y sin z * s
    # omega_y =  d_z u_x = -U sin x cos y sin z * s
    # omega_z = d_x u_y - d_y u_x = 2 U sin x sin y cos z * s
    cx, sx = np.cos(X), np.sin(X)
    ox = -U * s * np.einsum("z,y,x->zyx", sx, sx, cx)
    oy = -U * s * np.einsum("z,y,x->zyx", sx, cx, sx)
    oz = 2 * U * s * np.einsum("z,y,x->zyx", cx, sx, sx)
    ref = 0.5 * (ox ** 2 + oy ** 2 + oz ** 2).sum()
    assert abs(O.enstrophy(O.D3Q27, (n, n, n), f) - ref) < 1e-14
    # and the closed form of that sum: each sin^2/cos^2 sums to n/2
    assert abs(ref - 0.5 * U * U * s * s * (n / 2) ** 3 * (1 + 1 + 4)) < 1e-14


# ---------------------------------------------------------- whole scheme ----

def test_taylor_green_2d_decay():
    """Config D2Q9 128^2 Taylor-Green vortex, Re = 100, 1000 steps: the kinetic
    energy decays as exp(-4 nu k^2 t) with nu = cs2 (tau - 1/2) (Sec. 3.3 with
    the shifted tau of Sec. 3.4), fitted nu within 1%; the velocity field stays within 1%
    (L2) of the analytic field. The L2 tolerance covers the O(Ma^2) acoustic
    content of the weakly compressible scheme (measured 5.9e-3)."""
    n, U = 128, 0.05
    tau = W.taylor_green_2d_tau(n, U, 100.0)
    assert abs(tau - 0.692) < 1e-12
    rho, u = W.taylor_green_2d(n, U)
    shape = (n, n, 1)
    f = O.init(O.D2Q9, shape, tau, rho, u, O.INIT_EQ_NEQ_FD)
    ke0 = O.diagnostics(O.D2Q9, shape, f)[-1]
    t = 1000
    f = O.step(O.D2Q9, shape, tau, f, t)
    ke = O.diagnostics(O.D2Q9, shape, f)[-1]
    k = 2 * math.pi / n
    nu = CS2 * (tau - 0.5)
    nu_eff = -math.log(ke / ke0) / (4 * k * k * t)
    assert abs(nu_eff / nu - 1) < 0.01
    _, uu, _ = O.fields(O.D2Q9, shape, f)
    ua = u * math.exp(-2 * nu * k * k * t)
    assert np.linalg.norm(uu - ua) / np.linalg.norm(ua) < 1e-2


# ------------------------------------------------- linear stability pins ----

def _golden_stability():
    with open(os.path.join(GOLDEN, "stability_d2q9.json")) as fh:
        return json.load(fh)


def test_linear_stability_present_model_stable_at_ma_0346():
    """Sec. 3.6: at tau = 0.5001, u = (0.2, 0) the present model has no unstable
    mode anywhere in the k plane (growth rate ln|lambda| <= 0 up to the
    round-off of the numerical Jacobian)."""
    g = _golden_stability()
    rate, _ = stability.max_growth(O.D2Q9, g["rr_stable_velocity"], g["tau"], O.RR, nk=64)
    assert rate < 1e-10


def test_linear_stability_present_model_unstable_at_ma_043():
    """Sec. 3.6: at u_x = 0.248 unstable modes have appeared."""
    g = _golden_stability()
    rate, _ = stability.max_growth(O.D2Q9, g["rr_unstable_velocity"], g["tau"], O.RR, nk=64)
    assert rate > 1e-6


def test_linear_stability_order2_regularized_unstable_along_kx():
    """Sec. 3.8.1: the order-2 regularized model has an unstable (shear) mode
    along k_y = 0 at u_x = 0.2, while the present model has none there."""
    g = _golden_stability()
    u = g["reg2_unstable_velocity_ky0"]
    rate2, _ = stability.max_growth(O.D2Q9, u, g["tau"], O.REG2, nk=256, ky_zero=True)
    rate_rr, _ = stability.max_growth(O.D2Q9, u, g["tau"], O.RR, nk=256, ky_zero=True)
    assert rate2 > 1e-3
    assert rate_rr < 1e-10


def test_linear_stability_hydrodynamic_limit():
    """At small k the shear mode of the linearised scheme decays at the
    Navier-Stokes rate Im(omega_s) = -nu |k|^2 (Sec. 3.6), nu = cs2 (tau - 1/2)."""
    tau = 0.8
    nu = CS2 * (tau - 0.5)
    J = stability.jacobian(O.D2Q9, 1.0, (0.0, 0.0), tau)
    k = 0.02
    rates = np.sort(stability.growth_rates(O.D2Q9, J, (k, 0.0)))[::-1]
    # the three slowest modes: shear (-nu k^2) and two sound modes (-nu k^2 / 2
    # with the bulk viscosity of BGK, eta = nu in 2D)
    shear = -nu * k * k
    assert np.any(np.abs(rates[:3] - shear) < 1e-3 * abs(shear))


def test_linear_stability_onset_of_the_present_model():
    """Sec. 3.6: the smallest u_x with a growing mode anywhere in the k plane
    (tau = 0.5001). On a 128^2 map of wave vectors the oracle's onset is
    0.2305 (pinned to +-0.005, the precision the paper prints its value with;
    this pin guards the oracle against drift, the paper's statements are the
    two pins above). It lies below the paper's 0.248: see the next test for
    where the printed value falls."""
    onset = stability.onset_velocity(0.5001, 128, tol=5e-4)
    assert abs(onset - 0.2305) <= 0.005
    g = _golden_stability()
    assert g["rr_stable_velocity"][0] < onset < g["rr_unstable_velocity"][0]


def test_linear_stability_onset_is_steep_in_tau():
    """The onset rises steeply with the viscosity tau - 1/2 near tau = 1/2: on a
    64^2 map it moves from u_x ~ 0.21 at tau = 0.50005 through 0.232 at 0.5001
    to 0.257 at 0.5002, so the paper's u_x = 0.248, printed for tau = 0.5001
    (four decimals), lies inside the band of onsets for tau between 0.5001 and
    0.5002 (the oracle reaches it at tau ~ 0.50017)."""
    on = [stability.onset_velocity(t, 64, lo=0.15, hi=0.4, tol=5e-4)
          for t in (0.50005, 0.5001, 0.5002)]
    assert on[0] < on[1] < on[2]
    g = _golden_stability()
    assert on[1] < g["rr_unstable_velocity"][0] < on[2]
