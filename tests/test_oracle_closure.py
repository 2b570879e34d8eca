"""Pins of the FP64 learned-closure reference (oracle/closure.py) against
library routines, finite differences, brute force and special cases."""
import numpy as np
import pytest

import oracle as O
from oracle import closure as C

torch = pytest.importorskip("torch")


def rand_params(rng, scale=0.2):
    return C.unpack(scale * rng.standard_normal(C.N_PARAMS))


def test_forward_matches_torch_float64():
    rng = np.random.default_rng(0)
    p = rand_params(rng)
    X = rng.standard_normal((37, C.N_IN))
    Y, _ = C.forward(X, p)
    t = {k: torch.from_numpy(v) for k, v in p.items()}
    h = torch.tanh(torch.nn.functional.linear(torch.from_numpy(X), t["W1"], t["b1"]))
    h = torch.tanh(torch.nn.functional.linear(h, t["W2"], t["b2"]))
    ref = torch.nn.functional.linear(h, t["W3"], t["b3"]).numpy()
    assert np.abs(Y - ref).max() < 1e-13


def test_backward_matches_central_differences():
    rng = np.random.default_rng(1)
    p = rand_params(rng, 0.3)
    X = rng.standard_normal((9, C.N_IN))
    T = rng.standard_normal((9, C.N_OUT))
    Y, cache = C.forward(X, p)
    g = C.backward(Y, T, cache, p)
    flat, gflat = C.pack(p), C.pack(g)
    idx = rng.choice(C.N_PARAMS, 60, replace=False)
    # include biases and every layer
    idx = np.concatenate([idx, [0, 18432, 18432 + 64, 22592 + 64, C.N_PARAMS - 1]])
    h = 1e-5
    for k in idx:
        fp, fm = flat.copy(), flat.copy()
        fp[k] += h
        fm[k] -= h
        lp = C.loss(C.forward(X, C.unpack(fp))[0], T)
        lm = C.loss(C.forward(X, C.unpack(fm))[0], T)
        fd = (lp - lm) / (2 * h)
        assert abs(fd - gflat[k]) <= 1e-6 * max(1e-3, abs(fd)), (k, fd, gflat[k])


def test_loss_gradient_ignores_padded_outputs():
    rng = np.random.default_rng(2)
    p = rand_params(rng)
    X = rng.standard_normal((5, C.N_IN))
    T = rng.standard_normal((5, C.N_OUT))
    Y, cache = C.forward(X, p)
    g = C.backward(Y, T, cache, p)
    assert np.all(g["W3"][C.N_OUT_USED:] == 0) and np.all(g["b3"][C.N_OUT_USED:] == 0)


def test_adam_matches_torch():
    rng = np.random.default_rng(3)
    p = rand_params(rng)
    tp = {k: torch.tensor(v, requires_grad=True) for k, v in p.items()}
    opt = torch.optim.Adam(list(tp.values()), lr=1e-3, betas=(0.9, 0.999), eps=1e-8)
    state = {}
    for _ in range(3):
        g = {k: rng.standard_normal(v.shape) for k, v in p.items()}
        p = C.adam(p, g, state, 1e-3)
        for k, t in tp.items():
            t.grad = torch.from_numpy(g[k])
        opt.step()
    for k in p:
        assert np.abs(p[k] - tp[k].detach().numpy()).max() < 1e-14


def test_bf16_round_matches_torch():
    rng = np.random.default_rng(4)
    x = rng.standard_normal(10000) * np.exp(rng.uniform(-20, 20, 10000))
    ref = torch.from_numpy(x.astype(np.float32)).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(C.bf16_round(x), ref)


def test_coarsen_brute_force_and_mass():
    rng = np.random.default_rng(5)
    f = rng.standard_normal((27, 4, 6, 8))
    cf = C.coarsen(f)
    assert cf.shape == (27, 2, 3, 4)
    for (i, z, y, x) in [(0, 0, 0, 0), (5, 1, 2, 3), (26, 1, 0, 2)]:
        ref = np.mean([f[i, 2 * z + a, 2 * y + b, 2 * x + c]
                       for a in (0, 1) for b in (0, 1) for c in (0, 1)])
        assert abs(cf[i, z, y, x] - ref) < 1e-15
    assert abs(cf.sum() * 8 - f.sum()) < 1e-11


def test_features_brute_force():
    rng = np.random.default_rng(6)
    nx, ny, nz = 5, 4, 3
    mom = rng.standard_normal((10, nz, ny, nx))
    mean = rng.standard_normal(10)
    inv = rng.uniform(0.5, 2.0, 10)
    X = C.features(mom, mean, inv)
    for (x, y, z) in [(0, 0, 0), (4, 3, 2), (2, 1, 1)]:
        cell = (z * ny + y) * nx + x
        for nb in range(27):
            dx, dy, dz = nb % 3 - 1, (nb // 3) % 3 - 1, nb // 9 - 1
            for k in range(10):
                v = mom[k, (z + dz) % nz, (y + dy) % ny, (x + dx) % nx]
                assert abs(X[cell, 10 * nb + k] - (v - mean[k]) * inv[k]) < 1e-14
        assert np.all(X[cell, 270:] == 0)


def test_targets_vanish_on_regularized_populations_and_rebuild_f():
    c, w = O.lattice_tables(O.D3Q27)
    rng = np.random.default_rng(7)
    shape = (3, 2, 2)
    f = w[:, None, None, None] * (1 + 0.1 * rng.standard_normal((27, 2, 2, 3)))
    # the regularized populations (tau -> infinity) have no residual
    freg = np.stack([O.collide_cell(O.D3Q27, f[:, z, y, x], 1e15)
                     for z in range(2) for y in range(2) for x in range(3)], axis=1)
    freg = freg.reshape(27, 2, 2, 3)
    assert np.abs(C.targets(freg)).max() < 1e-13
    # f = f_RR + sum over the 17 members of w pref_k H_k delta_k
    H, pref = O.hermite_basis(O.D3Q27)
    d = C.targets(f)
    fr = f.reshape(27, -1)
    frr = freg.reshape(27, -1)
    rebuilt = frr + (w[:, None] * (H[10:27].T * pref[10:27]) @ d.T)
    assert np.abs(rebuilt - fr).max() < 1e-14


def test_closure_collision_special_cases():
    c, w = O.lattice_tables(O.D3Q27)
    H, _ = O.hermite_basis(O.D3Q27)
    rng = np.random.default_rng(8)
    f = w * (1 + 0.1 * rng.standard_normal(27))
    tau = 0.8
    rr = O.collide_cell(O.D3Q27, f, tau)
    assert np.array_equal(O.collide_cell_closure(f, tau, np.zeros(17)), rr)
    delta = 1e-3 * rng.standard_normal(17)
    post = O.collide_cell_closure(f, tau, delta)
    # orders 0..2 untouched, orders 3..6 shifted by (1 - 1/tau) delta
    assert np.abs(H[:10] @ (post - rr)).max() < 1e-16
    assert np.abs(H[10:] @ (post - rr) - (1 - 1 / tau) * delta).max() < 1e-16


def test_step_closure_with_zero_network_is_rr():
    from paper_1505_06900_gb300 import workloads as W
    shape = (4, 4, 4)
    rho, u = W.random_field(shape, 3, seed=9)
    tau = 0.7
    f = O.init(O.D3Q27, shape, tau, rho, u)
    p = C.unpack(np.zeros(C.N_PARAMS))
    got = C.step_closure(f, tau, p, np.zeros(10), np.ones(10), np.ones(17))
    assert np.abs(got - O.step(O.D3Q27, shape, tau, f, 1)).max() < 1e-16


# ----------------------------------------- step-matching targets, coarsening --
def _random_state(shape, seed, amp=0.03):
    """Positive D3Q27 populations near rest with every Hermite mode excited."""
    rng = np.random.default_rng(seed)
    nx, ny, nz = shape
    _, w = O.lattice_tables(O.D3Q27)
    return w[:, None, None, None] * (1.0 + amp * rng.standard_normal((27, nz, ny, nx)))


def _stream(post):
    cvel, _ = O.lattice_tables(O.D3Q27)
    out = np.empty_like(post)
    for i in range(27):
        out[i] = np.roll(post[i], shift=(cvel[i, 2], cvel[i, 1], cvel[i, 0]), axis=(0, 1, 2))
    return out


def test_step_targets_vanish_on_a_plain_rr_update():
    """If B is the plain RR update of A, no correction is needed: every target
    is zero (to round-off), whatever the state (brute force against the
    oracle's own collide-and-stream)."""
    shape, tau = (5, 4, 3), 0.63
    f = _random_state(shape, 10)
    g = O.step(O.D3Q27, shape, tau, f, 1)
    t = C.step_targets(f, g, tau)
    assert np.abs(t).max() < 1e-13


def test_step_targets_recover_a_planted_correction():
    """If B is A collided with a known correction delta (orders 3..6 added to
    the off-equilibrium coefficients before the relaxation, the oracle's
    closure collision) and streamed, the targets are delta, cell by cell."""
    shape, tau = (4, 5, 3), 0.58
    f = _random_state(shape, 11)
    rng = np.random.default_rng(12)
    n = int(np.prod(shape))
    delta = 1e-3 * rng.standard_normal((n, C.N_OUT_USED))
    ff = f.reshape(27, -1)
    post = np.stack([O.collide_cell_closure(ff[:, c], tau, delta[c]) for c in range(n)], axis=1)
    g = _stream(post.reshape(f.shape))
    t = C.step_targets(f, g, tau)
    assert np.abs(t - delta).max() < 1e-13


def test_coarsen_neq_keeps_moments_and_scales_the_off_equilibrium_part():
    shape = (4, 6, 2)
    f = _random_state((8, 12, 4), 13)
    fb = C.coarsen(f)
    assert np.abs(C.coarsen_neq(f, 1.0) - fb).max() < 1e-15
    H, _ = O.hermite_basis(O.D3Q27)
    rho, u, _ = O.fields(O.D3Q27, shape, fb)
    n = int(np.prod(shape))
    f0 = np.stack([O.feq_cell(O.D3Q27, rho.reshape(-1)[c], u.reshape(3, -1)[:, c])
                   for c in range(n)], axis=1)
    for s in (0.0, 1.7, 2.0):
        g = C.coarsen_neq(f, s)
        r2, u2, _ = O.fields(O.D3Q27, shape, g)
        assert np.abs(r2 - rho).max() < 1e-14 and np.abs(u2 - u).max() < 1e-14
        # every Hermite coefficient of the off-equilibrium part scales by s
        a = H @ (fb.reshape(27, -1) - f0)
        b = H @ (g.reshape(27, -1) - f0)
        assert np.abs(b - s * a).max() < 1e-14
    assert np.abs(C.coarsen_neq(f, 0.0).reshape(27, -1) - f0).max() < 1e-15


def test_coarsen_neq_scale_matches_the_constitutive_relation_on_the_coarse_grid():
    """Sec. 3.3: a1^(2) = -2 c_s^2 rho tau S in lattice units. A fine shear
    wave u_x = U sin(2 pi y / L), initialised with that off-equilibrium part at
    tau_f, box-filtered with s = 2 tau_c / tau_f carries the coarse grid's own
    relation at tau_c (S per coarse cell is twice S per fine cell); with s = 1
    the filtered Pi^(1) is tau_f / (2 tau_c) of it (here 0.62)."""
    nf, U = 32, 0.02
    nc = nf // 2
    tau_f = 0.8
    tau_c = 0.5 + (tau_f - 0.5) / 2
    y = (np.arange(nf) + 0.5) / nf
    u = np.zeros((3, 2, nf, 2))
    u[0] = U * np.sin(2 * np.pi * y)[None, :, None]
    rho = np.ones((2, nf, 2))
    f = O.init(O.D3Q27, (2, nf, 2), tau_f, rho, u, O.INIT_EQ_NEQ_FD)
    yc = (np.arange(nc) + 0.5) / nc
    s_xy = 0.5 * U * (2 * np.pi / nc) * np.cos(2 * np.pi * yc)  # du_x/dy per coarse cell / 2
    want = -2.0 * (1.0 / 3.0) * tau_c * s_xy
    for scale, tol in ((2 * tau_c / tau_f, 0.02), (1.0, None)):
        g = C.coarsen_neq(f, scale)
        _, _, pi = O.fields(O.D3Q27, (1, nc, 1), g)
        got = pi[1, 0, :, 0]  # xy
        err = np.abs(got - want).max() / np.abs(want).max()
        if tol is not None:
            assert err < tol, err
        else:
            assert err > 0.3, err


def test_closure_step_dead_zone():
    """A dead zone at least as wide as every standardised prediction leaves
    plain RR (the oracle's own collide-and-stream); none leaves the plain
    closure step; in between, the correction of a prediction y is the one of
    sign(y)(|y| - theta), continuous in theta."""
    shape, tau = (4, 3, 3), 0.6
    rng = np.random.default_rng(14)
    f = _random_state(shape, 15, amp=0.01)
    p = C.unpack(0.05 * rng.standard_normal(C.N_PARAMS))
    mean, inv = np.zeros(10), np.full(10, 30.0)
    out_scale = np.full(17, 1e-3)
    X = C.features(C.moment_field(f), mean, inv)
    ymax = np.abs(C.forward(X, p)[0][:, :17]).max()
    wide = C.step_closure(f, tau, p, mean, inv, out_scale, dead_zone=ymax * 1.01)
    assert np.abs(wide - O.step(O.D3Q27, shape, tau, f, 1)).max() < 1e-15
    none = C.step_closure(f, tau, p, mean, inv, out_scale, dead_zone=0.0)
    plain = C.step_closure(f, tau, p, mean, inv, out_scale)
    assert np.array_equal(none, plain)
    a = C.step_closure(f, tau, p, mean, inv, out_scale, dead_zone=0.3 * ymax)
    b = C.step_closure(f, tau, p, mean, inv, out_scale, dead_zone=0.3 * ymax + 1e-7)
    assert np.abs(a - b).max() < 1e-8
    assert np.abs(a - plain).max() > 1e-6 and np.abs(a - wide).max() > 1e-6
