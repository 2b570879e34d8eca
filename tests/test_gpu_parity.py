"""Parity of the CUDA library (through its C ABI) with the FP64 CPU oracle.

Tolerances (float32 arithmetic and storage):
  * one update:  max over cells and i of |f_gpu - f_oracle| / w_i <= 1e-6
  * 1000 updates: relative L2 error of u <= 1e-5 and of rho <= 1e-6
Inputs are seeded and rounded to float32 before both sides see them.
"""
import math

import numpy as np
import pytest

import oracle as O
from _common import f64_state, max_rel_to_weight, rel_l2, shifted, weights
from paper_1505_06900_gb300 import binding as B
from paper_1505_06900_gb300 import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

ONE_STEP_TOL = 1e-6

# shapes span several 128-wide x tiles with a ragged tail, and non-cubic extents
CASES = [
    (O.D2Q9, (300, 7, 1)),
    (O.D2Q9, (5, 3, 1)),
    (O.D3Q27, (150, 6, 5)),
    (O.D3Q27, (3, 4, 5)),
    (O.D3Q19, (150, 6, 5)),
    (O.D3Q19, (3, 4, 5)),
]
# one case per lattice, several tiles with a ragged tail
LARGE = [CASES[0], CASES[2], CASES[4]]


def _cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


def _random_state(lattice, shape, seed, amp=0.05):
    _, q = O.dims_of(lattice)
    return W.random_populations(q, shape, seed, amp).astype(np.float32)


def _solver(lattice, shape, tau, storage=B.STORE_F32, collision=B.COLLIDE_RR):
    return B.Solver(lattice, shape, tau, storage=storage, collision=collision)


@pytest.mark.parametrize("lattice,shape", CASES)
@pytest.mark.parametrize("collision", [B.COLLIDE_RR, B.COLLIDE_REG2, B.COLLIDE_BGK])
def test_steps_match_oracle(lattice, shape, collision):
    """Updates 1, 2 and 3 (both AA kernels) against the oracle's pull update."""
    tau = 0.62
    df = _random_state(lattice, shape, seed=100 + lattice)
    variant = {B.COLLIDE_RR: O.RR, B.COLLIDE_REG2: O.REG2, B.COLLIDE_BGK: O.BGK}[collision]
    with _solver(lattice, shape, tau, collision=collision) as s:
        s.set_populations(_cuda(df))
        f = f64_state(lattice, df)
        for k in range(1, 4):
            s.step(1)
            got = s.populations().cpu().numpy()
            f = O.step(lattice, shape, tau, f, 1, variant)
            err = max_rel_to_weight(lattice, got, shifted(lattice, f))
            assert err <= ONE_STEP_TOL, (k, err)


@pytest.mark.parametrize("lattice,shape", LARGE)
def test_moments_after_even_and_odd_updates(lattice, shape):
    d, _ = O.dims_of(lattice)
    tau = 0.75
    df = _random_state(lattice, shape, seed=7)
    with _solver(lattice, shape, tau) as s:
        s.set_populations(_cuda(df))
        f = f64_state(lattice, df)
        for k in range(3):
            rho, u, p = (t.cpu().numpy() for t in s.moments())
            r0, u0, p0 = O.fields(lattice, shape, f)
            assert np.max(np.abs(rho - r0)) < 1e-6
            assert np.max(np.abs(u - u0)) < 1e-6
            assert np.max(np.abs(p - p0)) < 1e-6
            s.step(1)
            f = O.step(lattice, shape, tau, f, 1)


@pytest.mark.parametrize("lattice,shape", LARGE)
@pytest.mark.parametrize("mode", [B.INIT_EQ, B.INIT_EQ_NEQ_FD])
def test_init_matches_oracle(lattice, shape, mode):
    d, _ = O.dims_of(lattice)
    rho, u = W.as_f32(*W.random_field(shape, d, seed=5))
    with _solver(lattice, shape, 0.7) as s:
        s.init_fields(_cuda(rho), _cuda(u), mode)
        got = s.populations().cpu().numpy()
    f = O.init(lattice, shape, 0.7, rho, u, mode)
    assert max_rel_to_weight(lattice, got, shifted(lattice, f)) <= ONE_STEP_TOL


def test_taylor_green_2d_1000_steps():
    """D2Q9 128^2 Taylor-Green vortex, Re = 100, 1000 updates vs the oracle."""
    n, u0 = 128, 0.05
    tau = W.taylor_green_2d_tau(n, u0)
    rho, u = W.as_f32(*W.taylor_green_2d(n, u0))
    shape = (n, n, 1)
    with _solver(O.D2Q9, shape, tau) as s:
        s.init_fields(_cuda(rho), _cuda(u))
        s.step(1000)
        r_g, u_g, _ = (t.cpu().numpy() for t in s.moments())
    f = O.step(O.D2Q9, shape, tau, O.init(O.D2Q9, shape, tau, rho, u), 1000)
    r_o, u_o, _ = O.fields(O.D2Q9, shape, f)
    assert rel_l2(u_g, u_o) <= 1e-5
    assert rel_l2(r_g, r_o) <= 1e-6


@pytest.mark.parametrize("mach", [0.1, 0.3, 0.5])
def test_double_shear_layer_128_1000_steps(mach):
    """The 128^2 copy of the D2Q9 double shear layer (Re 1000 on L = 128), 1000
    updates against the oracle, at each Mach number of the 2048^2 workload."""
    n = 128
    tau = W.double_shear_2d_tau(n, mach)
    rho, u = W.as_f32(*W.double_shear_2d(n, mach))
    shape = (n, n, 1)
    with _solver(O.D2Q9, shape, tau) as s:
        s.init_fields(_cuda(rho), _cuda(u))
        s.step(1000)
        r_g, u_g, _ = (t.cpu().numpy() for t in s.moments())
    f = O.step(O.D2Q9, shape, tau, O.init(O.D2Q9, shape, tau, rho, u), 1000)
    r_o, u_o, _ = O.fields(O.D2Q9, shape, f)
    assert rel_l2(u_g, u_o) <= 1e-5
    assert rel_l2(r_g, r_o) <= 1e-6


@pytest.mark.parametrize("lattice", [O.D3Q27, O.D3Q19])
def test_taylor_green_3d_1000_steps(lattice):
    """3-D Taylor-Green vortex (Ma = 0.1, Re = 1600) on 24^3, 1000 updates."""
    n, mach = 24, 0.1
    tau = W.taylor_green_3d_tau(n, mach)
    rho, u = W.as_f32(*W.taylor_green_3d(n, mach))
    shape = (n, n, n)
    with _solver(lattice, shape, tau) as s:
        s.init_fields(_cuda(rho), _cuda(u))
        s.step(1000)
        r_g, u_g, _ = (t.cpu().numpy() for t in s.moments())
    f = O.step(lattice, shape, tau, O.init(lattice, shape, tau, rho, u), 1000)
    r_o, u_o, _ = O.fields(lattice, shape, f)
    assert rel_l2(u_g, u_o) <= 1e-5
    assert rel_l2(r_g, r_o) <= 1e-6


@pytest.mark.parametrize("lattice,shape", [(O.D2Q9, (64, 48, 1)), (O.D3Q27, (20, 16, 12)),
                                           (O.D3Q19, (20, 16, 12))])
def test_diagnostics_and_enstrophy(lattice, shape):
    d, _ = O.dims_of(lattice)
    rho, u = W.as_f32(*W.random_field(shape, d, seed=9, a_u=0.03))
    tau = 0.8
    with _solver(lattice, shape, tau) as s:
        s.init_fields(_cuda(rho), _cuda(u))
        s.step(3)
        dg = s.diagnostics()
        en = s.enstrophy()
        df = s.populations().cpu().numpy()
    f = O.step(lattice, shape, tau, O.init(lattice, shape, tau, rho, u), 3)
    dref = O.diagnostics(lattice, shape, f)
    assert abs(dg[0] - dref[0]) <= 1e-9 * dref[0]
    assert np.allclose(dg[1:1 + d], dref[1:1 + d], rtol=0, atol=1e-5)
    assert abs(dg[-1] / dref[-1] - 1) < 1e-5
    assert abs(en / O.enstrophy(lattice, shape, f) - 1) < 1e-4
    # deterministic: the same state gives bit-identical diagnostics
    with _solver(lattice, shape, tau) as s:
        s.set_populations(_cuda(df))
        a, b = s.diagnostics(), s.diagnostics()
        assert np.array_equal(a, b)


def test_checkpoint_resume_is_bit_exact():
    shape = (40, 12, 10)
    rho, u = W.as_f32(*W.random_field(shape, 3, seed=3))
    with _solver(O.D3Q27, shape, 0.6) as s:
        s.init_fields(_cuda(rho), _cuda(u))
        s.step(7)
        buf = torch.empty(s.state_bytes(), dtype=torch.uint8, device="cuda")
        par = s.get_state(buf)
        assert par == 1
        s.step(5)
        a = s.populations().cpu().numpy()
        s.set_state(buf, par)
        s.step(5)
        b = s.populations().cpu().numpy()
    assert np.array_equal(a, b)


def test_step_zero_and_argument_errors():
    shape = (16, 8, 1)
    with _solver(O.D2Q9, shape, 0.7) as s:
        df = _random_state(O.D2Q9, shape, 1)
        s.set_populations(_cuda(df))
        s.step(0)
        assert np.array_equal(s.populations().cpu().numpy(), df)
        with pytest.raises(B.LBError) as e:
            s.step(-1)
        assert e.value.code == B.LB_EINVAL
        # a failed call leaves the state unchanged
        assert np.array_equal(s.populations().cpu().numpy(), df)


def test_divergence_is_reported():
    """A non-finite population makes the diagnostics return LB_EDIVERGED."""
    shape = (8, 8, 1)
    df = np.zeros((9, 1, 8, 8), np.float32)
    df[3, 0, 2, 2] = np.nan
    with _solver(O.D2Q9, shape, 0.7) as s:
        s.set_populations(_cuda(df))
        with pytest.raises(B.LBError) as e:
            s.diagnostics()
        assert e.value.code == B.LB_EDIVERGED


def test_run_host_matches_device_path():
    n = 64
    rho, u = W.as_f32(*W.taylor_green_2d(n, 0.05))
    tau = 0.6
    shape = (n, n, 1)
    rho_o = np.zeros((1, n, n), np.float32)
    u_o = np.zeros((2, 1, n, n), np.float32)
    diag = np.zeros(4)
    with _solver(O.D2Q9, shape, tau) as s:
        s.run_host(rho.astype(np.float32), u.astype(np.float32), 25, rho_out=rho_o, u_out=u_o,
                   diag_out=diag)
    with _solver(O.D2Q9, shape, tau) as s:
        s.init_fields(_cuda(rho), _cuda(u))
        s.step(25)
        r, uu, _ = (t.cpu().numpy() for t in s.moments())
        d2 = s.diagnostics()
    assert np.array_equal(rho_o, r) and np.array_equal(u_o, uu)
    assert np.array_equal(diag, d2)


@pytest.mark.parametrize("lattice,shape,walls", [(O.D2Q9, (40, 24, 1), 0), (O.D3Q27, (16, 12, 10), 0),
                                                 (O.D3Q19, (16, 12, 10), 0),
                                                 (O.D2Q9, (21, 21, 1), 3)])
@pytest.mark.parametrize("storage", [B.STORE_F32, B.STORE_F16])
def test_step_runs_replayed_as_graphs_equal_single_updates(lattice, shape, walls, storage):
    """lb_step(n) replays a captured CUDA graph for runs of updates; the
    result is bit for bit that of n calls of lb_step(1), from either parity."""
    d, _ = O.dims_of(lattice)
    rho, u = W.as_f32(*W.random_field(shape, d, seed=23, a_rho=0.01, a_u=0.03))
    with B.Solver(lattice, shape, 0.66, storage=storage, walls=walls) as a, \
            B.Solver(lattice, shape, 0.66, storage=storage, walls=walls) as b:
        for s in (a, b):
            s.init_fields(_cuda(rho), _cuda(u))
        a.step(37)
        a.step(1)
        a.step(20)  # a run that starts at the odd parity
        for _ in range(58):
            b.step(1)
        assert a.info()["steps"] == b.info()["steps"] == 58
        assert np.array_equal(a.populations().cpu().numpy(), b.populations().cpu().numpy())


@pytest.mark.parametrize("lattice,shape", [(O.D3Q27, (1, 1, 1)), (O.D3Q19, (1, 1, 1)),
                                           (O.D2Q9, (1, 1, 1)), (O.D3Q27, (1, 5, 4)),
                                           (O.D3Q19, (4, 1, 3)), (O.D2Q9, (1, 7, 1))])
def test_degenerate_grids_match_oracle(lattice, shape):
    """One-cell and one-column periodic grids: every neighbour along a unit
    axis is the cell itself (the wrap of the AA gather and scatter)."""
    tau = 0.7
    df = _random_state(lattice, shape, seed=61)
    with _solver(lattice, shape, tau) as s:
        s.set_populations(_cuda(df))
        f = f64_state(lattice, df)
        for k in range(3):
            s.step(1)
            f = O.step(lattice, shape, tau, f, 1)
            err = max_rel_to_weight(lattice, s.populations().cpu().numpy(), shifted(lattice, f))
            assert err <= ONE_STEP_TOL, (k, err)


@pytest.mark.parametrize("lattice", [O.D2Q9, O.D3Q19, O.D3Q27])
@pytest.mark.parametrize("storage", [B.STORE_F32, B.STORE_F16, B.STORE_BF16])
def test_rest_and_uniform_flow_are_kept(lattice, storage):
    """The rest state is a fixed point bit for bit (df = 0 stays 0), and a
    uniform flow stays uniform bit for bit: every cell runs the same
    arithmetic, whatever the AA parity and the kernel."""
    d, _ = O.dims_of(lattice)
    shape = (256, 4, 3) if d == 3 else (256, 6, 1)
    with _solver(lattice, shape, 0.6, storage=storage) as s:
        s.step(20)
        assert not np.any(s.populations().cpu().numpy())
        rho = np.full(shape[::-1], 1.01, np.float32)
        u = np.zeros((d,) + shape[::-1], np.float32)
        u[0], u[1] = 0.05, -0.02
        s.init_fields(_cuda(rho), _cuda(u), B.INIT_EQ)
        s.step(21)
        df = s.populations().cpu().numpy().reshape(s.q, -1)
        assert np.all(df == df[:, :1])
        r, uu, _ = (t.cpu().numpy() for t in s.moments())
        assert np.all(r == r.flat[0]) and np.all(uu[0] == uu[0].flat[0])
        assert abs(float(uu[0].flat[0]) - 0.05) < (1e-6 if storage == B.STORE_F32 else 2e-3)


def test_side_stream_and_caller_graph_capture():
    """A context on a side stream (graph replay included) gives the results of
    one on the default stream, bit for bit; inside the caller's own CUDA-graph
    capture lb_step records its updates one by one into that capture, and
    replaying the captured graph advances the state as the direct call does."""
    shape = (64, 12, 10)
    rho, u = W.as_f32(*W.random_field(shape, 3, seed=71, a_rho=0.01, a_u=0.03))
    rd, ud = _cuda(rho), _cuda(u)
    with _solver(O.D3Q27, shape, 0.62) as ref:
        ref.init_fields(rd, ud)
        ref.step(40)
        want = ref.populations().cpu().numpy()
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        with B.Solver(O.D3Q27, shape, 0.62, stream=side) as s:
            s.init_fields(rd, ud)
            s.step(24)
            g = torch.cuda.CUDAGraph()
            with torch.cuda.graph(g, stream=side, capture_error_mode="thread_local"):
                s.set_stream(side)
                s.step(16)
            g.replay()
            side.synchronize()
            assert s.info()["steps"] == 40
            got = s.populations().cpu().numpy()
    assert np.array_equal(got, want)

