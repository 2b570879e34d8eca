"""Entry points that take caller device buffers reject memory the context's
device cannot use as its own (here host numpy memory) with LB_EINVAL, before
any kernel runs, and the context keeps working afterwards."""
import ctypes

import numpy as np
import pytest

from paper_1505_06900_gb300 import binding as B
from paper_1505_06900_gb300 import workloads as W

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _host(n):
    a = np.zeros(n, dtype=np.float32)
    return a, a.ctypes.data


def test_host_pointers_are_rejected_and_the_context_survives():
    shape = (16, 8, 4)
    n = int(np.prod(shape))
    lib = B.load()
    rho, u = W.as_f32(*W.random_field(shape, 3, seed=5, a_u=0.02))
    rho_d = torch.from_numpy(rho.astype(np.float32)).cuda()
    u_d = torch.from_numpy(u.astype(np.float32)).cuda()
    keep = []
    with B.Solver(B.D3Q27, shape, 0.7) as s:
        s.init_fields(rho_d, u_d)
        s.step(3)
        before = s.populations().cpu().numpy()
        h = s.handle
        for call in (
            lambda p: lib.lb_init_fields(h, p, B._ptr(u_d), B.INIT_EQ_NEQ_FD),
            lambda p: lib.lb_moments(h, p, None, None),
            lambda p: lib.lb_get_populations(h, p),
            lambda p: lib.lb_set_populations(h, p),
        ):
            a, p = _host(27 * n)
            keep.append(a)
            assert call(p) == B.LB_EINVAL
            assert "device memory" in lib.lb_last_error(h).decode()
        # nothing was touched: the state is the one before, and updates go on
        assert np.array_equal(s.populations().cpu().numpy(), before)
        s.step(1)
        assert np.isfinite(s.diagnostics()).all()
    net = B.MLP()
    X = torch.zeros((64, 288), dtype=torch.bfloat16, device="cuda")
    a, p = _host(64 * 32)
    assert lib.lb_mlp_forward(net.handle, B._ptr(X), 64, p) == B.LB_EINVAL
    assert "device memory" in lib.lb_mlp_last_error(net.handle).decode()
    T = torch.zeros((64, 32), dtype=torch.float32, device="cuda")
    g, pg = _host(B.MLP_PARAMS)
    loss = ctypes.c_double()
    assert lib.lb_mlp_gradients(net.handle, B._ptr(X), B._ptr(T), 64, pg,
                                ctypes.byref(loss)) == B.LB_EINVAL
    Y = net.forward(X)  # the network still runs
    assert torch.isfinite(Y).all()
    net.close()


def test_closure_entry_points_validate_their_arguments():
    """Invalid closure arguments are refused with LB_EINVAL and a message:
    a non-finite off-equilibrium scale, states on different grids, a negative
    or non-finite dead zone, and the inspection step on a context without a
    fused closure."""
    lib = B.load()
    net = B.MLP()
    with B.Solver(B.D3Q27, (8, 6, 4), 0.7) as fine, B.Solver(B.D3Q27, (4, 3, 2), 0.6) as coarse, \
            B.Solver(B.D3Q27, (4, 3, 4), 0.6) as other:
        assert lib.lb_coarsen_neq(fine.handle, coarse.handle, float("nan")) == B.LB_EINVAL
        assert "neq_scale" in lib.lb_last_error(coarse.handle).decode()
        T = torch.empty((coarse.n, 32), device="cuda")
        assert lib.lb_closure_step_targets(coarse.handle, other.handle, net.handle,
                                           B._ptr(T)) == B.LB_EINVAL
        assert "grid" in lib.lb_last_error(coarse.handle).decode()
        for dz in (-0.1, float("inf")):
            assert lib.lb_set_closure_ex(coarse.handle, net.handle, 8.0, dz) == B.LB_EINVAL
            assert "dead_zone" in lib.lb_last_error(coarse.handle).decode()
    tr = torch.empty((80 * 3 * 4, 145), device="cuda")
    xs = torch.empty((6 * 5 * 82 * 16,), dtype=torch.bfloat16, device="cuda")
    with B.Solver(B.D3Q27, (80, 3, 4), 0.7) as s:
        # no closure set, then a closure on rows that are not whole 128-cell tiles
        assert lib.lb_closure_step_trace(s.handle, B._ptr(tr), B._ptr(xs)) == B.LB_EINVAL
        s.set_closure(net)
        assert lib.lb_closure_step_trace(s.handle, B._ptr(tr), B._ptr(xs)) == B.LB_EINVAL
        assert "128-cell" in lib.lb_last_error(s.handle).decode()
    net.close()
