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
