"""Failure detection on the GPU without a fault: a bounded wait that expires
is recorded in a device status word, reported once as LB_ETIMEOUT by the
next synchronising call, and the context stays usable.

The self-test waits on an mbarrier nothing arrives on, so its wait must
expire. The kernels' own waits are shortened to one try-wait; whether one
then expires depends on timing, so those tests check that a reported
timeout carries LB_ETIMEOUT and that, with the default limit restored, the
same context reproduces a fresh context's results bit for bit.
"""
import numpy as np
import pytest

from paper_1505_06900_gb300 import binding as B
from paper_1505_06900_gb300 import workloads as W

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def test_a_wait_that_nothing_completes_times_out():
    assert B.wait_selftest(1000) == B.LB_ETIMEOUT


def _fields(shape, seed):
    rho, u = W.as_f32(*W.random_field(shape, 3, seed=seed, a_rho=0.01, a_u=0.03))
    return (torch.from_numpy(rho.astype(np.float32)).cuda(),
            torch.from_numpy(u.astype(np.float32)).cuda())


def _reported(call):
    """True if the call raised LB_ETIMEOUT, False if it succeeded."""
    try:
        call()
        return False
    except B.LBError as e:
        assert e.code == B.LB_ETIMEOUT, e
        return True


def test_whole_row_kernel_timeout_and_recovery():
    shape = (144, 4, 3)  # nx % 16 == 0, not a multiple of 128: the whole-row 16-bit kernel
    rho, u = _fields(shape, 3)
    with B.Solver(B.D3Q27, shape, 0.6, storage=B.STORE_F16) as s, \
            B.Solver(B.D3Q27, shape, 0.6, storage=B.STORE_F16) as fresh:
        s.set_wait_limit(1)
        s.init_fields(rho, u)
        s.step(4)
        timed_out = _reported(s.diagnostics)
        print("whole-row kernel with one try-wait: timeout reported =", timed_out)
        assert not _reported(s.diagnostics)  # reported once, then cleared
        s.set_wait_limit(0)
        s.init_fields(rho, u)
        s.step(4)
        fresh.init_fields(rho, u)
        fresh.step(4)
        assert np.array_equal(s.populations().cpu().numpy(), fresh.populations().cpu().numpy())
        assert np.array_equal(s.diagnostics(), fresh.diagnostics())


def test_network_kernel_timeout_and_recovery():
    shape = (256, 16, 16)  # whole 128-cell row tiles: the TMA-fed network
    rng = np.random.default_rng(0)
    params = (0.02 * rng.standard_normal(B.MLP_PARAMS)).astype(np.float32)
    rho, u = _fields(shape, 4)
    net = B.MLP(params)
    net.set_scaling(np.zeros(10), np.full(10, 10.0), np.full(17, 1e-6))
    try:
        with B.Solver(B.D3Q27, shape, 0.6) as s, B.Solver(B.D3Q27, shape, 0.6) as fresh:
            s.init_fields(rho, u)
            s.set_closure(net, bound=1e6)
            net.set_wait_limit(1)
            s.step(2)
            timed_out = _reported(s.closure_fallbacks)
            print("network kernel with one try-wait: timeout reported =", timed_out)
            net.set_wait_limit(0)
            s.init_fields(rho, u)
            s.step(2)
            fresh.init_fields(rho, u)
            fresh.set_closure(net, bound=1e6)
            fresh.step(2)
            assert s.closure_fallbacks() == fresh.closure_fallbacks() or timed_out
            assert np.array_equal(s.populations().cpu().numpy(),
                                  fresh.populations().cpu().numpy())
    finally:
        net.close()


def test_training_kernel_timeout_changes_no_parameter():
    """The training kernel's waits shortened to one try-wait: a step whose
    wait expired reports LB_ETIMEOUT and leaves the parameters (and the Adam
    state) as they were; with the default limit the same network then trains
    exactly as a fresh copy does."""
    rng = np.random.default_rng(3)
    params = (0.05 * rng.standard_normal(B.MLP_PARAMS)).astype(np.float32)
    X = torch.from_numpy(rng.standard_normal((1000, 288)).astype(np.float32)).cuda()
    X[:, 270:] = 0
    X = X.to(torch.bfloat16)
    T = torch.from_numpy(rng.standard_normal((1000, 32)).astype(np.float32)).cuda()
    net, fresh = B.MLP(params), B.MLP(params)
    try:
        net.set_wait_limit(1)
        timed_out = _reported(lambda: net.train_step(X, T, 1e-3))
        print("training kernel with one try-wait: timeout reported =", timed_out)
        if timed_out:
            assert np.array_equal(net.get_params(), params)
        net.set_wait_limit(0)
        if not timed_out:
            fresh.train_step(X, T, 1e-3)
        for _ in range(3):
            assert net.train_step(X, T, 1e-3) == fresh.train_step(X, T, 1e-3)
        assert np.array_equal(net.get_params(), fresh.get_params())
    finally:
        net.close()
        fresh.close()
