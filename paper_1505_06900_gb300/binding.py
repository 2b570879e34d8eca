"""ctypes binding of liblbrr.so (the C ABI of include/lbrr.h).

Argument marshalling only: every step of the method runs in the library's CUDA
kernels. torch supplies device memory and the stream. The library must have
been built (``paper_1505_06900_gb300.build.build()``); ``load()`` raises if it
is missing rather than falling back to anything else.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "_build", "liblbrr.so")

LB_OK, LB_EINVAL, LB_ENOMEM, LB_ECUDA, LB_EDIVERGED, LB_ETIMEOUT = 0, 1, 2, 3, 4, 5
D2Q9, D3Q19, D3Q27 = 9, 19, 27
STORE_F32, STORE_F16, STORE_BF16 = 0, 1, 2
COLLIDE_RR, COLLIDE_REG2, COLLIDE_BGK = 0, 1, 2
WALL_X, WALL_Y, WALL_Z = 1, 2, 4
INIT_EQ, INIT_EQ_NEQ_FD = 0, 1

# every entry point of include/lbrr.h with its ctypes signature
_vp, _i, _d, _ll = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_longlong
SIGNATURES = {
    "lb_create": (_i, [ctypes.POINTER(_vp), _i, _i, _i, _i, _d, _i]),
    "lb_create_ex": (_i, [ctypes.POINTER(_vp), _vp]),
    "lb_destroy": (None, [_vp]),
    "lb_last_error": (ctypes.c_char_p, [_vp]),
    "lb_set_stream": (_i, [_vp, _vp]),
    "lb_init_fields": (_i, [_vp, _vp, _vp, _i]),
    "lb_step": (_i, [_vp, _i]),
    "lb_moments": (_i, [_vp, _vp, _vp, _vp]),
    "lb_diagnostics": (_i, [_vp, _vp]),
    "lb_enstrophy": (_i, [_vp, _vp]),
    "lb_get_populations": (_i, [_vp, _vp]),
    "lb_set_populations": (_i, [_vp, _vp]),
    "lb_state_bytes": (_ll, [_vp]),
    "lb_get_state": (_i, [_vp, _vp, ctypes.POINTER(_i)]),
    "lb_set_state": (_i, [_vp, _vp, _i]),
    "lb_run_host": (_i, [_vp, _vp, _vp, _i, _i, _vp, _vp, _vp]),
    "lb_info": (_i, [_vp, ctypes.POINTER(_ll)]),
    "lb_set_wait_limit": (_i, [_vp, _i]),
    "lb_mlp_set_wait_limit": (_i, [_vp, _i]),
    "lb_wait_selftest": (_i, [_i]),
    "lb_diagnostics_static": (_i, [_i, _i, _i, _i, _i, _i, _vp, _vp, _vp]),
    "lb_mlp_create": (_i, [ctypes.POINTER(_vp)]),
    "lb_mlp_destroy": (None, [_vp]),
    "lb_mlp_last_error": (ctypes.c_char_p, [_vp]),
    "lb_mlp_set_stream": (_i, [_vp, _vp]),
    "lb_mlp_set_params": (_i, [_vp, _vp]),
    "lb_mlp_get_params": (_i, [_vp, _vp]),
    "lb_mlp_set_scaling": (_i, [_vp, _vp, _vp, _vp]),
    "lb_mlp_forward": (_i, [_vp, _vp, _ll, _vp]),
    "lb_mlp_gradients": (_i, [_vp, _vp, _vp, _ll, _vp, _vp]),
    "lb_mlp_forward_trace": (_i, [_vp, _vp, _ll, _vp, _vp]),
    "lb_mlp_gradients_trace": (_i, [_vp, _vp, _vp, _ll, _vp, _vp, _vp]),
    "lb_mlp_train_step": (_i, [_vp, _vp, _vp, _ll, ctypes.c_float, _vp]),
    "lb_closure_features": (_i, [_vp, _vp, _vp]),
    "lb_closure_targets": (_i, [_vp, _vp, _vp]),
    "lb_coarsen": (_i, [_vp, _vp]),
    "lb_coarsen_neq": (_i, [_vp, _vp, _d]),
    "lb_set_closure_ex": (_i, [_vp, _vp, ctypes.c_float, ctypes.c_float]),
    "lb_closure_step_trace": (_i, [_vp, _vp, _vp]),
    "lb_closure_step_targets": (_i, [_vp, _vp, _vp, _vp]),
    "lb_set_closure": (_i, [_vp, _vp, ctypes.c_float]),
    "lb_closure_fallbacks": (_i, [_vp, ctypes.POINTER(_ll)]),
}
MLP_PARAMS, MLP_IN, MLP_OUT, MLP_OUT_USED = 24736, 288, 32, 17
LB_STATIC_MAX_CELLS = 134217728


class LBOptions(ctypes.Structure):
    _fields_ = [("lattice", _i), ("nx", _i), ("ny", _i), ("nz", _i), ("tau", _d),
                ("periodic", _i), ("storage", _i), ("collision", _i), ("walls", _i)]


class LBError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"lbrr error {code}: {msg}")
        self.code = code


_lock = threading.Lock()
_lib = None


def load(path: str | None = None):
    """Load liblbrr.so (once). Raises if the library has not been built."""
    global _lib
    with _lock:
        if _lib is None:
            p = path or LIB_PATH
            if not os.path.exists(p):
                raise RuntimeError(f"{p} not found: build it with paper_1505_06900_gb300.build")
            lib = ctypes.CDLL(p)
            for name, (res, args) in SIGNATURES.items():
                fn = getattr(lib, name)
                fn.restype = res
                fn.argtypes = args
            _lib = lib
    return _lib


def dims_of(lattice: int) -> tuple[int, int]:
    if lattice not in (D2Q9, D3Q19, D3Q27):
        raise ValueError(f"unknown lattice {lattice}")
    return (2, 9) if lattice == D2Q9 else (3, lattice)


def _ptr(t) -> int:
    """Device (or host) address of a contiguous torch tensor or numpy array."""
    if t is None:
        return None
    if isinstance(t, np.ndarray):
        assert t.flags["C_CONTIGUOUS"]
        return t.ctypes.data
    assert t.is_contiguous(), "tensors passed to lbrr must be contiguous"
    return t.data_ptr()


class Solver:
    """One lattice Boltzmann context (device population store) of liblbrr.so."""

    def __init__(self, lattice: int, shape, tau: float, storage: int = STORE_F32,
                 collision: int = COLLIDE_RR, stream=None, walls: int = 0):
        import torch
        self._lib = load()
        self.lattice = lattice
        self.d, self.q = dims_of(lattice)
        self.nx, self.ny, self.nz = (list(shape) + [1])[:3] if len(shape) == 2 else shape
        self.n = self.nx * self.ny * self.nz
        self.tau = float(tau)
        self.walls = int(walls)
        opt = LBOptions(lattice, self.nx, self.ny, self.nz, self.tau, 1, storage, collision,
                        self.walls)
        h = ctypes.c_void_p()
        rc = self._lib.lb_create_ex(ctypes.byref(h), ctypes.addressof(opt))
        if rc != LB_OK:
            raise LBError(rc, self._lib.lb_last_error(None).decode())
        self._h = h
        self.device = torch.device("cuda", torch.cuda.current_device())
        self.set_stream(stream if stream is not None else torch.cuda.current_stream())

    # -- plumbing ---------------------------------------------------------
    def _check(self, rc: int):
        if rc != LB_OK:
            raise LBError(rc, self._lib.lb_last_error(self._h).decode())

    def close(self):
        if getattr(self, "_h", None):
            self._lib.lb_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    @property
    def handle(self):
        return self._h

    def set_stream(self, stream):
        self.stream = stream
        self._check(self._lib.lb_set_stream(self._h, ctypes.c_void_p(stream.cuda_stream)))

    def _field(self, comps):
        import torch
        return torch.empty((comps, self.nz, self.ny, self.nx), device=self.device,
                           dtype=torch.float32)

    # -- the method -------------------------------------------------------
    def init_fields(self, rho, u, mode: int = INIT_EQ_NEQ_FD):
        """rho [nz,ny,nx] and u [D,nz,ny,nx] float32 CUDA tensors."""
        import torch
        rho = rho.contiguous()
        u = u.contiguous()
        assert rho.numel() == self.n and u.numel() == self.d * self.n
        assert rho.is_cuda and u.is_cuda
        if rho.dtype != torch.float32 or u.dtype != torch.float32:
            raise TypeError("rho and u must be float32 CUDA tensors")
        self._check(self._lib.lb_init_fields(self._h, _ptr(rho), _ptr(u), int(mode)))
        self._keep = (rho, u)  # keep alive until the stream has consumed them

    def step(self, n: int = 1):
        self._check(self._lib.lb_step(self._h, int(n)))

    def moments(self):
        """(rho [nz,ny,nx], u [D,...], pi1 [3|6,...]) as CUDA tensors."""
        rho, u, p = self._field(1), self._field(self.d), self._field(3 if self.d == 2 else 6)
        self._check(self._lib.lb_moments(self._h, _ptr(rho), _ptr(u), _ptr(p)))
        return rho[0], u, p

    def diagnostics(self) -> np.ndarray:
        out = np.zeros(2 + self.d)
        rc = self._lib.lb_diagnostics(self._h, out.ctypes.data)
        if rc == LB_EDIVERGED:
            raise LBError(rc, self._lib.lb_last_error(self._h).decode())
        self._check(rc)
        return out

    def enstrophy(self) -> float:
        out = np.zeros(1)
        self._check(self._lib.lb_enstrophy(self._h, out.ctypes.data))
        return float(out[0])

    def populations(self):
        """Shifted populations df [Q, nz, ny, nx] (float32, natural order)."""
        out = self._field(self.q)
        self._check(self._lib.lb_get_populations(self._h, _ptr(out)))
        return out

    def set_populations(self, df):
        df = df.contiguous()
        assert df.numel() == self.q * self.n and df.is_cuda
        self._check(self._lib.lb_set_populations(self._h, _ptr(df)))
        self._keep = (df,)

    def state_bytes(self) -> int:
        return int(self._lib.lb_state_bytes(self._h))

    def get_state(self, dst):
        par = ctypes.c_int()
        self._check(self._lib.lb_get_state(self._h, _ptr(dst), ctypes.byref(par)))
        return par.value

    def set_state(self, src, parity: int):
        self._check(self._lib.lb_set_state(self._h, _ptr(src), int(parity)))

    def run_host(self, rho_h: np.ndarray, u_h: np.ndarray, nsteps: int,
                 mode: int = INIT_EQ_NEQ_FD, rho_out=None, u_out=None, diag_out=None):
        """End-to-end run from host arrays (numpy or pinned CPU tensors)."""
        self._check(self._lib.lb_run_host(self._h, _ptr(rho_h), _ptr(u_h), int(mode), int(nsteps),
                                          _ptr(rho_out), _ptr(u_out), _ptr(diag_out)))

    # -- learned closure (D3Q27, FP32 store, RR) ---------------------------
    def coarsen_from(self, fine: "Solver", neq_scale: float | None = None):
        """2x2x2 box average of `fine`'s populations into this context; with
        neq_scale, the off-equilibrium part of each average scaled by it
        (lb_coarsen_neq)."""
        if neq_scale is None:
            self._check(self._lib.lb_coarsen(fine.handle, self._h))
        else:
            self._check(self._lib.lb_coarsen_neq(fine.handle, self._h, float(neq_scale)))

    def closure_step_targets(self, post: "Solver", mlp: "MLP"):
        """Step-matching targets [N, 32] of this state against `post`
        (lb_closure_step_targets)."""
        import torch
        T = torch.empty((self.n, MLP_OUT), device=self.device, dtype=torch.float32)
        self._check(self._lib.lb_closure_step_targets(self._h, post.handle, mlp.handle, _ptr(T)))
        return T

    def closure_features(self, mlp: "MLP"):
        import torch
        X = torch.empty((self.n, MLP_IN), device=self.device, dtype=torch.bfloat16)
        self._check(self._lib.lb_closure_features(self._h, mlp.handle, _ptr(X)))
        return X

    def closure_targets(self, mlp: "MLP"):
        import torch
        T = torch.empty((self.n, MLP_OUT), device=self.device, dtype=torch.float32)
        self._check(self._lib.lb_closure_targets(self._h, mlp.handle, _ptr(T)))
        return T

    def closure_step_trace(self):
        """One closure update with its inspection outputs (lb_closure_step_trace):
        trace [N, 145] FP32 and the feature source [nz+2, ny+2, nx+2, 16] BF16."""
        import torch
        tr = torch.empty((self.n, 145), device=self.device, dtype=torch.float32)
        xs = torch.empty((self.nz + 2, self.ny + 2, self.nx + 2, 16), device=self.device,
                         dtype=torch.bfloat16)
        self._check(self._lib.lb_closure_step_trace(self._h, _ptr(tr), _ptr(xs)))
        return tr, xs

    def set_closure(self, mlp, bound: float = 8.0, dead_zone: float = 0.0):
        """Learned closure for the following updates (None: plain RR); the
        dead zone shrinks each standardised prediction (lb_set_closure_ex)."""
        self._check(self._lib.lb_set_closure_ex(self._h, mlp.handle if mlp else None,
                                                float(bound), float(dead_zone)))
        self._closure = mlp

    def set_wait_limit(self, iterations: int):
        """Main-loop wait limit of this context's mbarrier kernels (0: default)."""
        self._check(self._lib.lb_set_wait_limit(self._h, int(iterations)))

    def closure_fallbacks(self) -> int:
        out = ctypes.c_longlong()
        self._check(self._lib.lb_closure_fallbacks(self._h, ctypes.byref(out)))
        return out.value

    def info(self) -> dict:
        out = (ctypes.c_longlong * 8)()
        self._check(self._lib.lb_info(self._h, out))
        keys = ["lattice", "nx", "ny", "nz", "storage", "collision", "steps", "bytes_per_update"]
        return dict(zip(keys, list(out)))


class MLP:
    """The learned closure's network (device parameters, Adam state, scaling)."""

    def __init__(self, params=None, stream=None):
        import torch
        self._lib = load()
        h = ctypes.c_void_p()
        rc = self._lib.lb_mlp_create(ctypes.byref(h))
        if rc != LB_OK:
            raise LBError(rc, self._lib.lb_last_error(None).decode())
        self._h = h
        self.device = torch.device("cuda", torch.cuda.current_device())
        stream = stream if stream is not None else torch.cuda.current_stream()
        self._check(self._lib.lb_mlp_set_stream(self._h, ctypes.c_void_p(stream.cuda_stream)))
        if params is not None:
            self.set_params(params)

    @property
    def handle(self):
        return self._h

    def _check(self, rc):
        if rc != LB_OK:
            raise LBError(rc, self._lib.lb_mlp_last_error(self._h).decode())

    def close(self):
        if getattr(self, "_h", None):
            self._lib.lb_mlp_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_params(self, params):
        p = np.ascontiguousarray(np.asarray(params, dtype=np.float32).reshape(-1))
        assert p.size == MLP_PARAMS
        self._check(self._lib.lb_mlp_set_params(self._h, p.ctypes.data))

    def get_params(self) -> np.ndarray:
        p = np.zeros(MLP_PARAMS, dtype=np.float32)
        self._check(self._lib.lb_mlp_get_params(self._h, p.ctypes.data))
        return p

    def set_wait_limit(self, iterations: int):
        """Main-loop wait limit of the network kernels (0: default)."""
        self._check(self._lib.lb_mlp_set_wait_limit(self._h, int(iterations)))

    def set_scaling(self, in_mean, in_inv_std, out_scale):
        a = [np.ascontiguousarray(np.asarray(v, dtype=np.float32)) for v in
             (in_mean, in_inv_std, out_scale)]
        assert a[0].size == 10 and a[1].size == 10 and a[2].size == 17
        self._check(self._lib.lb_mlp_set_scaling(self._h, a[0].ctypes.data, a[1].ctypes.data,
                                                 a[2].ctypes.data))
        self.scaling = a

    def forward(self, X, trace: bool = False):
        """Y [M][32]; with trace also H [M][128] (lb_mlp_forward_trace)."""
        import torch
        assert X.dtype == torch.bfloat16 and X.is_cuda and X.shape[1] == MLP_IN
        X = X.contiguous()
        Y = torch.empty((X.shape[0], MLP_OUT), device=X.device, dtype=torch.float32)
        if not trace:
            self._check(self._lib.lb_mlp_forward(self._h, _ptr(X), X.shape[0], _ptr(Y)))
            return Y
        H = torch.empty((X.shape[0], 128), device=X.device, dtype=torch.float32)
        self._check(self._lib.lb_mlp_forward_trace(self._h, _ptr(X), X.shape[0], _ptr(Y),
                                                   _ptr(H)))
        return Y, H

    def gradients(self, X, T, trace: bool = False):
        """(gradient, loss); with trace also the trace rows [M][320]
        (lb_mlp_gradients_trace)."""
        import torch
        X, T = X.contiguous(), T.contiguous()
        g = torch.empty(MLP_PARAMS, device=X.device, dtype=torch.float32)
        loss = ctypes.c_double()
        if not trace:
            self._check(self._lib.lb_mlp_gradients(self._h, _ptr(X), _ptr(T), X.shape[0],
                                                   _ptr(g), ctypes.byref(loss)))
            return g, loss.value
        tr = torch.empty((X.shape[0], 320), device=X.device, dtype=torch.float32)
        self._check(self._lib.lb_mlp_gradients_trace(self._h, _ptr(X), _ptr(T), X.shape[0],
                                                     _ptr(g), ctypes.byref(loss), _ptr(tr)))
        return g, loss.value, tr

    def train_step(self, X, T, lr: float, want_loss: bool = True):
        X, T = X.contiguous(), T.contiguous()
        loss = ctypes.c_double()
        self._check(self._lib.lb_mlp_train_step(self._h, _ptr(X), _ptr(T), X.shape[0],
                                                float(lr), ctypes.byref(loss) if want_loss
                                                else None))
        return loss.value if want_loss else None


def wait_selftest(iterations: int = 1000) -> int:
    """Status code of lb_wait_selftest (LB_ETIMEOUT when the bounded wait
    expired and was recorded, as it must)."""
    return int(load().lb_wait_selftest(int(iterations)))
