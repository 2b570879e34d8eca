"""FP64 CPU oracle of the recursive-regularized BGK lattice Boltzmann step.

TEST INFRASTRUCTURE. This package is imported only by the test suite, by
``__graft_entry__.smoke()`` and by the CPU-baseline leg of ``bench.py``. The
product path (``paper_1505_06900_gb300``) never imports it and shares no code
with it. The arithmetic lives in ``lbrr_oracle.c`` (plain C, double
precision), which follows the paper's equations one by one; this module only
compiles it with gcc and marshals numpy arrays through ctypes.

Functions with a pin are listed in the oracle tests; every function here has at
least one pin that does not go through the oracle's own formulas.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lbrr_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liblbrr_oracle.so")

D2Q9 = 9
D3Q27 = 27
D3Q19 = 19    # D3Q27 without the corners; order-3 basis of sums / differences
RR = 0        # recursive-regularized model (Sec. 3.5)
REG2 = 1      # order-2 regularized comparator (Sec. 3.8.1)
BGK = 2       # plain BGK with the full-basis equilibrium (Sec. 3.4)
INIT_EQ = 0
INIT_EQ_NEQ_FD = 1

_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle shared library with gcc (idempotent)."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp",
           "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            dp = ctypes.POINTER(ctypes.c_double)
            ip = ctypes.POINTER(ctypes.c_int)
            i, d = ctypes.c_int, ctypes.c_double
            sig = {
                "ora_lattice_tables": [i, ip, ip, ip, dp],
                "ora_hermite_basis": [i, dp, dp],
                "ora_feq_cell": [i, i, d, dp, dp],
                "ora_a1_coefficients": [i, dp, dp, dp],
                "ora_fneq_cell": [i, i, dp, dp, dp],
                "ora_moments_cell": [i, i, dp, dp, dp, dp],
                "ora_collide_cell": [i, i, d, dp, dp],
                "ora_step": [i, i, i, i, i, d, dp, i],
                "ora_init": [i, i, i, i, i, d, i, dp, dp, dp],
                "ora_fields": [i, i, i, i, i, dp, dp, dp, dp],
                "ora_diagnostics": [i, i, i, i, dp, dp],
                "ora_enstrophy": [i, i, i, i, dp, dp],
                "ora_collide_cell_closure": [d, dp, dp, dp],
                "ora_step_walls": [i, i, i, i, i, d, i, dp, i],
                "ora_init_walls": [i, i, i, i, i, d, i, i, dp, dp, dp],
                "ora_fields_walls": [i, i, i, i, i, i, dp, dp, dp, dp],
                "ora_enstrophy_walls": [i, i, i, i, i, dp, dp],
                "ora_num_threads": [],
                "ora_set_num_threads": [i],
            }
            for name, args in sig.items():
                fn = getattr(lib, name)
                fn.argtypes = args
                fn.restype = None if name == "ora_set_num_threads" else ctypes.c_int
            _lib = lib
    return _lib


def _dp(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def _check(rc: int, what: str):
    if rc != 0:
        raise ValueError(f"oracle {what} failed with code {rc}")


def dims_of(lattice: int) -> tuple[int, int]:
    """(D, Q) of a lattice."""
    if lattice == D2Q9:
        return 2, 9
    if lattice == D3Q27:
        return 3, 27
    if lattice == D3Q19:
        return 3, 19
    raise ValueError(f"unknown lattice {lattice}")


def lattice_tables(lattice: int):
    """Velocities c [Q,3] (int) and weights w [Q] of the oracle's lattice."""
    lib = _load()
    D, Q = dims_of(lattice)
    d, q = ctypes.c_int(), ctypes.c_int()
    c = np.zeros(Q * 3, dtype=np.int32)
    w = np.zeros(Q, dtype=np.float64)
    _check(lib.ora_lattice_tables(lattice, ctypes.byref(d), ctypes.byref(q),
                                  c.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), _dp(w)),
           "lattice_tables")
    return c.reshape(Q, 3), w


def hermite_basis(lattice: int):
    """Kept basis polynomials H [K,Q] (row k, column i) and prefactors [K]:
    K = Q for D2Q9 / D3Q27; K = 16 for D3Q19 (orders 0..2 and the six
    order-3 sums / differences H_aab +- H_bcc)."""
    lib = _load()
    _, Q = dims_of(lattice)
    H = np.zeros(Q * Q)
    p = np.zeros(Q)
    _check(lib.ora_hermite_basis(lattice, _dp(H), _dp(p)), "hermite_basis")
    K = 16 if lattice == D3Q19 else Q
    return H.reshape(Q, Q)[:K], p[:K]


def feq_cell(lattice: int, rho: float, u, variant: int = RR) -> np.ndarray:
    lib = _load()
    _, Q = dims_of(lattice)
    uu = _f64(list(u) + [0.0] * (3 - len(u)))
    out = np.zeros(Q)
    _check(lib.ora_feq_cell(lattice, variant, float(rho), _dp(uu), _dp(out)), "feq_cell")
    return out


def a1_coefficients(lattice: int, u, pi1) -> np.ndarray:
    lib = _load()
    D, _ = dims_of(lattice)
    uu = _f64(list(u) + [0.0] * (3 - len(u)))
    p = _f64(pi1)
    out = np.zeros(6 if D == 2 else 23)
    _check(lib.ora_a1_coefficients(lattice, _dp(uu), _dp(p), _dp(out)), "a1_coefficients")
    return out


def fneq_cell(lattice: int, u, pi1, variant: int = RR) -> np.ndarray:
    lib = _load()
    _, Q = dims_of(lattice)
    uu = _f64(list(u) + [0.0] * (3 - len(u)))
    p = _f64(pi1)
    out = np.zeros(Q)
    _check(lib.ora_fneq_cell(lattice, variant, _dp(uu), _dp(p), _dp(out)), "fneq_cell")
    return out


def moments_cell(lattice: int, f, variant: int = RR):
    """(rho, u[D], pi1[3 or 6]) of one cell."""
    lib = _load()
    D, _ = dims_of(lattice)
    ff = _f64(f)
    rho = ctypes.c_double()
    u = np.zeros(D)
    p = np.zeros(3 if D == 2 else 6)
    _check(lib.ora_moments_cell(lattice, variant, _dp(ff), ctypes.byref(rho), _dp(u), _dp(p)),
           "moments_cell")
    return rho.value, u, p


def collide_cell(lattice: int, f, tau: float, variant: int = RR) -> np.ndarray:
    lib = _load()
    _, Q = dims_of(lattice)
    ff = _f64(f)
    out = np.zeros(Q)
    _check(lib.ora_collide_cell(lattice, variant, float(tau), _dp(ff), _dp(out)), "collide_cell")
    return out


def collide_cell_closure(f, tau: float, delta) -> np.ndarray:
    """D3Q27 collision with delta[17] added to the order 3..6 off-equilibrium
    coefficients (the learned closure's correction)."""
    lib = _load()
    ff = _f64(f)
    dd = _f64(delta)
    assert ff.size == 27 and dd.size == 17
    out = np.zeros(27)
    _check(lib.ora_collide_cell_closure(float(tau), _dp(ff), _dp(dd), _dp(out)),
           "collide_cell_closure")
    return out


def init(lattice: int, shape, tau: float, rho, u, mode: int = INIT_EQ_NEQ_FD,
         variant: int = RR, walls: int = 0) -> np.ndarray:
    """Initial populations f [Q, nz, ny, nx] from rho [nz,ny,nx], u [D,nz,ny,nx].
    walls: bit a = no-slip walls through the end node planes of axis a (the
    boundary nodes start at rest)."""
    lib = _load()
    D, Q = dims_of(lattice)
    nx, ny, nz = shape
    r = _f64(rho).reshape(-1)
    uu = _f64(u).reshape(-1)
    assert r.size == nx * ny * nz and uu.size == D * r.size
    f = np.zeros(Q * r.size)
    if walls:
        _check(lib.ora_init_walls(lattice, variant, nx, ny, nz, float(tau), mode, int(walls),
                                  _dp(r), _dp(uu), _dp(f)), "init_walls")
    else:
        _check(lib.ora_init(lattice, variant, nx, ny, nz, float(tau), mode, _dp(r), _dp(uu),
                            _dp(f)), "init")
    return f.reshape(Q, nz, ny, nx)


def step(lattice: int, shape, tau: float, f: np.ndarray, nsteps: int = 1,
         variant: int = RR, walls: int = 0) -> np.ndarray:
    """Return the populations after nsteps updates (the input is not modified).
    With walls, populations that stream in from outside the domain are NaN
    in the result (the boundary rule rebuilds them)."""
    lib = _load()
    nx, ny, nz = shape
    out = np.array(f, dtype=np.float64, order="C", copy=True)
    if walls:
        _check(lib.ora_step_walls(lattice, variant, nx, ny, nz, float(tau), int(walls), _dp(out),
                                  int(nsteps)), "step_walls")
    else:
        _check(lib.ora_step(lattice, variant, nx, ny, nz, float(tau), _dp(out), int(nsteps)),
               "step")
    return out


def fields(lattice: int, shape, f: np.ndarray, variant: int = RR, walls: int = 0):
    """(rho [nz,ny,nx], u [D,...], pi1 [3|6,...]) of a population field; with
    walls, boundary nodes report their regularized state (u = 0)."""
    lib = _load()
    D, _ = dims_of(lattice)
    nx, ny, nz = shape
    n = nx * ny * nz
    ff = _f64(f)
    rho = np.zeros(n)
    u = np.zeros(D * n)
    p = np.zeros((3 if D == 2 else 6) * n)
    if walls:
        _check(lib.ora_fields_walls(lattice, variant, nx, ny, nz, int(walls), _dp(ff), _dp(rho),
                                    _dp(u), _dp(p)), "fields_walls")
    else:
        _check(lib.ora_fields(lattice, variant, nx, ny, nz, _dp(ff), _dp(rho), _dp(u), _dp(p)),
               "fields")
    return rho.reshape(nz, ny, nx), u.reshape(D, nz, ny, nx), p.reshape(-1, nz, ny, nx)


def diagnostics(lattice: int, shape, f: np.ndarray, walls: int = 0) -> np.ndarray:
    """[mass, momentum_0..D-1, kinetic energy]; with walls, of the fields of
    fields(..., walls) (plain sums over the nodes)."""
    lib = _load()
    D, _ = dims_of(lattice)
    nx, ny, nz = shape
    if walls:
        rho, u, _ = fields(lattice, shape, f, walls=walls)
        mom = [float(np.sum(rho * u[a])) for a in range(D)]
        return np.array([float(np.sum(rho))] + mom + [float(0.5 * np.sum(rho * np.sum(u * u, 0)))])
    out = np.zeros(2 + D)
    _check(lib.ora_diagnostics(lattice, nx, ny, nz, _dp(_f64(f)), _dp(out)), "diagnostics")
    return out


def enstrophy(lattice: int, shape, f: np.ndarray, walls: int = 0) -> float:
    """0.5 sum |curl u|^2 over the cells (periodic central differences); with
    walls, the trapezoidal rule over the nodes with one-sided differences on
    the wall planes."""
    lib = _load()
    nx, ny, nz = shape
    out = np.zeros(1)
    if walls:
        _check(lib.ora_enstrophy_walls(lattice, nx, ny, nz, int(walls), _dp(_f64(f)), _dp(out)),
               "enstrophy_walls")
    else:
        _check(lib.ora_enstrophy(lattice, nx, ny, nz, _dp(_f64(f)), _dp(out)), "enstrophy")
    return float(out[0])


def num_threads() -> int:
    return int(_load().ora_num_threads())


def set_num_threads(n: int) -> None:
    _load().ora_set_num_threads(int(n))
