"""Host-side checks of the C ABI that need no GPU: the library builds and loads,
exports every entry point include/lbrr.h declares, and validates arguments
before touching the device."""
import ctypes
import os
import re

import pytest

from paper_1505_06900_gb300 import binding as B
from paper_1505_06900_gb300 import build as build_mod

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "lbrr.h")


@pytest.fixture(scope="module")
def lib():
    build_mod.build()
    return B.load()


def declared_entry_points():
    text = open(HEADER).read()
    return sorted(set(re.findall(r"^LB_API[^;(]*?\b(lb_\w+)\(", text, flags=re.M)))


def test_header_declares_the_boundary():
    names = declared_entry_points()
    for core in ["lb_create", "lb_init_fields", "lb_step", "lb_moments", "lb_diagnostics",
                 "lb_destroy", "lb_last_error"]:
        assert core in names
    assert set(names) == set(B.SIGNATURES), "binding and header disagree"


def test_library_exports_every_declared_symbol(lib):
    for name in declared_entry_points():
        assert hasattr(lib, name), name


@pytest.mark.parametrize("args,fragment", [
    ((8, 16, 16, 1, 0.7, 1), "unknown lattice"),
    ((9, 0, 16, 1, 0.7, 1), "grid sizes"),
    ((9, 16, 16, 2, 0.7, 1), "D2Q9 needs nz"),
    ((27, 16, 16, 16, 0.5, 1), "tau"),
    ((27, 16, 16, 16, float("nan"), 1), "tau"),
    ((27, 16, 16, 16, 0.7, 0), "periodic"),
    ((27, 16, 70000, 16, 0.7, 1), "65535"),
])
def test_create_rejects_bad_arguments(lib, args, fragment):
    h = ctypes.c_void_p()
    rc = lib.lb_create(ctypes.byref(h), *args)
    assert rc == B.LB_EINVAL
    assert not h.value
    assert fragment in lib.lb_last_error(None).decode()


def test_create_ex_rejects_bad_options(lib):
    h = ctypes.c_void_p()
    o = B.LBOptions(27, 8, 8, 8, 0.7, 1, 7, 0)
    assert lib.lb_create_ex(ctypes.byref(h), ctypes.addressof(o)) == B.LB_EINVAL
    assert "storage" in lib.lb_last_error(None).decode()
    o = B.LBOptions(27, 8, 8, 8, 0.7, 1, 0, 5)
    assert lib.lb_create_ex(ctypes.byref(h), ctypes.addressof(o)) == B.LB_EINVAL
    assert lib.lb_create_ex(None, ctypes.addressof(o)) == B.LB_EINVAL


@pytest.mark.parametrize("opts,fragment", [
    ((9, 8, 8, 1, 0.7, 1, 0, 0, 4), "walls"),        # z walls on a 2D lattice
    ((27, 8, 8, 8, 0.7, 1, 0, 0, 8), "walls"),       # no fourth axis
    ((27, 8, 8, 8, 0.7, 1, 0, 0, -1), "walls"),
    ((9, 8, 2, 1, 0.7, 1, 0, 0, 2), "at least 3"),  # walled axis too short
])
def test_create_ex_rejects_bad_walls(lib, opts, fragment):
    h = ctypes.c_void_p()
    o = B.LBOptions(*opts)
    assert lib.lb_create_ex(ctypes.byref(h), ctypes.addressof(o)) == B.LB_EINVAL
    assert not h.value
    assert fragment in lib.lb_last_error(None).decode()


def test_status_codes_match_the_header():
    text = open(HEADER).read()
    codes = dict(re.findall(r"^#define (LB_E\w+|LB_OK) (\d+)", text, flags=re.M))
    for name in ["LB_OK", "LB_EINVAL", "LB_ENOMEM", "LB_ECUDA", "LB_EDIVERGED", "LB_ETIMEOUT"]:
        assert int(codes[name]) == getattr(B, name), name


def test_null_context_is_rejected(lib):
    assert lib.lb_step(None, 1) == B.LB_EINVAL
    assert lib.lb_moments(None, None, None, None) == B.LB_EINVAL
    assert lib.lb_state_bytes(None) == -1
    lib.lb_destroy(None)


def test_closure_entry_points_reject_null_handles(lib):
    """The learned-closure and inspection entry points validate their handles
    and buffers before any device work."""
    assert lib.lb_coarsen_neq(None, None, 2.0) == B.LB_EINVAL
    assert lib.lb_closure_step_targets(None, None, None, None) == B.LB_EINVAL
    assert lib.lb_set_closure_ex(None, None, 8.0, 0.25) == B.LB_EINVAL
    assert lib.lb_mlp_forward_trace(None, None, 1, None, None) == B.LB_EINVAL
    assert lib.lb_mlp_gradients_trace(None, None, None, 1, None, None, None) == B.LB_EINVAL


def test_product_path_does_not_use_the_oracle():
    """The CUDA package never imports, links or runs anything under oracle/."""
    pkg = os.path.join(ROOT, "paper_1505_06900_gb300")
    for dirpath, _, files in os.walk(pkg):
        for fn in files:
            if fn.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
                text = open(os.path.join(dirpath, fn)).read()
                assert not re.search(r"^\s*(import|from)\s+oracle\b|lbrr_oracle|\bora_\w+\(", text,
                                     flags=re.M), fn
