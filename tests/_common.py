"""Shared helpers of the test suite (no arithmetic of the method)."""
import numpy as np

import oracle as O


def weights(lattice):
    return O.lattice_tables(lattice)[1]


def f64_state(lattice, df32):
    """Absolute FP64 populations f = w + df from float32 shifted values."""
    w = weights(lattice)
    df = np.asarray(df32, dtype=np.float64)
    return df + w.reshape((-1,) + (1,) * (df.ndim - 1))


def shifted(lattice, f):
    w = weights(lattice)
    return f - w.reshape((-1,) + (1,) * (f.ndim - 1))


def max_rel_to_weight(lattice, a, b):
    """max over cells and i of |a_i - b_i| / w_i (populations [Q, ...])."""
    w = weights(lattice).reshape((-1,) + (1,) * (np.ndim(a) - 1))
    return float(np.max(np.abs(np.asarray(a, np.float64) - np.asarray(b, np.float64)) / w))


def rel_l2(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))
