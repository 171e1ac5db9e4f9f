"""Test helpers: velocity-order mapping between the oracle and the library,
and comparison utilities. Holds no arithmetic of the method."""
import numpy as np


def perm(c_from, c_to):
    """index p with c_to[p[a]] == c_from[a] for every a."""
    lut = {tuple(int(v) for v in c): b for b, c in enumerate(c_to)}
    return np.array([lut[tuple(int(v) for v in c)] for c in c_from])


def oracle_state_in_lib_order(N_oracle, c_oracle, c_lib):
    """Reorder an oracle population array [q][ncell] into library order."""
    p = perm(c_lib, c_oracle)       # library direction a is oracle direction p[a]
    return N_oracle[p]


def rel_err(a, b, scale=None):
    a = np.asarray(a)
    b = np.asarray(b)
    s = np.abs(b).max() if scale is None else scale
    return float(np.abs(a - b).max() / max(s, 1e-300))
