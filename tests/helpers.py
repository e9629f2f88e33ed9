"""Test helpers: map between the oracle's and the library's dof numberings (both expose a
per-patch local-to-global map over the same tile order)."""
import numpy as np


def permutation(space, lib_l2g):
    """perm[i_oracle] = i_library for every active dof."""
    l2g_o = np.concatenate([space.l2g[k].ravel() for k in range(len(space.l2g))])
    assert l2g_o.shape == lib_l2g.shape
    assert np.array_equal(l2g_o < 0, lib_l2g < 0)
    perm = np.full(space.N, -1, dtype=np.int64)
    perm[l2g_o[l2g_o >= 0]] = lib_l2g[l2g_o >= 0]
    assert np.array_equal(np.sort(perm), np.arange(space.N))
    return perm


def to_lib(perm, v):
    out = np.empty_like(v)
    out[perm] = v
    return out


def from_lib(perm, v):
    return v[perm]


def rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))
