"""Small numpy helpers for pinning the oracle: geometry of the numbering and
dense textbook forms of the operators (built with numpy.linalg, never with
oracle code)."""
from __future__ import annotations

import numpy as np


def node_coords(dim, N, coords=None):
    """(n_nodes, dim) coordinates of the Q2 nodes in the numbering
    id = I_0 + (2N+1)(I_1 + (2N+1) I_2); mid-nodes sit at cell midpoints."""
    M = 2 * N + 1
    axes = []
    for a in range(dim):
        v = np.linspace(0, 1, N + 1) if coords is None else np.asarray(coords[a], float)
        q = np.empty(M)
        q[0::2] = v
        q[1::2] = 0.5 * (v[:-1] + v[1:])
        axes.append(q)
    grids = np.meshgrid(*axes[::-1], indexing="ij")  # slowest axis first
    return np.stack([g.reshape(-1) for g in grids[::-1]], axis=-1)


def vertex_coords(dim, N, coords=None):
    axes = [np.linspace(0, 1, N + 1) if coords is None else np.asarray(coords[a], float) for a in range(dim)]
    grids = np.meshgrid(*axes[::-1], indexing="ij")
    return np.stack([g.reshape(-1) for g in grids[::-1]], axis=-1)


def vertex_index(dim, N):
    """(n_p, dim) integer index tuples of the pressure vertices."""
    r = np.arange(N + 1)
    grids = np.meshgrid(*([r] * dim), indexing="ij")
    return np.stack([g.reshape(-1) for g in grids[::-1]], axis=-1)


def interpolate(dim, N, ufun, pfun, coords=None):
    """Nodal vector (velocity interleaved per node, then pressure) of given fields."""
    X = node_coords(dim, N, coords)
    V = vertex_coords(dim, N, coords)
    u = np.stack([ufun(X, c) for c in range(dim)], axis=-1).reshape(-1)
    p = pfun(V) if pfun is not None else np.zeros(len(V))
    return np.concatenate([u, p])


def dense(o, lev):
    return o.matrix(lev).toarray()


def rav_matrix(L, off, dofs, owner, omega, restricted=True):
    """S = sum_i Rt_i^T omega_i L_i^{-1} R_i (Eq. 13; Eq. 12 when restricted=False)."""
    n = L.shape[0]
    S = np.zeros((n, n))
    om = np.broadcast_to(np.asarray(omega, float), (len(off) - 1,))
    for p in range(len(off) - 1):
        s = dofs[off[p]:off[p + 1]]
        Li = np.linalg.inv(L[np.ix_(s, s)])
        if restricted:
            keep = owner[s] == p
            S[np.ix_(s[keep], s)] += om[p] * Li[keep]
        else:
            S[np.ix_(s, s)] += om[p] * Li
    return S


def free_residual(L, x, b, dirmask):
    r = b - L @ x
    r[dirmask] = 0.0
    return r
