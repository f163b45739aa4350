"""Seeded synthetic inputs shared by the CUDA path, the oracle and the tests.

This module holds no arithmetic of the method: it only draws random numbers
and shapes them into problem descriptions (viscosity blobs, graded vertex
coordinates, right-hand sides, batched problem sizes).  Both the library and
the oracle receive the resulting arrays explicitly.

Generator: SplitMix64 (Steele, Lea, Flood, "Fast splittable pseudorandom
number generators", OOPSLA 2014), uniform = (z >> 11) * 2^-53, normal by
Box-Muller.  Base seed 2103.
"""
from __future__ import annotations

import numpy as np

BASE_SEED = 2103
_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed: int, n: int) -> np.ndarray:
    """The first n outputs of SplitMix64 started from state `seed`."""
    with np.errstate(over="ignore"):
        k = np.arange(1, n + 1, dtype=np.uint64)
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + k * _GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        return z ^ (z >> np.uint64(31))


def uniform(seed: int, n: int) -> np.ndarray:
    """n uniforms in [0, 1) with 53 random bits each."""
    return (splitmix64(seed, n) >> np.uint64(11)).astype(np.float64) * 2.0 ** -53


def normal(seed: int, n: int) -> np.ndarray:
    """n standard normals (Box-Muller on consecutive uniform pairs)."""
    m = (n + 1) // 2
    u = uniform(seed, 2 * m)
    u1, u2 = u[0::2], u[1::2]
    r = np.sqrt(-2.0 * np.log1p(-u1))
    z = np.empty(2 * m)
    z[0::2] = r * np.cos(2.0 * np.pi * u2)
    z[1::2] = r * np.sin(2.0 * np.pi * u2)
    return z[:n]


def viscosity_blobs(seed: int, k: int = 20, s_max: float = 3.0,
                    rho=(0.05, 0.15)) -> np.ndarray:
    """(k, 5) blobs (cx, cy, cz, rho, s): centres U[0,1]^3, rho U[rho0,rho1], s U[0,s_max].

    With eta(x) = eta0 * 10**max_k s_k exp(-|x-c_k|^2/(2 rho_k^2)) the contrast is
    at most 10**s_max (1e3 for the 3-D variable-viscosity case, 1e4 for the
    anisotropic one)."""
    u = uniform(seed, 5 * k).reshape(k, 5)
    out = np.empty((k, 5))
    out[:, 0:3] = u[:, 0:3]
    out[:, 3] = rho[0] + (rho[1] - rho[0]) * u[:, 3]
    out[:, 4] = s_max * u[:, 4]
    return out


def graded_coordinates(N: int, aspect: float, dim: int = 3, axis: int = None) -> np.ndarray:
    """(dim, N+1) vertex coordinates on [0,1]: uniform on every axis but `axis`
    (default the last), which is geometrically graded so that the largest ratio
    of a cell's edge lengths on the finest grid is `aspect`.

    The grading is applied to the coarsest-spacing pattern by a geometric
    sequence in the vertex index, so every coarser grid of the hierarchy
    (every other line dropped) stays a tensor grid of the same family."""
    if axis is None:
        axis = dim - 1
    c = np.tile(np.linspace(0.0, 1.0, N + 1), (dim, 1))
    if aspect > 1.0:
        # spacing h_k = h_0 q^k ; uniform spacing 1/N on the other axes.  The
        # smallest cell has z-extent h_0 and x-extent 1/N: choose h_0 = 1/(N*aspect)
        # and q such that sum h_k = 1.
        h0 = 1.0 / (N * aspect)
        lo, hi = 1.0, 2.0
        for _ in range(200):  # bisection on q: sum_{k<N} h0 q^k = 1
            q = 0.5 * (lo + hi)
            s = h0 * (q ** N - 1.0) / (q - 1.0)
            lo, hi = (q, hi) if s < 1.0 else (lo, q)
        q = 0.5 * (lo + hi)
        h = h0 * q ** np.arange(N)
        z = np.concatenate([[0.0], np.cumsum(h)])
        z /= z[-1]
        c[axis] = z
    return c


def random_vector(seed: int, n: int) -> np.ndarray:
    """iid N(0,1) vector of length n."""
    return normal(seed, n)


def batched_sizes(seed: int, nprob: int = 256, lo: int = 2, hi: int = 16, unit: int = 16) -> np.ndarray:
    """Mesh sizes N = unit * m with m uniform on {lo..hi} (32^2 .. 256^2 cavities)."""
    u = uniform(seed, nprob)
    m = lo + np.floor(u * (hi - lo + 1)).astype(np.int64)
    return unit * np.minimum(m, hi)


def levels_for(N: int, coarsest_min: int = 4) -> int:
    """1 + max{k : N / 2^k integral and >= coarsest_min}."""
    k = 0
    while N % (2 ** (k + 1)) == 0 and N // 2 ** (k + 1) >= coarsest_min:
        k += 1
    return k + 1
