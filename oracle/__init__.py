"""Serial FP64 oracle for the restricted additive Vanka multigrid method.

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` may import this package; the product library never
does.  The arithmetic lives in ``rav_oracle.cpp`` (plain serial C++, compiled
with ``-O2 -ffp-contract=off`` so that x86 and Arm hosts round identically);
this module only marshals numpy arrays through ctypes.

Paper map (Saberi, Meschke, Vogel, "A restricted additive Vanka smoother for
geometric multigrid"):
  * system and discretisation ............ Sec. 2, Eqs. 5-7 (C = 0 for Q2-Q1)
  * smoother update ....................... Eq. 10
  * subdomains, R_i, L_i .................. Sec. 3, Eq. 11
  * MV / AV / RAV ......................... Eqs. 11 / 12 / 13, Eq. 15
  * stored owned rows ..................... Sec. 4.3
  * V-cycle, LU coarse solve, stopping .... Sec. 2 (Fig. 1), Sec. 4
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "rav_oracle.cpp")
_LIB = os.path.join(_HERE, "librav_oracle.so")

RAV, AV, MV, MV_COLOURED = 0, 1, 2, 3
F64, F32, BF16, FP8 = 0, 1, 2, 3
F32_FACT, BF16_FACT = 5, 6  # factored storage rounded to fp32 / bf16
BC_CAVITY, BC_NOSLIP, BC_QUADRATIC = 0, 1, 2
ELEM_Q2Q1, ELEM_Q1Q1 = 0, 1  # Taylor-Hood; stabilised equal order (Eq. 8)
F_NONE, F_PSI, F_SINKER, F_QUADRATIC = 0, 1, 2, 3


def build(force: bool = False) -> str:
    """Compile the oracle shared library next to its source (with OpenMP for
    the independent subdomain loops when the compiler has it, else serial)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        base = ["g++", "-O2", "-ffp-contract=off", "-std=c++17", "-shared", "-fPIC", _SRC, "-o", tmp]
        if subprocess.call(base[:1] + ["-fopenmp"] + base[1:], stderr=subprocess.DEVNULL) != 0:
            subprocess.check_call(base)
        os.replace(tmp, _LIB)
    return _LIB


_lib = None


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        P = ctypes.c_void_p
        i, d, ll = ctypes.c_int, ctypes.c_double, ctypes.c_longlong
        sig = {
            "orc_create": (P, [i, i, i, P, d, i, P, i]),
            "orc_create_elem": (P, [i, i, i, P, d, i, P, i, i, d]),
            "orc_destroy": (None, [P]),
            "orc_error": (i, [P]),
            "orc_count": (ll, [P, i, i]),
            "orc_get_csr": (None, [P, i, P, P, P]),
            "orc_get_prolongation": (None, [P, i, P, P, P]),
            "orc_get_dirichlet": (None, [P, i, P, P]),
            "orc_rhs": (None, [P, i, P]),
            "orc_viscosity": (d, [P, P]),
            "orc_setup_smoother": (i, [P, i, d, i]),
            "orc_build_patches": (None, [P, i]),
            "orc_set_patches": (i, [P, i, ll, P, P, P, d]),
            "orc_set_omega": (None, [P, i, P]),
            "orc_get_patches": (None, [P, i, P, P, P]),
            "orc_get_inverse": (ll, [P, i, ll, i, P, P]),
            "orc_patch_rows": (i, [P, i, ll, P]),
            "orc_residual": (None, [P, i, P, P, P]),
            "orc_smooth": (None, [P, i, P, P, i]),
            "orc_restrict": (None, [P, i, P, P]),
            "orc_prolong_add": (None, [P, i, P, P]),
            "orc_coarse_solve": (None, [P, P, P]),
            "orc_vcycle": (None, [P, P, P, i, i]),
            "orc_solve": (i, [P, P, P, d, i, i, i, P]),
            "orc_fgmres": (i, [P, P, P, d, i, i, i, i, P]),
            "orc_round_format": (None, [i, P, P, ll]),
            "orc_labels": (None, [P, i, P, P, d, P]),
            "orc_mlp_nparam": (ll, []),
            "orc_mlp_forward": (None, [P, P, ll, P]),
            "orc_mlp_loss_grad": (d, [P, P, P, ll, P]),
            "orc_set_threads": (i, [i]),
            "orc_patch_features": (None, [P, i, P]),
        }
        for name, (res, args) in sig.items():
            f = getattr(lib, name)
            f.restype = res
            f.argtypes = args
        _lib = lib
    return _lib


def set_threads(n: int) -> int:
    """Threads of the oracle's loops over independent subdomains (local
    inverses, RAV corrections); the results do not depend on it.  Returns the
    number in effect (1 without OpenMP)."""
    return _load().orc_set_threads(int(n))


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def round_format(prec: int, v) -> np.ndarray:
    """Round-to-nearest-even into fp32 (1), bf16 (2) or saturating fp8 e4m3 (3), returned as fp64."""
    v = _f64(v)
    out = np.empty_like(v)
    _load().orc_round_format(prec, _ptr(v), _ptr(out), v.size)
    return out


def mlp_nparam() -> int:
    return _load().orc_mlp_nparam()


def mlp_forward(params, X) -> np.ndarray:
    """omega = 1.5 sigmoid(MLP(x)) for the rows of X (n, 8), fp64."""
    P, X = _f64(params), _f64(X).reshape(-1, 8)
    out = np.empty(X.shape[0])
    _load().orc_mlp_forward(_ptr(P), _ptr(X), X.shape[0], _ptr(out))
    return out


def mlp_loss_grad(params, X, y):
    """(mean squared error, gradient with respect to the 4801 parameters), fp64."""
    P, X, y = _f64(params), _f64(X).reshape(-1, 8), _f64(y)
    g = np.empty(mlp_nparam())
    loss = _load().orc_mlp_loss_grad(_ptr(P), _ptr(X), _ptr(y), X.shape[0], _ptr(g))
    return loss, g


class Oracle:
    """A multigrid hierarchy on the unit square/cube, level 0 = coarsest.

    coords: optional (dim, N+1) fine-level vertex coordinates per axis.
    blobs:  optional (k, 5) array of (cx, cy, cz, rho, s) viscosity blobs,
            eta(x) = eta0 * 10**max_k s_k exp(-|x-c_k|^2 / (2 rho_k^2)).
    bc:     BC_CAVITY (lid u = e_0 on the top face), BC_NOSLIP, BC_QUADRATIC.
    element: ELEM_Q2Q1 (Taylor-Hood, C = 0) or ELEM_Q1Q1 (equal order with the
            pressure stabilisation C = -beta sum_e h_e^2 (grad q, grad p)_e, Eq. 8).
    """

    def __init__(self, dim, N, nlev, coords=None, eta0=1.0, blobs=None, bc=BC_CAVITY,
                 element=0, beta=0.0):
        lib = _load()
        self.dim, self.N, self.nlev = dim, N, nlev
        self.element = element
        c = None if coords is None else _f64(coords).reshape(dim, N + 1)
        bl = np.zeros((0, 5)) if blobs is None else _f64(blobs).reshape(-1, 5)
        self._keep = (c, bl)
        self.h = lib.orc_create_elem(dim, N, nlev, _ptr(c), float(eta0), bl.shape[0], _ptr(bl), bc,
                                     int(element), float(beta))

    def check_coarse(self):
        """Factorises the bordered coarse system; raises if it is singular."""
        if _lib.orc_error(self.h) != 0:
            raise RuntimeError("oracle: singular coarse system")

    def __del__(self):
        if getattr(self, "h", None) and _lib is not None:
            _lib.orc_destroy(self.h)
            self.h = None

    # ---- counts and exports -------------------------------------------------
    def count(self, lev, what):
        return _lib.orc_count(self.h, lev, what)

    def sizes(self, lev):
        return dict(n_u=self.count(lev, 0), n_p=self.count(lev, 1), n=self.count(lev, 2),
                    nnz=self.count(lev, 3), N=self.count(lev, 4))

    def csr(self, lev):
        n, nnz = self.count(lev, 2), self.count(lev, 3)
        rp, ci, va = np.empty(n + 1, np.int64), np.empty(nnz, np.int64), np.empty(nnz)
        _lib.orc_get_csr(self.h, lev, _ptr(rp), _ptr(ci), _ptr(va))
        return rp, ci, va

    def matrix(self, lev):
        import scipy.sparse as sp
        rp, ci, va = self.csr(lev)
        n = self.count(lev, 2)
        return sp.csr_matrix((va, ci, rp), shape=(n, n))

    def prolongation(self, lev):
        """Sparse P mapping level lev-1 into level lev (fine Dirichlet rows empty)."""
        import scipy.sparse as sp
        n, nc, nnz = self.count(lev, 2), self.count(lev - 1, 2), self.count(lev, 7)
        rp, ci, va = np.empty(n + 1, np.int64), np.empty(nnz, np.int64), np.empty(nnz)
        _lib.orc_get_prolongation(self.h, lev, _ptr(rp), _ptr(ci), _ptr(va))
        return sp.csr_matrix((va, ci, rp), shape=(n, nc))

    def dirichlet(self, lev):
        n = self.count(lev, 2)
        m, g = np.empty(n, np.uint8), np.empty(n)
        _lib.orc_get_dirichlet(self.h, lev, _ptr(m), _ptr(g))
        return m.astype(bool), g

    def rhs(self, forcing):
        b = np.empty(self.count(self.nlev - 1, 2))
        _lib.orc_rhs(self.h, forcing, _ptr(b))
        return b

    def initial_guess(self):
        """x0: Dirichlet values g on boundary DoFs, 0 elsewhere."""
        return self.dirichlet(self.nlev - 1)[1].copy()

    def viscosity(self, x):
        x = _f64(x)
        return _lib.orc_viscosity(self.h, _ptr(x))

    # ---- smoother -----------------------------------------------------------
    def setup_smoother(self, kind=RAV, omega=0.5, prec=F64):
        rc = _lib.orc_setup_smoother(self.h, kind, float(omega), prec)
        if rc != 0:
            raise RuntimeError(f"oracle: singular subdomain system ({rc})")
        self.kind = kind

    def build_patches(self, lev):
        _lib.orc_build_patches(self.h, lev)

    def patches(self, lev):
        """(offsets, dofs, owner) of the subdomains of level lev."""
        np_, tot, n = self.count(lev, 5), self.count(lev, 6), self.count(lev, 2)
        off, dofs, own = np.empty(np_ + 1, np.int64), np.empty(tot, np.int64), np.empty(n, np.int64)
        _lib.orc_get_patches(self.h, lev, _ptr(off), _ptr(dofs), _ptr(own))
        return off, dofs, own

    def set_patches(self, lev, off, dofs, owner, omega):
        off, dofs, owner = (np.ascontiguousarray(a, np.int64) for a in (off, dofs, owner))
        rc = _lib.orc_set_patches(self.h, lev, len(off) - 1, _ptr(off), _ptr(dofs), _ptr(owner), float(omega))
        if rc != 0:
            raise RuntimeError("oracle: singular subdomain system")

    def set_omega(self, lev, w):
        w = _f64(w)
        _lib.orc_set_omega(self.h, lev, _ptr(w))

    def inverse(self, lev, p, quantised=False):
        """Owned rows (RAV) or full inverse (AV/MV) of subdomain p, as (rows, n_i) array."""
        off = self.patches(lev)[0]
        ni = int(off[p + 1] - off[p])
        size = _lib.orc_get_inverse(self.h, lev, p, int(quantised), None, None)
        out = np.empty(size)
        sc = np.empty(size // max(ni, 1))
        _lib.orc_get_inverse(self.h, lev, p, int(quantised), _ptr(out), _ptr(sc))
        out = out.reshape(-1, ni)
        return (out, sc) if quantised else out

    def patch_features(self, lev):
        """The 8 learned-damping features of every subdomain of level lev, (n_p, 8)."""
        out = np.zeros((self.count(lev, 1), 8))
        _lib.orc_patch_features(self.h, lev, _ptr(out))
        return out

    def labels(self, lev, r, omega=None, fallback=0.5):
        """Coordinate line-search damping per subdomain for residual r given the
        current weights omega (default: `fallback` everywhere); needs patches on lev."""
        r = _f64(r)
        out = np.empty(self.count(lev, 5))
        om = None if omega is None else _f64(omega)
        _lib.orc_labels(self.h, lev, _ptr(r), _ptr(om), float(fallback), _ptr(out))
        return out

    def patch_rows(self, lev, p, max_rows=64, max_n=512):
        """Owned rows of L_p^{-1} computed on demand (needs build_patches(lev))."""
        out = np.empty(max_rows * max_n)
        k = _lib.orc_patch_rows(self.h, lev, p, _ptr(out))
        if k < 0:
            raise RuntimeError("oracle: singular subdomain system")
        return out

    # ---- operators ----------------------------------------------------------
    def residual(self, lev, x, b):
        x, b = _f64(x), _f64(b)
        r = np.empty_like(x)
        _lib.orc_residual(self.h, lev, _ptr(x), _ptr(b), _ptr(r))
        return r

    def smooth(self, lev, x, b, steps=1):
        x, b = _f64(x).copy(), _f64(b)
        _lib.orc_smooth(self.h, lev, _ptr(x), _ptr(b), steps)
        return x

    def restrict(self, lev, rf):
        rf = _f64(rf)
        bc = np.empty(self.count(lev - 1, 2))
        _lib.orc_restrict(self.h, lev, _ptr(rf), _ptr(bc))
        return bc

    def prolong_add(self, lev, xc, xf):
        xc, xf = _f64(xc), _f64(xf).copy()
        _lib.orc_prolong_add(self.h, lev, _ptr(xc), _ptr(xf))
        return xf

    def coarse_solve(self, b):
        b = _f64(b)
        x = np.empty_like(b)
        _lib.orc_coarse_solve(self.h, _ptr(b), _ptr(x))
        return x

    def vcycle(self, x, b, nu1=2, nu2=2):
        x, b = _f64(x).copy(), _f64(b)
        _lib.orc_vcycle(self.h, _ptr(x), _ptr(b), nu1, nu2)
        return x

    def solve(self, x, b, tol=1e-8, maxit=100, nu1=2, nu2=2):
        """Stationary V-cycle iteration; returns (x, iterations, history)."""
        x, b = _f64(x).copy(), _f64(b)
        hist = np.zeros(maxit + 1)
        it = _lib.orc_solve(self.h, _ptr(x), _ptr(b), tol, maxit, nu1, nu2, _ptr(hist))
        k = it if it >= 0 else maxit
        return x, it, hist[: k + 1]

    def fgmres(self, x, b, tol=1e-8, maxit=200, restart=30, nu1=2, nu2=2):
        x, b = _f64(x).copy(), _f64(b)
        hist = np.zeros(maxit + 1)
        it = _lib.orc_fgmres(self.h, _ptr(x), _ptr(b), tol, maxit, restart, nu1, nu2, _ptr(hist))
        k = it if it >= 0 else maxit
        return x, it, hist[: k + 1]
