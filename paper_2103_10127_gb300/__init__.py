"""GB300 restricted additive Vanka (RAV) multigrid for Q2-Q1 and stabilised Q1-Q1 Stokes.

Python binding of the C ABI in include/ravanka.h.  Every numerical step runs
in the CUDA library (libravanka.so); this module only marshals torch device
tensors (memory) and the current torch stream into the C calls.  There is no
CPU path: without a CUDA device or the library, the calls raise.

Method: Saberi, Meschke, Vogel, "A restricted additive Vanka smoother for
geometric multigrid" (Sec. 3, Eq. 13).
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import _capi
from ._capi import RavError, check

RAV, AV, MV_COLOURED = 0, 1, 3
F64, F32, BF16, FP8, F64_ROWS, F32_FACT, BF16_FACT = 0, 1, 2, 3, 4, 5, 6
BC_CAVITY, BC_NOSLIP, BC_QUADRATIC = 0, 1, 2
ELEM_Q2Q1, ELEM_Q1Q1 = 0, 1
F_NONE, F_PSI, F_SINKER, F_QUADRATIC = 0, 1, 2, 3

__all__ = ["Multigrid", "Smoother", "Batch", "RavError", "RAV", "AV", "MV_COLOURED", "F64", "F32", "BF16", "FP8", "F64_ROWS",
           "F32_FACT", "BF16_FACT",
           "BC_CAVITY", "BC_NOSLIP", "BC_QUADRATIC", "ELEM_Q2Q1", "ELEM_Q1Q1", "F_NONE", "F_PSI", "F_SINKER", "F_QUADRATIC"]


def _torch():
    import torch
    return torch


def _stream(stream=None):
    torch = _torch()
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _ptr(t):
    if t is None:
        return None
    if not t.is_cuda or not t.is_contiguous():
        raise ValueError("expected a contiguous CUDA tensor")
    return ctypes.c_void_p(t.data_ptr())


class Multigrid:
    """Grid hierarchy and assembled operators (mg_setup).

    element: ELEM_Q2Q1 (Taylor-Hood) or ELEM_Q1Q1 (equal order with the
    pressure stabilisation of Eq. 8, constant beta)."""

    def __init__(self, dim, N, n_levels, coords=None, eta0=1.0, blobs=None, bc=BC_CAVITY, element=ELEM_Q2Q1,
                 beta=0.0, stream=None):
        lib = _capi.load()
        self._coords = None if coords is None else np.ascontiguousarray(coords, np.float64).reshape(-1)
        self._blobs = np.zeros((0, 5)) if blobs is None else np.ascontiguousarray(blobs, np.float64).reshape(-1, 5)
        prob = _capi.RavProblem(dim, N, None if self._coords is None else self._coords.ctypes.data, float(eta0),
                                self._blobs.shape[0], self._blobs.ctypes.data if self._blobs.size else None, bc,
                                int(element), float(beta))
        h = ctypes.c_void_p()
        check(lib.mg_setup(ctypes.byref(prob), n_levels, _stream(stream), ctypes.byref(h)), "mg_setup")
        self.h = h
        self.dim, self.N, self.nlev = dim, N, n_levels
        self.element = element

    def __del__(self):
        if getattr(self, "h", None) is not None and _capi._lib is not None:
            _capi._lib.mg_destroy(self.h)
            self.h = None

    def counts(self, level):
        out = (ctypes.c_int64 * 5)()
        check(_capi.load().rav_get_counts(self.h, level, out), "rav_get_counts")
        return dict(n_u=out[0], n_p=out[1], n=out[2], nnz=out[3], N=out[4])

    def n(self, level=None):
        return self.counts(self.nlev - 1 if level is None else level)["n"]

    def csr(self, level, stream=None):
        torch = _torch()
        c = self.counts(level)
        rp = torch.empty(c["n"] + 1, dtype=torch.int64, device="cuda")
        ci = torch.empty(c["nnz"], dtype=torch.int32, device="cuda")
        va = torch.empty(c["nnz"], dtype=torch.float64, device="cuda")
        check(_capi.load().rav_get_csr(self.h, level, _ptr(rp), _ptr(ci), _ptr(va), _stream(stream)), "rav_get_csr")
        return rp, ci, va

    def vector(self, level=None):
        return _torch().zeros(self.n(level), dtype=_torch().float64, device="cuda")

    def rhs(self, forcing, out=None, stream=None):
        b = self.vector() if out is None else out
        check(_capi.load().rav_assemble_rhs(self.h, forcing, _ptr(b), _stream(stream)), "rav_assemble_rhs")
        return b

    def initial_guess(self, out=None, stream=None):
        x = self.vector() if out is None else out
        check(_capi.load().rav_initial_guess(self.h, _ptr(x), _stream(stream)), "rav_initial_guess")
        return x

    def residual(self, level, x, b, r=None, norm=False, stream=None):
        r = _torch().empty_like(x) if r is None else r
        nrm = ctypes.c_double(0.0)
        check(_capi.load().rav_residual(self.h, level, _ptr(x), _ptr(b), _ptr(r),
                                        ctypes.byref(nrm) if norm else None, _stream(stream)), "rav_residual")
        return (r, nrm.value) if norm else r

    def restrict(self, level, rf, out=None, stream=None):
        bc = self.vector(level - 1) if out is None else out
        check(_capi.load().rav_restrict(self.h, level, _ptr(rf), _ptr(bc), _stream(stream)), "rav_restrict")
        return bc

    def prolong_add(self, level, xc, xf, stream=None):
        check(_capi.load().rav_prolong_add(self.h, level, _ptr(xc), _ptr(xf), _stream(stream)), "rav_prolong_add")
        return xf

    def coarse_solve(self, b, out=None, stream=None):
        x = self.vector(0) if out is None else out
        check(_capi.load().rav_coarse_solve(self.h, _ptr(b), _ptr(x), _stream(stream)), "rav_coarse_solve")
        return x

    def residual_split(self, level, threads_per_row=None):
        """Threads per row of the residual kernel on `level`; sets it when given."""
        lib = _capi.load()
        if threads_per_row is not None:
            check(lib.rav_set_residual_split(self.h, level, int(threads_per_row)), "rav_set_residual_split")
        k = lib.rav_get_residual_split(self.h, level)
        if k < 0:
            raise RavError(k, "rav_get_residual_split")
        return k

    def coarse_residual_f32(self, enable=None, min_dofs=0, stream=None):
        """FP32 residuals on the levels between the coarsest and the finest with
        at least min_dofs DoFs (rav_set_coarse_residual_f32); sets it when
        given, returns 0/1."""
        lib = _capi.load()
        if enable is not None:
            check(lib.rav_set_coarse_residual_f32(self.h, int(bool(enable)), int(min_dofs), _stream(stream)),
                  "rav_set_coarse_residual_f32")
        k = lib.rav_get_coarse_residual_f32(self.h)
        if k < 0:
            raise RavError(k, "rav_get_coarse_residual_f32")
        return k

    def transfers_f32(self, enable=None, stream=None):
        """FP32 restriction and prolongation in the V-cycle (rav_set_transfers_f32);
        sets it when given, returns 0/1."""
        lib = _capi.load()
        if enable is not None:
            check(lib.rav_set_transfers_f32(self.h, int(bool(enable)), _stream(stream)), "rav_set_transfers_f32")
        k = lib.rav_get_transfers_f32(self.h)
        if k < 0:
            raise RavError(k, "rav_get_transfers_f32")
        return k

    def residual_blocked(self, level, enable=None, stream=None):
        """Node-blocked residual on `level` (Q2-Q1); sets it when given, returns 0/1."""
        lib = _capi.load()
        if enable is not None:
            check(lib.rav_set_residual_blocked(self.h, level, int(bool(enable)), _stream(stream)),
                  "rav_set_residual_blocked")
        k = lib.rav_get_residual_blocked(self.h, level)
        if k < 0:
            raise RavError(k, "rav_get_residual_blocked")
        return k

    def set_graphs(self, enable=True):
        """Replay V-cycles as captured CUDA graphs (default) or launch kernel by kernel."""
        check(_capi.load().rav_set_graphs(self.h, int(enable)), "rav_set_graphs")

    def vcycle(self, sm, x, b, nu_pre=2, nu_post=2, stream=None):
        check(_capi.load().vcycle(self.h, sm.h, _ptr(x), _ptr(b), nu_pre, nu_post, _stream(stream)), "vcycle")
        return x

    def solve(self, sm, x, b, tol=1e-8, maxit=100, nu_pre=2, nu_post=2, outer=0, restart=30, diverge=1e6,
              fallback_rho=0.0, stream=None, raise_on_error=True, info_out=None):
        """Returns (iterations, history ||r_k||/||r_0||, status); info_out (dict) gets 'fell_back'."""
        opts = _capi.RavSolveOpts(tol, maxit, nu_pre, nu_post, outer, restart, diverge, fallback_rho)
        hist = np.zeros(maxit + 1)
        info = _capi.RavSolveInfo(0, 0, 0.0, hist.ctypes.data, 0)
        rc = _capi.load().solve(self.h, sm.h, _ptr(x), _ptr(b), ctypes.byref(opts), ctypes.byref(info),
                                _stream(stream))
        if raise_on_error and rc != 0:
            raise RavError(rc, "solve")
        if info_out is not None:
            info_out["fell_back"] = bool(info.fell_back)
        return info.iterations, hist[: info.iterations + 1].copy(), rc


class Batch:
    """Many problems x nrhs right-hand sides advanced together (batch_setup).

    Vectors are RHS-interleaved: a problem's x has n * nrhs entries, entry
    (row, k) at row * nrhs + k (a torch tensor of shape (n, nrhs), contiguous)."""

    def __init__(self, mgs, sms, nrhs, stream=None):
        lib = _capi.load()
        self.mgs, self.sms, self.nrhs = list(mgs), list(sms), nrhs
        self._mg_arr = (ctypes.c_void_p * len(mgs))(*[m.h.value for m in mgs])
        self._sm_arr = (ctypes.c_void_p * len(sms))(*[s.h.value for s in sms])
        h = ctypes.c_void_p()
        check(lib.batch_setup(self._mg_arr, self._sm_arr, len(mgs), nrhs, _stream(stream), ctypes.byref(h)),
              "batch_setup")
        self.h = h

    def __del__(self):
        if getattr(self, "h", None) is not None and _capi._lib is not None:
            _capi._lib.batch_destroy(self.h)
            self.h = None

    def tuning(self):
        out = (ctypes.c_int * 2)()
        check(_capi.load().batch_get_tuning(self.h, out), "batch_get_tuning")
        return {"residual_threads": out[0], "apply_threads": out[1]}

    def apply_tile(self, ty=None, split=1, stream=None):
        """(rows of vertices per block, warps per row) of the tiled apply at
        each depth, (0, 1) where untiled; ty = 2, 4, 0 or -1 (the set-up
        tuner's choice) first sets every depth (batch_set_apply_tile)."""
        lib = _capi.load()
        if ty is not None:
            check(lib.batch_set_apply_tile(self.h, int(ty), int(split), _stream(stream)), "batch_set_apply_tile")
        out = []
        v = (ctypes.c_int * 2)()
        for d in range(max(m.nlev for m in self.mgs) - 1):
            check(lib.batch_get_apply_tile(self.h, d, v), "batch_get_apply_tile")
            out.append((v[0], v[1]))
        return out

    def tensor_apply(self, enable=True, stream=None):
        """Shared-inverse apply of interior subdomains on the tensor cores
        (batch_set_tensor_apply); returns how many (problem, level) pairs use it."""
        lib = _capi.load()
        check(lib.batch_set_tensor_apply(self.h, int(bool(enable)), _stream(stream)), "batch_set_tensor_apply")
        n = lib.batch_tensor_apply_levels(self.h)
        if n < 0:
            raise RavError(n, "batch_tensor_apply_levels")
        return n

    def coarse_residual_f32(self, enable=True, stream=None):
        """FP32 residuals on the depths below the finest (batch_set_coarse_residual_f32);
        returns whether it is on."""
        lib = _capi.load()
        check(lib.batch_set_coarse_residual_f32(self.h, int(bool(enable)), _stream(stream)),
              "batch_set_coarse_residual_f32")
        k = lib.batch_coarse_residual_f32(self.h)
        if k < 0:
            raise RavError(k, "batch_coarse_residual_f32")
        return bool(k)

    def transfers_f32(self, enable=True, stream=None):
        """FP32 restriction and prolongation (batch_set_transfers_f32); returns whether it is on."""
        lib = _capi.load()
        check(lib.batch_set_transfers_f32(self.h, int(bool(enable)), _stream(stream)), "batch_set_transfers_f32")
        k = lib.batch_transfers_f32(self.h)
        if k < 0:
            raise RavError(k, "batch_transfers_f32")
        return bool(k)

    def profile(self, on=True):
        """Phase-by-phase CUDA-event timing of batched cycles (batch_profile_enable)."""
        check(_capi.load().batch_profile_enable(self.h, int(on)), "batch_profile_enable")

    def profile_read(self, depth, kind):
        """(launches, total ms) of kernel class `kind` at `depth` below the finest grid."""
        n = ctypes.c_int64(0)
        ms = ctypes.c_double(0.0)
        check(_capi.load().batch_profile_read(self.h, depth, kind, ctypes.byref(n), ctypes.byref(ms)),
              "batch_profile_read")
        return n.value, ms.value

    @staticmethod
    def _ptrs(ts):
        return (ctypes.c_void_p * len(ts))(*[_ptr(t).value for t in ts])

    def vcycle(self, xs, bs, nu_pre=2, nu_post=2, stream=None):
        check(_capi.load().batch_vcycle(self.h, self._ptrs(xs), self._ptrs(bs), nu_pre, nu_post, _stream(stream)),
              "batch_vcycle")
        return xs

    def solve(self, xs, bs, tol=1e-8, maxit=100, nu_pre=2, nu_post=2, stream=None, raise_on_error=True):
        """Returns (iterations[nprob, nrhs], ratios[nprob, nrhs], status)."""
        opts = _capi.RavSolveOpts(tol, maxit, nu_pre, nu_post, 0, 30, 0.0, 0.0)
        it = np.zeros(len(xs) * self.nrhs, np.int32)
        ra = np.zeros(len(xs) * self.nrhs)
        rc = _capi.load().solve_batched(self.h, self._ptrs(xs), self._ptrs(bs), ctypes.byref(opts),
                                        it.ctypes.data, ra.ctypes.data, _stream(stream))
        if raise_on_error and rc != 0:
            raise RavError(rc, "solve_batched")
        return it.reshape(len(xs), self.nrhs), ra.reshape(len(xs), self.nrhs), rc


class Smoother:
    """Vanka subdomains and stored inverses (vanka_setup)."""

    def __init__(self, mg: Multigrid, kind=RAV, precision=F64, omega=0.5, stream=None):
        h = ctypes.c_void_p()
        check(_capi.load().vanka_setup(mg.h, kind, precision, float(omega), _stream(stream), ctypes.byref(h)),
              "vanka_setup")
        self.h = h
        self.mg, self.kind, self.precision = mg, kind, precision

    def __del__(self):
        if getattr(self, "h", None) is not None and _capi._lib is not None:
            _capi._lib.vanka_destroy(self.h)
            self.h = None

    def smooth(self, level, x, b, steps=1, stream=None):
        check(_capi.load().vanka_smooth(self.h, level, _ptr(x), _ptr(b), steps, _stream(stream)), "vanka_smooth")
        return x

    def apply(self, level, r, x, stream=None):
        """x += S r (the subdomain part of one RAV/AV step for a given residual r)."""
        check(_capi.load().vanka_apply(self.h, level, _ptr(r), _ptr(x), _stream(stream)), "vanka_apply")
        return x

    def apply_split(self, level, split=None, stream=None):
        """Threads per owned node of the factored apply on `level`; sets it when given."""
        lib = _capi.load()
        if split is not None:
            check(lib.rav_set_apply_split(self.h, level, int(split), _stream(stream)), "rav_set_apply_split")
        k = lib.rav_get_apply_split(self.h, level)
        if k < 0:
            raise RavError(k, "rav_get_apply_split")
        return k

    def apply_staged(self, level, threads_per_subdomain=None, stream=None):
        """Threads per subdomain of the staged reduced-precision apply on
        `level` (0: the grouped kernel); sets it when given."""
        lib = _capi.load()
        if threads_per_subdomain is not None:
            check(lib.rav_set_apply_staged(self.h, level, int(threads_per_subdomain), _stream(stream)),
                  "rav_set_apply_staged")
        k = lib.rav_get_apply_staged(self.h, level)
        if k < 0:
            raise RavError(k, "rav_get_apply_staged")
        return k

    def fused(self, enable=True):
        """Q1-Q1 RAV fp64: run each smoothing step as one fused residual + apply kernel."""
        check(_capi.load().rav_set_fused_smoothing(self.h, int(bool(enable))), "rav_set_fused_smoothing")

    def set_omega(self, level, w, stream=None):
        w = w.to(dtype=_torch().float32).contiguous()
        check(_capi.load().rav_set_patch_omega(self.h, level, _ptr(w), _stream(stream)), "rav_set_patch_omega")

    def patch_counts(self, level):
        out = (ctypes.c_int64 * 2)()
        check(_capi.load().rav_get_patch_counts(self.h, level, out), "rav_get_patch_counts")
        return out[0], out[1]

    def patches(self, level, stream=None):
        torch = _torch()
        np_, tot = self.patch_counts(level)
        n = self.mg.n(level)
        off = torch.empty(np_ + 1, dtype=torch.int32, device="cuda")
        dofs = torch.empty(tot, dtype=torch.int32, device="cuda")
        own = torch.empty(n, dtype=torch.int32, device="cuda")
        check(_capi.load().rav_get_patches(self.h, level, _ptr(off), _ptr(dofs), _ptr(own), _stream(stream)),
              "rav_get_patches")
        return off, dofs, own

    def inverse_rows(self, level, first, count, stream=None):
        d = self.mg.dim
        if self.mg.element == ELEM_Q1Q1:
            nc = 3 ** d * d + 1
            nr = d + 1 if self.kind == RAV else nc
        else:
            nc = 5 ** d * d + 1
            nr = (2 ** d * d + 1) if self.kind == RAV else nc
        out = _torch().empty((count, nr, nc), dtype=_torch().float64, device="cuda")
        check(_capi.load().rav_get_inverse_rows(self.h, level, first, count, _ptr(out), _stream(stream)),
              "rav_get_inverse_rows")
        return out
