"""Error paths of the C ABI, driven by faults injected on the host.

Every failure here is made by the caller's data or options: a NaN written
into the smoother's per-subdomain damping or into b, a viscosity that makes
the local systems indefinite, an iteration cap below what the tolerance
needs, a damping beyond the smoother's stable range.  No test faults, traps or
stalls the GPU.  Each checks the status code and the filled rav_solve_info
(iterations, status, final ratio, history) against what the oracle's own run
of the same iteration gives.
"""
import ctypes

import numpy as np
import pytest

import oracle as O

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

import paper_2103_10127_gb300 as R  # noqa: E402
from paper_2103_10127_gb300 import _capi  # noqa: E402

RAV_ERR_SINGULAR_PATCH, RAV_ERR_NOT_CONVERGED, RAV_ERR_DIVERGED, RAV_ERR_NAN = -3, -5, -6, -7


def _solve_raw(mg, sm, x, b, tol=1e-8, maxit=40, outer=0, diverge=1e6):
    """solve() through the C ABI, returning the status and the filled info."""
    lib = _capi.load()
    opts = _capi.RavSolveOpts(tol, maxit, 2, 2, outer, 30, diverge, 0.0)
    hist = np.full(maxit + 1, -1.0)
    info = _capi.RavSolveInfo(-99, 99, -1.0, hist.ctypes.data, 7)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = lib.solve(mg.h, sm.h, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(b.data_ptr()), ctypes.byref(opts),
                   ctypes.byref(info), stream)
    return rc, info, hist


@pytest.mark.parametrize("outer", [0, 1], ids=["stationary", "fgmres"])
def test_nan_in_the_stored_damping_gives_nan_status(outer):
    """One subdomain's damping set to NaN from the host: the first cycle's
    residual is non-finite, solve stops there with RAV_ERR_NAN."""
    mg = R.Multigrid(2, 16, 3, bc=R.BC_CAVITY)
    sm = R.Smoother(mg, R.RAV, R.F64, 0.5)
    fine = mg.nlev - 1
    w = torch.full((mg.counts(fine)["n_p"],), 0.5, dtype=torch.float32, device="cuda")
    w[17 * 8 + 8] = float("nan")  # an interior vertex of the 16x16 grid
    sm.set_omega(fine, w)
    x = mg.initial_guess()
    rc, info, hist = _solve_raw(mg, sm, x, mg.rhs(R.F_NONE), outer=outer)
    assert rc == RAV_ERR_NAN and info.status == RAV_ERR_NAN
    assert info.iterations == 1
    assert hist[0] == 1.0 and not np.isfinite(hist[1]) and not np.isfinite(info.final_ratio)
    assert info.fell_back == 0


def test_nan_in_the_right_hand_side_gives_nan_status():
    mg = R.Multigrid(2, 16, 3, bc=R.BC_CAVITY)
    sm = R.Smoother(mg, R.RAV, R.F64, 0.5)
    b = mg.rhs(R.F_NONE)
    b[2 * (33 * 16 + 16)] = float("nan")  # velocity DoF of the centre node
    rc, info, hist = _solve_raw(mg, sm, mg.initial_guess(), b)
    assert rc == RAV_ERR_NAN and info.status == RAV_ERR_NAN and info.iterations == 1
    assert not np.isfinite(info.final_ratio)


@pytest.mark.parametrize("dim,N,element", [(2, 8, R.ELEM_Q2Q1), (3, 4, R.ELEM_Q2Q1), (2, 8, R.ELEM_Q1Q1)],
                         ids=["q2q1-2d", "q2q1-3d", "q1q1-2d"])
@pytest.mark.parametrize("kind", [R.RAV, R.AV])
def test_indefinite_subdomains_give_singular_patch(dim, N, element, kind):
    """A negative viscosity makes every velocity block K_i negative definite:
    the coarse bordered system is still invertible (mg_setup succeeds), but the
    subdomain factorisation meets a non-positive pivot and vanka_setup returns
    RAV_ERR_SINGULAR_PATCH without leaving a handle."""
    mg = R.Multigrid(dim, N, 2, eta0=-1.0, bc=R.BC_NOSLIP, element=element, beta=0.02)
    with pytest.raises(R.RavError) as e:
        R.Smoother(mg, kind, R.F64, 0.5)
    assert e.value.code == RAV_ERR_SINGULAR_PATCH
    # the hierarchy stays usable: a healthy hierarchy next to it still sets up
    ok = R.Multigrid(dim, N, 2, bc=R.BC_NOSLIP, element=element, beta=0.02)
    R.Smoother(ok, kind, R.F64, 0.5)


@pytest.mark.parametrize("outer", [0, 1], ids=["stationary", "fgmres"])
def test_iteration_cap_gives_not_converged_with_history(outer):
    """maxit = 2 is below what 1e-8 needs: RAV_ERR_NOT_CONVERGED, two
    iterations, and the history of the oracle's same iteration."""
    mg = R.Multigrid(2, 16, 3, bc=R.BC_CAVITY)
    sm = R.Smoother(mg, R.RAV, R.F64, 0.5)
    orc = O.Oracle(2, 16, 3, bc=O.BC_CAVITY)
    orc.setup_smoother(O.RAV, 0.5)
    rc, info, hist = _solve_raw(mg, sm, mg.initial_guess(), mg.rhs(R.F_NONE), maxit=2, outer=outer)
    assert rc == RAV_ERR_NOT_CONVERGED and info.status == RAV_ERR_NOT_CONVERGED
    assert info.iterations == 2
    if outer == 0:
        _, oit, ohist = orc.solve(orc.initial_guess(), orc.rhs(O.F_NONE), tol=1e-8, maxit=2)
    else:
        _, oit, ohist = orc.fgmres(orc.initial_guess(), orc.rhs(O.F_NONE), tol=1e-8, maxit=2)
    assert oit == RAV_ERR_NOT_CONVERGED or oit == 2
    assert np.allclose(hist[:3], ohist[:3], rtol=1e-6 if outer == 0 else 1e-4, atol=0)
    assert info.final_ratio == hist[2] and info.final_ratio > 1e-8


def test_unstable_damping_gives_diverged():
    """RAV with damping 1.5 on the 16x16 cavity amplifies the residual every
    cycle (the oracle's run of the same iteration does too); solve stops with
    RAV_ERR_DIVERGED at the first cycle whose ratio passes the guard 1e6."""
    mg = R.Multigrid(2, 16, 3, bc=R.BC_CAVITY)
    sm = R.Smoother(mg, R.RAV, R.F64, 1.5)
    orc = O.Oracle(2, 16, 3, bc=O.BC_CAVITY)
    orc.setup_smoother(O.RAV, 1.5)
    rc, info, hist = _solve_raw(mg, sm, mg.initial_guess(), mg.rhs(R.F_NONE), maxit=40)
    _, oit, ohist = orc.solve(orc.initial_guess(), orc.rhs(O.F_NONE), tol=1e-8, maxit=40)
    assert rc == RAV_ERR_DIVERGED and info.status == RAV_ERR_DIVERGED
    k = int(np.argmax(ohist > 1e6))  # the oracle's first cycle beyond the guard
    assert k > 1 and info.iterations == k
    assert info.final_ratio == hist[k] and hist[k] > 1e6
    assert np.allclose(hist[:k + 1], ohist[:k + 1], rtol=1e-6, atol=0)


def test_batched_iteration_cap_gives_not_converged():
    """Two problems x 2 right-hand sides, one cycle allowed: every system
    misses 1e-8, solve_batched returns RAV_ERR_NOT_CONVERGED and marks each
    with -1 cycles and its last ratio."""
    mgs = [R.Multigrid(2, 16, 3, bc=R.BC_CAVITY), R.Multigrid(2, 32, 3, bc=R.BC_CAVITY)]
    sms = [R.Smoother(m, R.RAV, R.F32, 0.5) for m in mgs]
    bt = R.Batch(mgs, sms, 2)
    xs, bs = [], []
    for m in mgs:
        x0, b0 = m.initial_guess(), m.rhs(R.F_NONE)
        xs.append(x0[:, None].repeat(1, 2).contiguous())
        bs.append(b0[:, None].repeat(1, 2).contiguous())
    it, ra, rc = bt.solve(xs, bs, tol=1e-8, maxit=1, raise_on_error=False)
    assert rc == RAV_ERR_NOT_CONVERGED
    assert np.all(it == -1)
    assert np.all((ra > 1e-8) & (ra < 1.0))
