"""Edge cases of the CUDA path through the C ABI: the degenerate hierarchies,
weights and inputs the method admits, against the oracle or exact answers."""
import ctypes

import numpy as np
import pytest

import oracle as O

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

import paper_2103_10127_gb300 as R  # noqa: E402
from paper_2103_10127_gb300 import _capi, inputs  # noqa: E402


def cpu(t):
    return t.detach().cpu().numpy()


def gpu(a):
    return torch.from_numpy(np.ascontiguousarray(a, np.float64)).cuda()


@pytest.mark.parametrize("dim,N", [(2, 4), (3, 2)])
def test_single_level_cycle_is_the_exact_coarse_solve(dim, N):
    """One level: the V-cycle is the bordered LU solve, so one cycle leaves a
    residual at roundoff and equals the oracle's coarse solve."""
    mg = R.Multigrid(dim, N, 1, bc=R.BC_QUADRATIC)
    sm = R.Smoother(mg, R.RAV, R.F64, 0.5)
    b = mg.rhs(R.F_QUADRATIC)
    x = mg.initial_guess()
    mg.vcycle(sm, x, b, 2, 2)
    _, r = mg.residual(0, x, b, norm=True)
    _, r0 = mg.residual(0, mg.initial_guess(), b, norm=True)
    assert r <= 1e-11 * r0
    orc = O.Oracle(dim, N, 1, bc=O.BC_QUADRATIC)
    ob = orc.rhs(O.F_QUADRATIC)
    ox = orc.initial_guess()
    want = ox + orc.coarse_solve(orc.residual(0, ox, ob))
    nu = mg.counts(0)["n_u"]
    assert np.abs(cpu(x)[:nu] - want[:nu]).max() <= 1e-10 * max(1.0, np.abs(want[:nu]).max())
    it, hist, rc = mg.solve(sm, mg.initial_guess(), b, tol=1e-8, maxit=5)
    assert rc == 0 and it == 1


def test_zero_problem_needs_no_iteration():
    mg = R.Multigrid(2, 8, 2, bc=R.BC_NOSLIP)
    sm = R.Smoother(mg, R.RAV, R.F64, 0.5)
    x = mg.initial_guess()
    for outer in (0, 1):
        it, hist, rc = mg.solve(sm, x, mg.rhs(R.F_NONE), tol=1e-8, maxit=10, outer=outer)
        assert rc == 0 and it == 0
    assert not cpu(x).any()


@pytest.mark.parametrize("prec", [R.F64, R.F64_ROWS, R.F32, R.BF16_FACT])
def test_zero_damping_and_zero_steps_leave_x_unchanged(prec):
    mg = R.Multigrid(2, 8, 2, bc=R.BC_CAVITY)
    sm = R.Smoother(mg, R.RAV, prec, 0.0)
    rng = np.random.default_rng(1)
    n = mg.n()
    x0, b = rng.standard_normal(n), rng.standard_normal(n)
    x = gpu(x0)
    sm.smooth(1, x, gpu(b), 3)
    assert np.array_equal(cpu(x), x0)
    sm2 = R.Smoother(mg, R.RAV, prec, 0.5)
    sm2.smooth(1, x, gpu(b), 0)
    assert np.array_equal(cpu(x), x0)


@pytest.mark.parametrize("prec", [R.F64, R.F32, R.FP8, R.F32_FACT])
def test_zero_residual_gives_zero_correction(prec):
    mg = R.Multigrid(3, 4, 2, bc=R.BC_NOSLIP)
    sm = R.Smoother(mg, R.RAV, prec, 0.5)
    n = mg.n()
    x0 = np.random.default_rng(2).standard_normal(n)
    x = gpu(x0)
    sm.apply(1, torch.zeros(n, dtype=torch.float64, device="cuda"), x)
    assert np.array_equal(cpu(x), x0)


@pytest.mark.parametrize("dim,N,nlev", [(2, 4, 2), (3, 4, 2), (2, 6, 2)])
def test_smallest_hierarchies_match_the_oracle(dim, N, nlev):
    """Coarsest grids of 2 or 3 cells per axis, where every subdomain touches
    the boundary."""
    coords = inputs.graded_coordinates(N, 3.0, dim)
    mg = R.Multigrid(dim, N, nlev, coords=coords, bc=R.BC_NOSLIP)
    orc = O.Oracle(dim, N, nlev, coords=coords, bc=O.BC_NOSLIP)
    sm = R.Smoother(mg, R.RAV, R.F64, 0.5)
    orc.setup_smoother(O.RAV, 0.5)
    rng = np.random.default_rng(3)
    n = mg.n()
    x, b = rng.standard_normal(n), rng.standard_normal(n)
    want = orc.vcycle(x, b, 2, 2)
    xg = gpu(x)
    mg.vcycle(sm, xg, gpu(b), 2, 2)
    assert np.abs(cpu(xg) - want).max() <= 1e-11 * np.abs(want).max()


def test_invalid_calls_are_rejected_without_side_effects():
    mg = R.Multigrid(2, 8, 2, bc=R.BC_NOSLIP)
    sm = R.Smoother(mg, R.RAV, R.F64, 0.5)
    x = mg.initial_guess()
    x0 = cpu(x).copy()
    for bad in (lambda: sm.smooth(0, x, x, 1), lambda: sm.smooth(2, x, x, 1), lambda: sm.apply_split(1, 16),
                lambda: mg.residual_split(2, 1), lambda: R.Smoother(mg, R.AV, R.F32, 0.1)):
        with pytest.raises(R.RavError):
            bad()
    assert np.array_equal(cpu(x), x0)


def test_measured_read_rate_is_a_bandwidth():
    """rav_hbm_read_rate (the size-matched context of the memory-bound
    rooflines): a positive finite GB/s below any HBM3e figure, and a read of
    256 MB runs at least as fast per byte as one of 1 MB (launch and ramp-up
    weigh less)."""
    lib = _capi.load()
    rates = []
    for nbytes in (1 << 20, 256 << 20):
        r = ctypes.c_double()
        assert lib.rav_hbm_read_rate(nbytes, ctypes.byref(r), None) == 0
        assert 10.0 < r.value < 20000.0
        rates.append(r.value)
    assert rates[1] >= rates[0]
