"""Batched multi-problem, multi-RHS solves (batch_setup / batch_vcycle /
solve_batched) against the single-problem path and the oracle."""
import numpy as np
import pytest

import oracle as O
from paper_2103_10127_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

import paper_2103_10127_gb300 as R  # noqa: E402


def free_velocity(dim, N):
    M = 2 * N + 1
    idx = np.indices((M,) * dim).reshape(dim, -1)[::-1]  # axis 0 fastest
    inner = np.all((idx > 0) & (idx < M - 1), axis=0)
    return np.concatenate([np.repeat(inner, dim), np.zeros((N + 1) ** dim, bool)])


def random_rhs(mg, seed):
    """Lid values on Dirichlet rows plus iid N(0,1) forcing on free velocity rows."""
    b = mg.rhs(R.F_NONE).cpu().numpy()
    m = free_velocity(mg.dim, mg.N)
    b[m] += inputs.normal(seed, int(m.sum()))
    return b


def make_batch(sizes, nrhs, prec, seed=0):
    mgs, sms, xs, bs = [], [], [], []
    for i, N in enumerate(sizes):
        L = inputs.levels_for(N)
        mg = R.Multigrid(2, N, L, bc=R.BC_CAVITY)
        sm = R.Smoother(mg, R.RAV, prec, 0.5)
        n = mg.n()
        b = np.stack([random_rhs(mg, 1000 * seed + 10 * i + k) for k in range(nrhs)], axis=1)
        x0 = mg.initial_guess().cpu().numpy()
        x = np.repeat(x0[:, None], nrhs, axis=1)
        mgs.append(mg)
        sms.append(sm)
        xs.append(torch.from_numpy(np.ascontiguousarray(x)).cuda())
        bs.append(torch.from_numpy(np.ascontiguousarray(b)).cuda())
    return mgs, sms, xs, bs


SIZES = [16, 24, 32, 48, 20]


@pytest.mark.parametrize("prec", [R.F32, R.F64_ROWS])
def test_batched_vcycle_equals_single_problem_cycles_bitwise(prec):
    nrhs = 4
    mgs, sms, xs, bs = make_batch(SIZES, nrhs, prec)
    bt = R.Batch(mgs, sms, nrhs)
    x_in = [x.clone() for x in xs]
    bt.vcycle(xs, bs, 2, 2)
    bt.vcycle(xs, bs, 2, 2)
    for p, (mg, sm) in enumerate(zip(mgs, sms)):
        for lev in range(mg.nlev):  # the batched residual sums a row in one thread, as split 1 does
            mg.residual_split(lev, 1)
        for k in range(nrhs):
            x = x_in[p][:, k].contiguous()
            b = bs[p][:, k].contiguous()
            mg.vcycle(sm, x, b, 2, 2)
            mg.vcycle(sm, x, b, 2, 2)
            assert torch.equal(x, xs[p][:, k]), (p, k)
    assert bt.tuning()["residual_threads"] in (128, 256, 512)


def test_batched_vcycle_matches_the_oracle():
    nrhs = 2
    mgs, sms, xs, bs = make_batch([16, 24], nrhs, R.F64_ROWS, seed=3)
    bt = R.Batch(mgs, sms, nrhs)
    x_in = [x.cpu().numpy() for x in xs]
    bt.vcycle(xs, bs, 2, 2)
    for p, N in enumerate([16, 24]):
        orc = O.Oracle(2, N, inputs.levels_for(N), bc=O.BC_CAVITY)
        orc.setup_smoother(O.RAV, 0.5)
        for k in range(nrhs):
            want = orc.vcycle(x_in[p][:, k], bs[p][:, k].cpu().numpy(), 2, 2)
            got = xs[p][:, k].cpu().numpy()
            assert np.abs(got - want).max() <= 1e-11 * np.abs(want).max()


def test_batched_solve_matches_single_solves():
    nrhs = 2
    mgs, sms, xs, bs = make_batch(SIZES, nrhs, R.F32, seed=5)
    bt = R.Batch(mgs, sms, nrhs)
    x_in = [x.clone() for x in xs]
    it, ratios, rc = bt.solve(xs, bs, tol=1e-8, maxit=100)
    assert rc == 0 and np.all(it > 0) and np.all(ratios <= 1e-8)
    for p, (mg, sm) in enumerate(zip(mgs, sms)):
        for k in range(nrhs):
            x = x_in[p][:, k].contiguous()
            b = bs[p][:, k].contiguous()
            its, hist, rcs = mg.solve(sm, x, b, tol=1e-8, maxit=100)
            assert rcs == 0 and its == it[p, k]


@pytest.mark.parametrize("prec", [R.F32, R.F64_ROWS])
def test_batched_3d_cycles_equal_single_problem_cycles_bitwise(prec):
    """Two 3-D problems of different depth (8^3 with 2 levels, 16^3 with 3),
    blob viscosity, 2 right-hand sides each."""
    nrhs = 2
    mgs, sms, xs, bs = [], [], [], []
    for i, (N, nlev) in enumerate([(8, 2), (16, 3)]):
        mg = R.Multigrid(3, N, nlev, blobs=inputs.viscosity_blobs(40 + i, k=4, s_max=2.0), bc=R.BC_CAVITY)
        sm = R.Smoother(mg, R.RAV, prec, 0.5)
        b = np.stack([random_rhs(mg, 300 + 10 * i + k) for k in range(nrhs)], axis=1)
        x0 = mg.initial_guess().cpu().numpy()
        mgs.append(mg)
        sms.append(sm)
        xs.append(torch.from_numpy(np.ascontiguousarray(np.repeat(x0[:, None], nrhs, axis=1))).cuda())
        bs.append(torch.from_numpy(np.ascontiguousarray(b)).cuda())
    bt = R.Batch(mgs, sms, nrhs)
    x_in = [x.clone() for x in xs]
    bt.vcycle(xs, bs, 2, 2)
    for p, (mg, sm) in enumerate(zip(mgs, sms)):
        for lev in range(mg.nlev):
            mg.residual_split(lev, 1)
        for k in range(nrhs):
            x = x_in[p][:, k].contiguous()
            mg.vcycle(sm, x, bs[p][:, k].contiguous(), 2, 2)
            assert torch.equal(x, xs[p][:, k]), (p, k)


@pytest.mark.slow
def test_full_size_batch_sampled_bitwise():
    """The batched benchmark's configuration: 256 cavities of N = 16 m,
    m ~ U{2..16} (seed 2103), 8 right-hand sides each, FP32 inverses.  One
    batched V(2,2) cycle; the smallest, the largest and two seeded problems are
    checked right-hand side by right-hand side, bit for bit, against
    single-problem cycles."""
    sizes = inputs.batched_sizes(inputs.BASE_SEED, 256)
    nrhs = 8
    mgs, sms, xs, bs = [], [], [], []
    for i, N in enumerate(sizes):
        N = int(N)
        mg = R.Multigrid(2, N, inputs.levels_for(N), bc=R.BC_CAVITY)
        sm = R.Smoother(mg, R.RAV, R.F32, 0.5)
        m = free_velocity(2, N)
        b0 = mg.rhs(R.F_NONE).cpu().numpy()
        b = np.repeat(b0[:, None], nrhs, axis=1)
        b[m, :] += inputs.normal(inputs.BASE_SEED + 7919 * (i + 1), int(m.sum()) * nrhs).reshape(-1, nrhs)
        x0 = mg.initial_guess().cpu().numpy()
        mgs.append(mg)
        sms.append(sm)
        xs.append(torch.from_numpy(np.ascontiguousarray(np.repeat(x0[:, None], nrhs, axis=1))).cuda())
        bs.append(torch.from_numpy(np.ascontiguousarray(b)).cuda())
    bt = R.Batch(mgs, sms, nrhs)
    x_in = {}
    picks = sorted({int(np.argmin(sizes)), int(np.argmax(sizes))} |
                   set((inputs.uniform(77, 2) * len(sizes)).astype(int).tolist()))
    for p in picks:
        x_in[p] = xs[p].clone()
    bt.vcycle(xs, bs, 2, 2)
    for p in picks:
        mg, sm = mgs[p], sms[p]
        for lev in range(mg.nlev):
            mg.residual_split(lev, 1)
        for k in range(nrhs):
            x = x_in[p][:, k].contiguous()
            mg.vcycle(sm, x, bs[p][:, k].contiguous(), 2, 2)
            assert torch.equal(x, xs[p][:, k]), (p, k)


def test_tensor_core_shared_inverse_apply_matches_the_cuda_core_apply():
    """Uniform constant-viscosity cavities: every interior subdomain of a level
    shares its owned rows, so the batch applies them as one tcgen05 GEMM per 16
    subdomains x 8 right-hand sides (tf32 split into high and low parts, fp32
    accumulation).  One batched cycle equals the fp32 CUDA-core cycle to fp32
    roundoff of the step, a solve takes the same cycles per system, and
    switching it off restores the CUDA-core result bit for bit."""
    nrhs = 8
    sizes = [16, 32, 48, 64, 24]
    mgs, sms, xs, bs = make_batch(sizes, nrhs, R.F32, seed=5)
    bt = R.Batch(mgs, sms, nrhs)
    x_in = [x.clone() for x in xs]
    bt.vcycle(xs, bs, 2, 2)
    ref = [x.clone() for x in xs]
    nlev = sum(m.nlev - 1 for m in mgs)  # levels with subdomains; N >= 4 everywhere here
    assert bt.tensor_apply(True) == nlev
    for x, xi in zip(xs, x_in):
        x.copy_(xi)
    bt.vcycle(xs, bs, 2, 2)
    for p in range(len(sizes)):
        step_ref = (ref[p] - x_in[p]).cpu().numpy()
        step_tc = (xs[p] - x_in[p]).cpu().numpy()
        for k in range(nrhs):
            d = np.linalg.norm(step_tc[:, k] - step_ref[:, k])
            assert d <= 1e-5 * np.linalg.norm(step_ref[:, k]), (p, k, d)
    for x, xi in zip(xs, x_in):
        x.copy_(xi)
    it_tc, ra_tc, rc = bt.solve(xs, bs, tol=1e-8, maxit=60)
    assert rc == 0 and np.all(ra_tc <= 1e-8)
    assert bt.tensor_apply(False) == 0
    for x, xi in zip(xs, x_in):
        x.copy_(xi)
    bt.vcycle(xs, bs, 2, 2)
    for p in range(len(sizes)):
        assert torch.equal(xs[p], ref[p]), p
    for x, xi in zip(xs, x_in):
        x.copy_(xi)
    it_cc, _, rc = bt.solve(xs, bs, tol=1e-8, maxit=60)
    assert rc == 0 and np.array_equal(it_tc, it_cc)


def test_tensor_core_apply_only_where_rows_are_shared():
    """Blob viscosity breaks the translation invariance of the local systems:
    those levels keep the CUDA-core apply (and give its result bit for bit),
    while a uniform problem in the same batch uses the tensor cores; the
    uniform problem's step still matches the CUDA-core step."""
    nrhs = 8
    mg_u = R.Multigrid(2, 32, 3, bc=R.BC_CAVITY)
    mg_b = R.Multigrid(2, 32, 3, bc=R.BC_CAVITY, blobs=inputs.viscosity_blobs(9, k=4, s_max=1.0))
    mgs = [mg_u, mg_b]
    sms = [R.Smoother(m, R.RAV, R.F32, 0.5) for m in mgs]
    xs, bs = [], []
    for i, m in enumerate(mgs):
        b = np.stack([random_rhs(m, 77 + 10 * i + k) for k in range(nrhs)], axis=1)
        xs.append(torch.from_numpy(np.repeat(m.initial_guess().cpu().numpy()[:, None], nrhs, axis=1).copy()).cuda())
        bs.append(torch.from_numpy(np.ascontiguousarray(b)).cuda())
    bt = R.Batch(mgs, sms, nrhs)
    x_in = [x.clone() for x in xs]
    bt.vcycle(xs, bs, 2, 2)
    ref = [x.clone() for x in xs]
    assert bt.tensor_apply(True) == mg_u.nlev - 1
    for x, xi in zip(xs, x_in):
        x.copy_(xi)
    bt.vcycle(xs, bs, 2, 2)
    assert torch.equal(xs[1], ref[1])
    d = (xs[0] - ref[0]).norm() / (ref[0] - x_in[0]).norm()
    assert 0.0 < d.item() <= 1e-5
    with pytest.raises(R.RavError):
        R.Batch(mgs, sms, 4).tensor_apply(True)  # 8 right-hand sides only


@pytest.mark.parametrize("nrhs", [1, 2, 8])
def test_coarse_residual_f32_batched_cycle(nrhs):
    """batch_set_coarse_residual_f32: with fp64 rows (the apply reads r in
    fp64) one batched V-cycle with fp32 residuals below the finest depth
    differs from the fp64-residual cycle only by their fp32 rounding; switching
    back restores the fp64 cycle bit for bit."""
    mgs, sms, xs, bs = make_batch(SIZES, nrhs, R.F64_ROWS, seed=7)
    bt = R.Batch(mgs, sms, nrhs)
    x_in = [x.clone() for x in xs]
    ref = [x.clone() for x in x_in]
    bt.vcycle(ref, bs, 2, 2)
    assert bt.coarse_residual_f32(True)
    got = [x.clone() for x in x_in]
    bt.vcycle(got, bs, 2, 2)
    for p in range(len(SIZES)):
        d = (got[p] - x_in[p]).cpu().numpy()
        w = (ref[p] - x_in[p]).cpu().numpy()
        assert np.linalg.norm(d - w) <= 1e-5 * np.linalg.norm(w), p
    assert not bt.coarse_residual_f32(False)
    again = [x.clone() for x in x_in]
    bt.vcycle(again, bs, 2, 2)
    for p in range(len(SIZES)):
        assert torch.equal(again[p], ref[p]), p


@pytest.mark.parametrize("nrhs", [2, 8])
def test_coarse_residual_f32_batched_solve_takes_the_same_cycles(nrhs):
    """FP32 rows with fp32 residuals below the finest depth reach 1e-8 in the
    same number of cycles per system as with fp64 residuals there."""
    mgs, sms, xs, bs = make_batch(SIZES, nrhs, R.F32, seed=9)
    out = []
    for on in (False, True):
        bt = R.Batch(mgs, sms, nrhs)
        bt.coarse_residual_f32(on)
        x = [t.clone() for t in xs]
        it, ratios, rc = bt.solve(x, bs, tol=1e-8, maxit=100)
        assert rc == 0 and np.all(ratios <= 1e-8)
        out.append(it)
        del bt
    assert np.array_equal(out[0], out[1])


@pytest.mark.parametrize("nrhs", [1, 8])
def test_transfers_f32_batched_cycle_equals_single_problem_cycles(nrhs):
    """batch_set_transfers_f32: one batched V-cycle with fp32 restriction and
    prolongation differs from the fp64-transfer cycle only by their fp32
    rounding, gives each right-hand side's single-problem cycle with
    rav_set_transfers_f32 bit for bit (same sums in the same order), and off
    restores the fp64 cycle bit for bit."""
    sizes = SIZES[:3]
    mgs, sms, xs, bs = make_batch(sizes, nrhs, R.F32, seed=11)
    bt = R.Batch(mgs, sms, nrhs)
    x_in = [x.clone() for x in xs]
    ref = [x.clone() for x in x_in]
    bt.vcycle(ref, bs, 2, 2)
    assert bt.transfers_f32(True)
    got = [x.clone() for x in x_in]
    bt.vcycle(got, bs, 2, 2)
    for p in range(len(sizes)):
        d = (got[p] - x_in[p]).cpu().numpy()
        w = (ref[p] - x_in[p]).cpu().numpy()
        assert 0.0 < np.linalg.norm(d - w) <= 1e-5 * np.linalg.norm(w), p
    for p, (mg, sm) in enumerate(zip(mgs, sms)):
        for lev in range(mg.nlev):
            mg.residual_split(lev, 1)
        assert mg.transfers_f32(True) == 1
        for k in range(nrhs):
            x = x_in[p][:, k].clone()  # a copy also when the column is contiguous (nrhs = 1)
            mg.vcycle(sm, x, bs[p][:, k].contiguous(), 2, 2)
            assert torch.equal(x, got[p][:, k]), (p, k)
        mg.transfers_f32(False)
    assert not bt.transfers_f32(False)
    again = [x.clone() for x in x_in]
    bt.vcycle(again, bs, 2, 2)
    for p in range(len(sizes)):
        assert torch.equal(again[p], ref[p]), p


def test_transfers_f32_batched_refuses_fp64_rows():
    """The fp32 restriction reads the fp32 residual copy that only fp32 rows keep."""
    mgs, sms, xs, bs = make_batch(SIZES[:2], 2, R.F64_ROWS, seed=3)
    bt = R.Batch(mgs, sms, 2)
    with pytest.raises(R.RavError):
        bt.transfers_f32(True)
    assert not bt.transfers_f32(False)


@pytest.mark.parametrize("nrhs", [2, 8])
def test_f32_coarse_grid_work_batched_solve_takes_the_same_cycles(nrhs):
    """FP32 rows with fp32 residuals below the finest depth and fp32 transfers
    reach 1e-8 in the same number of cycles per system as with fp64 ones."""
    mgs, sms, xs, bs = make_batch(SIZES, nrhs, R.F32, seed=13)
    out = []
    for on in (False, True):
        bt = R.Batch(mgs, sms, nrhs)
        bt.coarse_residual_f32(on)
        bt.transfers_f32(on)
        x = [t.clone() for t in xs]
        it, ratios, rc = bt.solve(x, bs, tol=1e-8, maxit=100)
        assert rc == 0 and np.all(ratios <= 1e-8)
        out.append(it)
        del bt
    assert np.array_equal(out[0], out[1])


@pytest.mark.parametrize("tc", [False, True])
def test_tiled_apply_equals_untiled_bitwise(tc):
    """batch_set_apply_tile: the tiled apply (32 x 2 or 32 x 4 vertices per
    block, one warp or two per row of vertices; several blocks per row and
    ragged edges on these sizes) gives the untiled kernel's cycle bit for bit,
    also where the tensor-core apply owns the interior subdomains."""
    nrhs = 8
    mgs, sms, xs, bs = make_batch(SIZES, nrhs, R.F32, seed=17)
    bt = R.Batch(mgs, sms, nrhs)
    auto = bt.apply_tile()
    assert all(t in ((0, 1), (2, 1), (4, 1), (2, 2), (4, 2)) for t in auto)
    if tc:
        assert bt.tensor_apply(True) > 0
    x_in = [x.clone() for x in xs]
    assert bt.apply_tile(0) == [(0, 1)] * len(auto)
    ref = [x.clone() for x in x_in]
    bt.vcycle(ref, bs, 2, 2)
    bt.vcycle(ref, bs, 2, 2)
    for ty, split in ((2, 1), (4, 1), (2, 2), (4, 2)):
        assert bt.apply_tile(ty, split) == [(ty, split)] * len(auto)
        got = [x.clone() for x in x_in]
        bt.vcycle(got, bs, 2, 2)
        bt.vcycle(got, bs, 2, 2)
        for p in range(len(SIZES)):
            assert torch.equal(got[p], ref[p]), (ty, split, p)
    assert bt.apply_tile(-1) == auto


def test_tiled_apply_arguments():
    """Tiles only for 2-D Q2-Q1 batches with fp32 rows and 8 right-hand sides;
    ty in {-1, 0, 2, 4}, split in {1, 2}."""
    mgs, sms, xs, bs = make_batch(SIZES[:2], 8, R.F32, seed=19)
    bt = R.Batch(mgs, sms, 8)
    for ty, split in ((1, 1), (3, 1), (8, 1), (-2, 1), (2, 0), (2, 3), (4, 4)):
        with pytest.raises(R.RavError):
            bt.apply_tile(ty, split)
    mgs4, sms4, _, _ = make_batch(SIZES[:2], 4, R.F32, seed=19)
    bt4 = R.Batch(mgs4, sms4, 4)
    assert bt4.apply_tile() == [(0, 1)] * (max(m.nlev for m in mgs4) - 1)
    with pytest.raises(R.RavError):
        bt4.apply_tile(2)
    mgs64, sms64, _, _ = make_batch(SIZES[:2], 8, R.F64_ROWS, seed=19)
    bt64 = R.Batch(mgs64, sms64, 8)
    with pytest.raises(R.RavError):
        bt64.apply_tile(4)
    assert bt64.apply_tile(0) == [(0, 1)] * (max(m.nlev for m in mgs64) - 1)


def test_misaligned_vectors_are_rejected():
    """With nrhs >= 2 the batched kernels read rows of x and b two doubles at a
    time: batch_vcycle and solve_batched refuse vectors that do not start on a
    16-byte boundary (RAV_ERR_ARG, before any launch); aligned ones still run."""
    mgs, sms, xs, bs = make_batch(SIZES[:2], 2, R.F32, seed=23)
    bt = R.Batch(mgs, sms, 2)
    buf = torch.zeros(xs[0].numel() + 1, dtype=torch.float64, device="cuda")
    shifted = buf[1:].view(xs[0].shape)
    assert shifted.data_ptr() % 16 == 8
    with pytest.raises(R.RavError):
        bt.vcycle([shifted, xs[1]], bs, 2, 2)
    with pytest.raises(R.RavError):
        bt.solve(xs, [shifted, bs[1]], tol=1e-8, maxit=3)
    x_in = [x.clone() for x in xs]
    bt.vcycle(xs, bs, 2, 2)
    assert all(not torch.equal(x, xi) for x, xi in zip(xs, x_in))
