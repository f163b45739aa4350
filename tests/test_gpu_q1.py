"""Parity of the CUDA path on the stabilised Q1-Q1 element (Sec. 2, Eq. 8;
subdomains of Sec. 3 owning exactly their vertex's DoFs) with the FP64 oracle.

Bars as for Q2-Q1: structure and patch/owner lists bit-exact; assembled values,
right-hand sides and transfers to 1e-13 relative; stored rows to 1e-11; one
FP64 smoothing step and a V-cycle to 1e-12 / 1e-11; per-cycle convergence
factors within 2 %; factored reduced storage within fp32 roundoff of the
oracle's step.
"""
import numpy as np
import pytest

import oracle as O
from paper_2103_10127_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

import paper_2103_10127_gb300 as R  # noqa: E402

BETA = 0.02
OMEGA = 0.66


def make_pair(dim, N, nlev, graded=False, nblobs=0, bc=O.BC_CAVITY, eta0=1.0, seed=21, s_max=2.0, beta=BETA):
    coords = inputs.graded_coordinates(N, 4.0, dim) if graded else None
    blobs = inputs.viscosity_blobs(seed, k=nblobs, s_max=s_max) if nblobs else None
    mg = R.Multigrid(dim, N, nlev, coords=coords, eta0=eta0, blobs=blobs, bc=bc, element=R.ELEM_Q1Q1, beta=beta)
    orc = O.Oracle(dim, N, nlev, coords=coords, eta0=eta0, blobs=blobs, bc=bc, element=O.ELEM_Q1Q1, beta=beta)
    return mg, orc


CASES = [
    dict(dim=2, N=8, nlev=3),
    dict(dim=2, N=12, nlev=2, graded=True, nblobs=6, bc=O.BC_NOSLIP),
    dict(dim=3, N=4, nlev=2, nblobs=4),
    dict(dim=3, N=6, nlev=2, graded=True, nblobs=5, bc=O.BC_NOSLIP),
]
IDS = ["2d-8-cavity", "2d-12-graded-blobs", "3d-4-blobs", "3d-6-graded-blobs"]


def cpu(t):
    return t.detach().cpu().numpy()


def gpu(a):
    return torch.from_numpy(np.ascontiguousarray(a, np.float64)).cuda()


def rel(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


@pytest.mark.parametrize("case", CASES, ids=IDS)
def test_assembled_operators_match(case):
    mg, orc = make_pair(**case)
    for lev in range(case["nlev"]):
        assert mg.counts(lev)["n"] == orc.sizes(lev)["n"]
        rp, ci, va = (cpu(t) for t in mg.csr(lev))
        orp, oci, ova = orc.csr(lev)
        assert np.array_equal(rp, orp)
        assert np.array_equal(ci.astype(np.int64), oci)
        assert np.abs(va - ova).max() <= 1e-13 * np.abs(ova).max()


@pytest.mark.parametrize("case", CASES, ids=IDS)
def test_rhs_and_initial_guess_match(case):
    mg, orc = make_pair(**case)
    forcings = [O.F_NONE, O.F_QUADRATIC] + ([O.F_PSI] if case["dim"] == 2 else [O.F_SINKER])
    for f in forcings:
        b = cpu(mg.rhs(f))
        ob = orc.rhs(f)
        assert np.abs(b - ob).max() <= 1e-13 * max(np.abs(ob).max(), 1.0), f
    assert np.array_equal(cpu(mg.initial_guess()), orc.initial_guess())


@pytest.mark.parametrize("case", CASES, ids=IDS)
def test_patch_lists_and_owners_bit_exact(case):
    mg, orc = make_pair(**case)
    sm = R.Smoother(mg, R.RAV, R.F64, OMEGA)
    for lev in range(1, case["nlev"]):
        orc.build_patches(lev)
        off, dofs, own = (cpu(t).astype(np.int64) for t in sm.patches(lev))
        ooff, odofs, oown = orc.patches(lev)
        assert np.array_equal(off, ooff)
        assert np.array_equal(dofs, odofs)
        assert np.array_equal(own, oown)
        assert sm.patch_counts(lev) == (len(ooff) - 1, len(odofs))


@pytest.mark.parametrize("case", CASES, ids=IDS)
def test_stored_inverse_rows_match(case):
    mg, orc = make_pair(**case)
    sm = R.Smoother(mg, R.RAV, R.F64, OMEGA)
    orc.setup_smoother(O.RAV, OMEGA)
    lev = case["nlev"] - 1
    npatch = mg.counts(lev)["n_p"]
    got = cpu(sm.inverse_rows(lev, 0, npatch))
    for p in range(npatch):
        want = orc.inverse(lev, p)
        g = got[p, : want.shape[0], : want.shape[1]]
        assert np.abs(g - want).max() <= 1e-11 * np.abs(want).max(), p
        assert not got[p, want.shape[0]:, :].any() and not got[p, :, want.shape[1]:].any()


@pytest.mark.parametrize("case", CASES, ids=IDS)
def test_fp64_smoothing_steps_match(case):
    mg, orc = make_pair(**case)
    sm = R.Smoother(mg, R.RAV, R.F64, OMEGA)
    orc.setup_smoother(O.RAV, OMEGA)
    rng = np.random.default_rng(3)
    for lev in range(1, case["nlev"]):
        n = mg.n(lev)
        x, b = rng.standard_normal(n), rng.standard_normal(n)
        want = orc.smooth(lev, x, b, 2)
        xg = gpu(x)
        sm.smooth(lev, xg, gpu(b), 2)
        got = cpu(xg)
        assert rel(got, want) <= 1e-12
        assert np.linalg.norm(got - want) <= 1e-11 * np.linalg.norm(want - x)


@pytest.mark.parametrize("case", [CASES[1], CASES[3]], ids=[IDS[1], IDS[3]])
def test_per_patch_damping_is_applied(case):
    mg, orc = make_pair(**case)
    sm = R.Smoother(mg, R.RAV, R.F64, OMEGA)
    orc.setup_smoother(O.RAV, OMEGA)
    lev = case["nlev"] - 1
    w = (0.2 + 0.9 * inputs.uniform(8, mg.counts(lev)["n_p"])).astype(np.float32)
    sm.set_omega(lev, torch.from_numpy(w).cuda())
    orc.set_omega(lev, w.astype(np.float64))
    rng = np.random.default_rng(4)
    n = mg.n(lev)
    x, b = rng.standard_normal(n), rng.standard_normal(n)
    xg = gpu(x)
    sm.smooth(lev, xg, gpu(b), 1)
    assert rel(cpu(xg), orc.smooth(lev, x, b, 1)) <= 1e-12


@pytest.mark.parametrize("case", CASES, ids=IDS)
def test_residual_transfers_and_coarse_solve_match(case):
    mg, orc = make_pair(**case)
    rng = np.random.default_rng(5)
    for lev in range(case["nlev"]):
        n = mg.n(lev)
        x, b = rng.standard_normal(n), rng.standard_normal(n)
        r, nrm = mg.residual(lev, gpu(x), gpu(b), norm=True)
        want = orc.residual(lev, x, b)
        assert rel(cpu(r), want) <= 1e-13
        assert abs(nrm - np.linalg.norm(want)) <= 1e-13 * np.linalg.norm(want)
        if lev > 0:
            bc = cpu(mg.restrict(lev, gpu(want)))
            assert rel(bc, orc.restrict(lev, want)) <= 1e-14
            xc = rng.standard_normal(mg.n(lev - 1))
            xf = rng.standard_normal(n)
            got = cpu(mg.prolong_add(lev, gpu(xc), gpu(xf)))
            assert rel(got, orc.prolong_add(lev, xc, xf)) <= 1e-14
    b0 = rng.standard_normal(mg.n(0))
    assert rel(cpu(mg.coarse_solve(gpu(b0))), orc.coarse_solve(b0)) <= 1e-11


@pytest.mark.parametrize("prec", [R.F32_FACT, R.BF16_FACT], ids=["f32-factored", "bf16-factored"])
@pytest.mark.parametrize("case", [CASES[1], CASES[2]], ids=[IDS[1], IDS[2]])
def test_factored_reduced_storage_matches_the_oracle(case, prec):
    """Rows rebuilt from the rounded K^{-1} centre row, w and 1/s equal the
    oracle's rebuild (one fp32 unit of slack for fp64 differences of the two
    factorisations), and one step with fp32 accumulation stays within fp32
    roundoff of the oracle's step."""
    mg, orc = make_pair(**case)
    lev = case["nlev"] - 1
    npatch = mg.counts(lev)["n_p"]
    sq = R.Smoother(mg, R.RAV, prec, OMEGA)
    orc.setup_smoother(O.RAV, OMEGA, {R.F32_FACT: O.F32_FACT, R.BF16_FACT: O.BF16_FACT}[prec])
    got = cpu(sq.inverse_rows(lev, 0, npatch))
    for p in range(npatch):
        want, _ = orc.inverse(lev, p, quantised=True)
        g = got[p, : want.shape[0], : want.shape[1]]
        assert np.abs(g - want).max() <= 2.0 ** -22 * np.abs(want).max(), p
    rng = np.random.default_rng(17)
    n = mg.n(lev)
    x, b = rng.standard_normal(n), rng.standard_normal(n)
    xg = gpu(x)
    sq.smooth(lev, xg, gpu(b), 1)
    d = cpu(xg) - x
    want = orc.smooth(lev, x, b, 1) - x
    assert np.linalg.norm(d - want) <= 1e-5 * np.linalg.norm(want)


@pytest.mark.parametrize("case", CASES, ids=IDS)
@pytest.mark.parametrize("kind,omega", [(R.AV, 0.1), (R.MV_COLOURED, OMEGA)], ids=["av", "mv"])
def test_comparator_inverses_and_steps_match(case, kind, omega):
    """AV (Eq. 12) and coloured MV (Eqs. 11, 15) on Q1-Q1: the full stored
    L_i^{-1} to 1e-11 and two smoothing steps to 1e-12 against the oracle (MV in
    the same 4^d colour order)."""
    mg, orc = make_pair(**case)
    sm = R.Smoother(mg, kind, R.F64, omega)
    orc.setup_smoother(O.AV if kind == R.AV else O.MV_COLOURED, omega)
    lev = case["nlev"] - 1
    npatch = mg.counts(lev)["n_p"]
    got = cpu(sm.inverse_rows(lev, 0, npatch))
    for p in range(npatch):
        want = orc.inverse(lev, p)
        g = got[p, : want.shape[0], : want.shape[1]]
        assert np.abs(g - want).max() <= 1e-11 * np.abs(want).max(), p
        assert not got[p, want.shape[0]:, :].any() and not got[p, :, want.shape[1]:].any()
    rng = np.random.default_rng(31)
    for lv in range(1, case["nlev"]):
        n = mg.n(lv)
        x, b = rng.standard_normal(n), rng.standard_normal(n)
        want = orc.smooth(lv, x, b, 2)
        xg = gpu(x)
        sm.smooth(lv, xg, gpu(b), 2)
        assert rel(cpu(xg), want) <= 1e-12


@pytest.mark.parametrize("nu", [1, 3])
@pytest.mark.parametrize("kind,omega", [(R.RAV, OMEGA), (R.AV, 0.1), (R.MV_COLOURED, OMEGA)],
                         ids=["rav", "av", "mv"])
def test_smoothing_steps_study_matches_the_oracle(kind, omega, nu):
    """The smoothing-steps comparison (Sec. 4.2) on the paper's element: a 16^2
    Q1-Q1 cavity, 3 levels, V(nu, nu) to 1e-8 with every smoother: equal cycle
    counts and per-cycle factors within 2 % of the oracle."""
    mg, orc = make_pair(2, 16, 3)
    sm = R.Smoother(mg, kind, R.F64, omega)
    orc.setup_smoother({R.RAV: O.RAV, R.AV: O.AV, R.MV_COLOURED: O.MV_COLOURED}[kind], omega)
    it, hist, rc = mg.solve(sm, mg.initial_guess(), mg.rhs(R.F_NONE), tol=1e-8, maxit=300, nu_pre=nu,
                            nu_post=nu)
    _, oit, ohist = orc.solve(orc.initial_guess(), orc.rhs(O.F_NONE), tol=1e-8, maxit=300, nu1=nu, nu2=nu)
    assert rc == 0 and it == oit
    fac, ofac = hist[1:] / hist[:-1], ohist[1:] / ohist[:-1]
    assert np.all(np.abs(fac / ofac - 1.0) <= 0.02)


@pytest.mark.parametrize("case", CASES, ids=IDS)
def test_dense_fp64_rows_match(case):
    """The paper's storage (Sec. 4.3), the owned rows of L_i^{-1} in fp64: the
    stored rows to 1e-11 and one step to 1e-12 against the oracle."""
    mg, orc = make_pair(**case)
    sm = R.Smoother(mg, R.RAV, R.F64_ROWS, OMEGA)
    orc.setup_smoother(O.RAV, OMEGA)
    lev = case["nlev"] - 1
    npatch = mg.counts(lev)["n_p"]
    got = cpu(sm.inverse_rows(lev, 0, npatch))
    for p in range(npatch):
        want = orc.inverse(lev, p)
        g = got[p, : want.shape[0], : want.shape[1]]
        assert np.abs(g - want).max() <= 1e-11 * np.abs(want).max(), p
    rng = np.random.default_rng(19)
    n = mg.n(lev)
    x, b = rng.standard_normal(n), rng.standard_normal(n)
    xg = gpu(x)
    sm.smooth(lev, xg, gpu(b), 1)
    assert rel(cpu(xg), orc.smooth(lev, x, b, 1)) <= 1e-12


@pytest.mark.parametrize("prec", [R.F32, R.BF16, R.FP8])
@pytest.mark.parametrize("case", [CASES[1], CASES[2]], ids=[IDS[1], IDS[2]])
def test_reduced_precision_row_codes_and_step(case, prec):
    """Reduced-precision rows: the codes equal the oracle's rounding of the same
    fp64 rows (bit-exact, fp8 with its fp32 row scale), and one step (fp32
    accumulation) is within the format's error of the fp64 step and close to
    the oracle's emulation of the same format."""
    mg, orc = make_pair(**case)
    lev = case["nlev"] - 1
    npatch = mg.counts(lev)["n_p"]
    s64 = R.Smoother(mg, R.RAV, R.F64_ROWS, OMEGA)
    sq = R.Smoother(mg, R.RAV, prec, OMEGA)
    rows64 = cpu(s64.inverse_rows(lev, 0, npatch))
    rowsq = cpu(sq.inverse_rows(lev, 0, npatch))
    if prec == R.FP8:
        m = np.abs(rows64).max(axis=2, keepdims=True)
        sc = np.where(m == 0, 1.0, (m / 448.0).astype(np.float32).astype(np.float64))
    else:
        sc = np.ones_like(rows64[..., :1])
    assert np.array_equal(rowsq, O.round_format(prec, rows64 / sc) * sc)
    orc.setup_smoother(O.RAV, OMEGA, prec)
    rng = np.random.default_rng(7)
    n = mg.n(lev)
    x, b = rng.standard_normal(n), rng.standard_normal(n)
    xg = gpu(x)
    sq.smooth(lev, xg, gpu(b), 1)
    got = cpu(xg) - x
    want_q = orc.smooth(lev, x, b, 1) - x
    x64 = gpu(x)
    s64.smooth(lev, x64, gpu(b), 1)
    d64 = cpu(x64) - x
    fmt_err = np.linalg.norm(want_q - d64) / np.linalg.norm(d64)
    assert np.linalg.norm(got - want_q) <= 1e-5 * np.linalg.norm(d64) + 0.05 * fmt_err * np.linalg.norm(d64)
    assert fmt_err <= {R.F32: 1e-6, R.BF16: 2e-2, R.FP8: 2e-1}[prec]


@pytest.mark.parametrize("case", CASES[:3], ids=IDS[:3])
def test_vcycle_matches(case):
    mg, orc = make_pair(**case)
    sm = R.Smoother(mg, R.RAV, R.F64, OMEGA)
    orc.setup_smoother(O.RAV, OMEGA)
    rng = np.random.default_rng(6)
    n = mg.n()
    x, b = rng.standard_normal(n), rng.standard_normal(n)
    want = orc.vcycle(x, b, 2, 2)
    xg = gpu(x)
    mg.vcycle(sm, xg, gpu(b), 2, 2)
    assert rel(cpu(xg), want) <= 1e-11


def test_cavity_convergence_factors_within_two_percent():
    """32x32 Q1-Q1 lid-driven cavity, 4 levels, RAV(0.66), V(2,2), to 1e-8."""
    mg, orc = make_pair(2, 32, 4)
    sm = R.Smoother(mg, R.RAV, R.F64, OMEGA)
    orc.setup_smoother(O.RAV, OMEGA)
    x = mg.initial_guess()
    it, hist, rc = mg.solve(sm, x, mg.rhs(R.F_NONE), tol=1e-8, maxit=100)
    ox, oit, ohist = orc.solve(orc.initial_guess(), orc.rhs(O.F_NONE), tol=1e-8, maxit=100)
    assert rc == 0 and it == oit and it <= 20
    fac, ofac = hist[1:] / hist[:-1], ohist[1:] / ohist[:-1]
    assert np.all(np.abs(fac / ofac - 1.0) <= 0.02)
    assert rel(cpu(x), ox) <= 1e-6


@pytest.mark.parametrize("prec", [R.F64, R.F32_FACT, R.BF16_FACT, R.F64_ROWS, R.F32, R.BF16, R.FP8],
                         ids=["f64", "f32", "bf16", "f64-rows", "f32-rows", "bf16-rows", "fp8-rows"])
def test_fgmres_reaches_the_fp64_tolerance(prec):
    """3-D Q1-Q1 with viscosity blobs: FGMRES preconditioned by RAV V-cycles
    reaches 1e-8 in fp64 with every factored storage; the fp64 run matches the
    oracle's FGMRES history."""
    mg, orc = make_pair(3, 8, 2, nblobs=10, s_max=2.0, bc=O.BC_NOSLIP)
    sm = R.Smoother(mg, R.RAV, prec, OMEGA)
    x = mg.initial_guess()
    b = mg.rhs(R.F_SINKER)
    it, hist, rc = mg.solve(sm, x, b, tol=1e-8, maxit=200, outer=1)
    assert rc == 0 and hist[-1] <= 1e-8
    _, nrm = mg.residual(1, x, b, norm=True)
    _, nrm0 = mg.residual(1, mg.initial_guess(), b, norm=True)
    assert nrm <= 1.01e-8 * nrm0
    if prec == R.F64:
        orc.setup_smoother(O.RAV, OMEGA)
        _, oit, ohist = orc.fgmres(orc.initial_guess(), orc.rhs(O.F_SINKER), tol=1e-8, maxit=200)
        assert abs(it - oit) <= 1
        k = min(it, oit)
        assert np.all(np.abs(hist[1:k] / ohist[1:k] - 1.0) <= 1e-4)


def test_unsupported_combinations_are_rejected():
    """Q1-Q1 AV/MV take fp64 only; a batch holds one element and dense-row
    storage; the apply has no split."""
    mg, _ = make_pair(2, 8, 2)
    for kind, prec in ((R.AV, R.F32), (R.MV_COLOURED, R.BF16_FACT), (R.AV, R.FP8)):
        with pytest.raises(R.RavError):
            R.Smoother(mg, kind, prec, 0.5)
    sm = R.Smoother(mg, R.RAV, R.F64, OMEGA)
    assert sm.apply_split(1) == 1
    assert sm.apply_split(1, 1) == 1
    with pytest.raises(R.RavError):
        sm.apply_split(1, 2)
    with pytest.raises(R.RavError):
        R.Batch([mg], [sm], 1)  # factored storage: the batch takes dense rows
    mg2 = R.Multigrid(2, 8, 2, bc=R.BC_CAVITY)
    with pytest.raises(R.RavError):
        R.Batch([mg, mg2], [R.Smoother(mg, R.RAV, R.F32, OMEGA), R.Smoother(mg2, R.RAV, R.F32, 0.5)], 1)


@pytest.mark.parametrize("dim,N,per_patch", [(2, 12, False), (3, 6, True)])
def test_learned_damping_labels_match_the_oracle(dim, N, per_patch):
    """Line-search labels of the learned damping on Q1-Q1 subdomains (graded
    blob problems; in 3-D gathered at non-uniform current weights) equal the
    oracle's coordinate minimisers."""
    from paper_2103_10127_gb300 import _capi, learned
    mg, orc = make_pair(dim, N, 2, graded=True, nblobs=5, bc=O.BC_NOSLIP, s_max=2.0, seed=12)
    sm = R.Smoother(mg, R.RAV, R.F64, OMEGA)
    npatch = mg.counts(1)["n_p"]
    w = None
    if per_patch:
        w = (0.2 + 0.8 * inputs.uniform(13, npatch)).astype(np.float32)
        sm.set_omega(1, torch.from_numpy(w).cuda())
    orc.build_patches(1)
    n = mg.n(1)
    x, b = inputs.normal(14, n), inputs.normal(15, n)
    lib = _capi.load()
    assert lib.rav_label_collection(sm.h, 1) == 0
    sm.smooth(1, torch.from_numpy(x).cuda(), torch.from_numpy(b).cuda(), 1)
    y = torch.empty(npatch, dtype=torch.float32, device="cuda")
    assert lib.rav_read_labels(sm.h, 1, learned._p(y), learned._s()) == 0
    assert lib.rav_label_collection(sm.h, 0) == 0
    om = np.full(npatch, OMEGA) if w is None else w.astype(np.float64)
    want = orc.labels(1, orc.residual(1, x, b), omega=om)
    assert np.abs(y.cpu().numpy() - want).max() <= 1e-6


def test_learned_damping_features_on_q1_subdomains():
    """The cell-based features (viscosity, aspect, level, diagonal) equal those
    of the Q2-Q1 hierarchy on the same grid (the same cells surround a vertex);
    the size feature is n_i / (3^d d + 1) from the subdomain lists and the
    Dirichlet feature the boundary share of the in-domain box vertices."""
    from paper_2103_10127_gb300 import learned
    N = 8
    coords = inputs.graded_coordinates(N, 4.0, 2)
    blobs = inputs.viscosity_blobs(11, k=3, s_max=3.0)
    mg1 = R.Multigrid(2, N, 2, coords=coords, blobs=blobs, bc=R.BC_NOSLIP, element=R.ELEM_Q1Q1, beta=BETA)
    mg2 = R.Multigrid(2, N, 2, coords=coords, blobs=blobs, bc=R.BC_NOSLIP)
    s1, s2 = R.Smoother(mg1, R.RAV, R.F64, OMEGA), R.Smoother(mg2, R.RAV, R.F64, 0.5)
    f1, f2 = learned.features(s1, 1).cpu().numpy(), learned.features(s2, 1).cpu().numpy()
    keep = [0, 1, 2, 3, 4, 7]
    assert np.array_equal(f1[:, keep], f2[:, keep])
    off, _, _ = (cpu(t) for t in s1.patches(1))
    assert np.allclose(f1[:, 5], np.diff(off) / (2 * 9 + 1), rtol=1e-6)
    for p in range((N + 1) ** 2):
        v = (p % (N + 1), p // (N + 1))
        box = [(v[0] - 1 + a, v[1] - 1 + c) for a in range(3) for c in range(3)]
        inside = [(i, j) for i, j in box if 0 <= i <= N and 0 <= j <= N]
        bnd = [(i, j) for i, j in inside if i in (0, N) or j in (0, N)]
        assert abs(f1[p, 6] - len(bnd) / len(inside)) <= 1e-6, p


@pytest.mark.slow
def test_full_size_1024_sampled_parity():
    """1024^2 Q1-Q1 (3,151,875 DoFs), the benchmark's launch configuration:
    the whole assembled fine operator, and one RAV step at sampled subdomains
    (boundary corners and 60 random vertices) against rows the oracle
    factorises one by one."""
    N, nlev = 1024, 8
    mg = R.Multigrid(2, N, nlev, bc=R.BC_NOSLIP, element=R.ELEM_Q1Q1, beta=BETA)
    orc = O.Oracle(2, N, 1, bc=O.BC_NOSLIP, element=O.ELEM_Q1Q1, beta=BETA)
    rp, ci, va = (cpu(t) for t in mg.csr(nlev - 1))
    orp, oci, ova = orc.csr(0)
    assert np.array_equal(rp, orp) and np.array_equal(ci.astype(np.int64), oci)
    assert np.abs(va - ova).max() <= 1e-13 * np.abs(ova).max()
    del oci, ova
    sm = R.Smoother(mg, R.RAV, R.F64, OMEGA)
    rng = np.random.default_rng(8)
    n = mg.n()
    x, b = rng.standard_normal(n), rng.standard_normal(n)
    xg = gpu(x)
    sm.smooth(nlev - 1, xg, gpu(b), 1)
    got = cpu(xg)
    r = orc.residual(0, x, b)
    orc.build_patches(0)
    off, dofs, own = orc.patches(0)
    samples = np.concatenate([[0, N, N * (N + 1), (N + 1) ** 2 - 1],
                              (inputs.uniform(9, 60) * (N + 1) ** 2).astype(np.int64)])
    for p in samples:
        s = dofs[off[p]:off[p + 1]]
        mine = s[own[s] == p]
        rows = orc.patch_rows(0, int(p))[: len(mine) * len(s)].reshape(len(mine), len(s))
        want = x[mine] + OMEGA * rows @ r[s]
        assert np.abs(got[mine] - want).max() <= 1e-12 * max(np.abs(want).max(), 1.0), p


# --------------------------------------------------------------------------- edge cases
@pytest.mark.parametrize("dim,N", [(2, 4), (3, 2)])
def test_single_level_cycle_is_the_exact_coarse_solve(dim, N):
    """One Q1-Q1 level: the V-cycle is the bordered LU solve (residual at
    roundoff after one cycle, equal to the oracle's coarse solve)."""
    mg, orc = make_pair(dim, N, 1, bc=O.BC_QUADRATIC)
    sm = R.Smoother(mg, R.RAV, R.F64, OMEGA)
    b = mg.rhs(R.F_QUADRATIC)
    x = mg.initial_guess()
    mg.vcycle(sm, x, b, 2, 2)
    _, r = mg.residual(0, x, b, norm=True)
    _, r0 = mg.residual(0, mg.initial_guess(), b, norm=True)
    assert r <= 1e-11 * r0
    ob, ox = orc.rhs(O.F_QUADRATIC), orc.initial_guess()
    want = ox + orc.coarse_solve(orc.residual(0, ox, ob))
    nu = mg.counts(0)["n_u"]
    assert np.abs(cpu(x)[:nu] - want[:nu]).max() <= 1e-10 * max(1.0, np.abs(want[:nu]).max())
    it, _, rc = mg.solve(sm, mg.initial_guess(), b, tol=1e-8, maxit=5)
    assert rc == 0 and it == 1


def test_zero_problem_needs_no_iteration():
    mg, _ = make_pair(2, 8, 2, bc=O.BC_NOSLIP)
    sm = R.Smoother(mg, R.RAV, R.F64, OMEGA)
    x = mg.initial_guess()
    for outer in (0, 1):
        it, _, rc = mg.solve(sm, x, mg.rhs(R.F_NONE), tol=1e-8, maxit=10, outer=outer)
        assert rc == 0 and it == 0
    assert not cpu(x).any()


@pytest.mark.parametrize("kind,prec", [(R.RAV, R.F64), (R.RAV, R.F32_FACT), (R.RAV, R.BF16_FACT), (R.AV, R.F64),
                                       (R.MV_COLOURED, R.F64)], ids=["rav", "rav-f32", "rav-bf16", "av", "mv"])
def test_zero_damping_zero_steps_and_zero_residual_leave_x_unchanged(kind, prec):
    mg, _ = make_pair(2, 8, 2, bc=O.BC_CAVITY)
    rng = np.random.default_rng(1)
    n = mg.n()
    x0, b = rng.standard_normal(n), rng.standard_normal(n)
    x = gpu(x0)
    R.Smoother(mg, kind, prec, 0.0).smooth(1, x, gpu(b), 3)
    assert np.array_equal(cpu(x), x0)
    sm = R.Smoother(mg, kind, prec, OMEGA)
    sm.smooth(1, x, gpu(b), 0)
    assert np.array_equal(cpu(x), x0)
    if kind != R.MV_COLOURED:  # MV has no apply of a given residual
        sm.apply(1, torch.zeros(n, dtype=torch.float64, device="cuda"), x)
        assert np.array_equal(cpu(x), x0)


@pytest.mark.parametrize("dim,N,nlev", [(2, 4, 2), (3, 4, 2), (2, 6, 2)])
def test_smallest_hierarchies_match_the_oracle(dim, N, nlev):
    """Coarsest Q1-Q1 grids of 2 or 3 cells per axis (one or four free vertices)."""
    mg, orc = make_pair(dim, N, nlev, graded=True, bc=O.BC_NOSLIP)
    sm = R.Smoother(mg, R.RAV, R.F64, OMEGA)
    orc.setup_smoother(O.RAV, OMEGA)
    rng = np.random.default_rng(3)
    n = mg.n()
    x, b = rng.standard_normal(n), rng.standard_normal(n)
    want = orc.vcycle(x, b, 2, 2)
    xg = gpu(x)
    mg.vcycle(sm, xg, gpu(b), 2, 2)
    assert rel(cpu(xg), want) <= 1e-11


@pytest.mark.slow
def test_full_size_64cube_sampled_parity():
    """3-D 64^3 Q1-Q1 with 20 seeded blobs (1,098,500 DoFs), the 3-D Q1-Q1
    benchmark's launch configuration: the fine operator in full, and one RAV
    step at sampled subdomains against rows the oracle factorises one by one."""
    N, nlev = 64, 5
    blobs = inputs.viscosity_blobs(inputs.BASE_SEED, k=20, s_max=2.0)
    mg = R.Multigrid(3, N, nlev, blobs=blobs, bc=R.BC_NOSLIP, element=R.ELEM_Q1Q1, beta=BETA)
    orc = O.Oracle(3, N, 1, blobs=blobs, bc=O.BC_NOSLIP, element=O.ELEM_Q1Q1, beta=BETA)
    rp, ci, va = (cpu(t) for t in mg.csr(nlev - 1))
    orp, oci, ova = orc.csr(0)
    assert np.array_equal(rp, orp) and np.array_equal(ci.astype(np.int64), oci)
    assert np.abs(va - ova).max() <= 1e-13 * np.abs(ova).max()
    del ci, va, oci, ova
    sm = R.Smoother(mg, R.RAV, R.F64, OMEGA)
    rng = np.random.default_rng(44)
    n = mg.n()
    x, b = rng.standard_normal(n), rng.standard_normal(n)
    xg = gpu(x)
    sm.smooth(nlev - 1, xg, gpu(b), 1)
    got = cpu(xg)
    r = orc.residual(0, x, b)
    orc.build_patches(0)
    off, dofs, own = orc.patches(0)
    samples = np.concatenate([[0, N, (N + 1) ** 2 - 1, (N + 1) ** 3 - 1],
                              (inputs.uniform(45, 60) * (N + 1) ** 3).astype(np.int64)])
    for p in samples:
        s = dofs[off[p]:off[p + 1]]
        mine = s[own[s] == p]
        rows = orc.patch_rows(0, int(p))[: len(mine) * len(s)].reshape(len(mine), len(s))
        want = x[mine] + OMEGA * rows @ r[s]
        assert np.abs(got[mine] - want).max() <= 1e-12 * max(np.abs(want).max(), 1.0), p


# --------------------------------------------------------------------------- batched
def _free_velocity_q1(dim, N):
    idx = np.indices((N + 1,) * dim).reshape(dim, -1)[::-1]  # axis 0 fastest
    inner = np.all((idx > 0) & (idx < N), axis=0)
    return np.concatenate([np.repeat(inner, dim), np.zeros((N + 1) ** dim, bool)])


def _q1_batch(specs, nrhs, prec, seed):
    """specs: (dim, N, levels, blobs); lid values plus iid N(0,1) forcing on
    the free velocity rows per right-hand side."""
    mgs, sms, xs, bs = [], [], [], []
    for i, (dim, N, nlev, blobs) in enumerate(specs):
        mg = R.Multigrid(dim, N, nlev, blobs=blobs, bc=R.BC_CAVITY, element=R.ELEM_Q1Q1, beta=BETA)
        sm = R.Smoother(mg, R.RAV, prec, OMEGA)
        m = _free_velocity_q1(dim, N)
        b0 = mg.rhs(R.F_NONE).cpu().numpy()
        cols = []
        for k in range(nrhs):
            bk = b0.copy()
            bk[m] += inputs.normal(1000 * seed + 10 * i + k, int(m.sum()))
            cols.append(bk)
        x0 = mg.initial_guess().cpu().numpy()
        mgs.append(mg)
        sms.append(sm)
        xs.append(torch.from_numpy(np.ascontiguousarray(np.repeat(x0[:, None], nrhs, axis=1))).cuda())
        bs.append(torch.from_numpy(np.ascontiguousarray(np.stack(cols, axis=1))).cuda())
    return mgs, sms, xs, bs


@pytest.mark.parametrize("prec", [R.F32, R.F64_ROWS], ids=["f32-rows", "f64-rows"])
@pytest.mark.parametrize("dim", [2, 3])
def test_batched_q1_cycles_equal_single_problem_cycles_bitwise(dim, prec):
    """Uneven Q1-Q1 problems (2-D 16^2..32^2 of 3-4 levels; 3-D 8^3 and 16^3 with
    blobs) advanced together: two batched V(2,2) cycles equal, bit for bit, two
    single-problem cycles of every right-hand side."""
    if dim == 2:
        specs = [(2, N, inputs.levels_for(N), None) for N in (16, 24, 32, 20)]
        nrhs = 4
    else:
        specs = [(3, 8, 2, inputs.viscosity_blobs(40, k=4, s_max=2.0)),
                 (3, 16, 3, inputs.viscosity_blobs(41, k=4, s_max=2.0))]
        nrhs = 2
    mgs, sms, xs, bs = _q1_batch(specs, nrhs, prec, seed=dim)
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


def test_batched_q1_cycle_matches_the_oracle_and_solves():
    """One batched Q1-Q1 V-cycle (fp64 rows) against the oracle's, and a batched
    solve (fp32 rows) reaching 1e-8 in the cycles of the single solves."""
    specs = [(2, 16, 3, None), (2, 24, 2, None)]
    mgs, sms, xs, bs = _q1_batch(specs, 2, R.F64_ROWS, seed=3)
    bt = R.Batch(mgs, sms, 2)
    x_in = [x.cpu().numpy() for x in xs]
    bt.vcycle(xs, bs, 2, 2)
    for p, (_, N, nlev, _) in enumerate(specs):
        orc = O.Oracle(2, N, nlev, bc=O.BC_CAVITY, element=O.ELEM_Q1Q1, beta=BETA)
        orc.setup_smoother(O.RAV, OMEGA)
        for k in range(2):
            want = orc.vcycle(x_in[p][:, k], bs[p][:, k].cpu().numpy(), 2, 2)
            assert rel(xs[p][:, k].cpu().numpy(), want) <= 1e-11
    mgs, sms, xs, bs = _q1_batch(specs + [(2, 32, 4, None)], 2, R.F32, seed=5)
    bt = R.Batch(mgs, sms, 2)
    x_in = [x.clone() for x in xs]
    it, ratios, rc = bt.solve(xs, bs, tol=1e-8, maxit=100)
    assert rc == 0 and np.all(it > 0) and np.all(ratios <= 1e-8)
    for p, (mg, sm) in enumerate(zip(mgs, sms)):
        for k in range(2):
            its, _, rcs = mg.solve(sm, x_in[p][:, k].contiguous(), bs[p][:, k].contiguous(), tol=1e-8, maxit=100)
            assert rcs == 0 and its == it[p, k]


# --------------------------------------------------------------------------- fused smoothing
@pytest.mark.parametrize("case", CASES, ids=IDS)
def test_fused_smoothing_matches_two_kernel_steps_and_the_oracle(case):
    """The fused residual + apply step (one kernel per step, tile halos) gives
    the two-kernel steps to rounding and the oracle's steps to 1e-12, for an
    odd and an even number of steps; a V-cycle with it matches the oracle's."""
    mg, orc = make_pair(**case)
    sm = R.Smoother(mg, R.RAV, R.F64, OMEGA)
    orc.setup_smoother(O.RAV, OMEGA)
    rng = np.random.default_rng(37)
    lev = case["nlev"] - 1
    n = mg.n(lev)
    x, b = rng.standard_normal(n), rng.standard_normal(n)
    ref = {}
    for steps in (1, 2, 3):
        xg = gpu(x)
        sm.smooth(lev, xg, gpu(b), steps)
        ref[steps] = cpu(xg)
    sm.fused(True)
    for steps in (1, 2, 3):
        xg = gpu(x)
        sm.smooth(lev, xg, gpu(b), steps)
        got = cpu(xg)
        assert rel(got, ref[steps]) <= 1e-13, steps
        assert rel(got, orc.smooth(lev, x, b, steps)) <= 1e-12, steps
    if case["nlev"] > 2:
        xn = rng.standard_normal(mg.n())
        bn = rng.standard_normal(mg.n())
        xg = gpu(xn)
        mg.vcycle(sm, xg, gpu(bn), 2, 2)
        assert rel(cpu(xg), orc.vcycle(xn, bn, 2, 2)) <= 1e-11
    sm.fused(False)


def test_fused_smoothing_solves_like_the_two_kernel_path():
    mg, orc = make_pair(2, 32, 4)
    sm = R.Smoother(mg, R.RAV, R.F64, OMEGA)
    b = mg.rhs(R.F_NONE)
    it0, h0, rc0 = mg.solve(sm, mg.initial_guess(), b, tol=1e-8, maxit=100)
    sm.fused(True)
    it1, h1, rc1 = mg.solve(sm, mg.initial_guess(), b, tol=1e-8, maxit=100)
    assert rc0 == rc1 == 0 and it0 == it1
    assert np.all(np.abs(h1[1:] / h0[1:] - 1.0) <= 1e-6)
    for kind, prec in ((R.RAV, R.F32_FACT), (R.RAV, R.F64_ROWS), (R.AV, R.F64)):
        with pytest.raises(R.RavError):
            R.Smoother(mg, kind, prec, 0.5).fused(True)
    q2 = R.Multigrid(2, 8, 2, bc=R.BC_CAVITY)  # Q2-Q1: the factored storages only
    for kind, prec in ((R.RAV, R.F64_ROWS), (R.RAV, R.F32), (R.AV, R.F64)):
        with pytest.raises(R.RavError):
            R.Smoother(q2, kind, prec, 0.5).fused(True)
