"""Learned per-subdomain damping: GPU kernels against the oracle, and what the
trained network gains over fixed damping on a held-out problem."""
import numpy as np
import pytest

import oracle as O
from paper_2103_10127_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

import paper_2103_10127_gb300 as R  # noqa: E402
from paper_2103_10127_gb300 import learned  # noqa: E402


def _problem(dim, N, nlev, seed, s_max=4.0, aspect=8.0, nblobs=12):
    coords = inputs.graded_coordinates(N, aspect, dim) if aspect > 1 else None
    blobs = inputs.viscosity_blobs(seed, k=nblobs, s_max=s_max)
    return dict(dim=dim, N=N, n_levels=nlev, coords=coords, blobs=blobs, bc=R.BC_NOSLIP)


def test_mlp_gradient_matches_the_oracle():
    P = learned.init_params(3)
    X = torch.from_numpy(inputs.normal(4, 8 * 300).reshape(300, 8).astype(np.float32)).cuda()
    y = torch.from_numpy((1.5 * inputs.uniform(5, 300)).astype(np.float32)).cuda()
    loss, g = learned.loss_grad(P, X, y)
    oloss, og = O.mlp_loss_grad(P.cpu().numpy().astype(np.float64), X.cpu().numpy(), y.cpu().numpy())
    g = g.cpu().numpy()
    assert abs(loss.item() - oloss) <= 1e-5 * oloss
    assert np.linalg.norm(g - og) <= 1e-3 * np.linalg.norm(og)
    assert np.abs(g - og).max() <= 1e-3 * np.abs(og).max()


def test_mlp_forward_matches_the_oracle_with_fp16_weights():
    P = learned.init_params(6)
    X = torch.from_numpy(inputs.normal(7, 8 * 500).reshape(500, 8).astype(np.float32)).cuda()
    got = learned.forward(P, X).cpu().numpy()
    P16 = P.half().double().cpu().numpy()
    want = O.mlp_forward(P16, X.cpu().numpy())
    assert np.abs(got - want).max() <= 2e-5


def test_labels_match_the_oracle():
    spec = _problem(2, 12, 2, seed=8, s_max=2.0, aspect=3.0, nblobs=4)
    mg = R.Multigrid(**spec)
    sm = R.Smoother(mg, R.RAV, R.F64, 0.5)
    orc = O.Oracle(2, 12, 2, coords=spec["coords"], blobs=spec["blobs"], bc=O.BC_NOSLIP)
    orc.build_patches(1)
    n = mg.n(1)
    x = inputs.normal(9, n)
    b = inputs.normal(10, n)
    from paper_2103_10127_gb300 import _capi
    lib = _capi.load()
    assert lib.rav_label_collection(sm.h, 1) == 0
    xg = torch.from_numpy(x).cuda()
    sm.smooth(1, xg, torch.from_numpy(b).cuda(), 1)
    y = torch.empty(mg.counts(1)["n_p"], dtype=torch.float32, device="cuda")
    assert lib.rav_read_labels(sm.h, 1, learned._p(y), learned._s()) == 0
    assert lib.rav_label_collection(sm.h, 0) == 0
    r = orc.residual(1, x, b)
    want = orc.labels(1, r)
    assert np.abs(y.cpu().numpy() - want).max() <= 1e-6


def test_labels_match_the_oracle_in_3d_with_per_patch_weights():
    """3-D graded blob problem, labels gathered at non-uniform current weights."""
    spec = _problem(3, 6, 2, seed=12, s_max=3.0, aspect=4.0, nblobs=5)
    mg = R.Multigrid(**spec)
    sm = R.Smoother(mg, R.RAV, R.F64, 0.5)
    npatch = mg.counts(1)["n_p"]
    w = (0.2 + 0.8 * inputs.uniform(13, npatch)).astype(np.float32)
    sm.set_omega(1, torch.from_numpy(w).cuda())
    orc = O.Oracle(3, 6, 2, coords=spec["coords"], blobs=spec["blobs"], bc=O.BC_NOSLIP)
    orc.build_patches(1)
    n = mg.n(1)
    x = inputs.normal(14, n)
    b = inputs.normal(15, n)
    from paper_2103_10127_gb300 import _capi
    lib = _capi.load()
    assert lib.rav_label_collection(sm.h, 1) == 0
    sm.smooth(1, torch.from_numpy(x).cuda(), torch.from_numpy(b).cuda(), 1)
    y = torch.empty(npatch, dtype=torch.float32, device="cuda")
    assert lib.rav_read_labels(sm.h, 1, learned._p(y), learned._s()) == 0
    assert lib.rav_label_collection(sm.h, 0) == 0
    want = orc.labels(1, orc.residual(1, x, b), omega=w.astype(np.float64))
    assert np.abs(y.cpu().numpy() - want).max() <= 1e-6


@pytest.mark.parametrize("dim,N,nlev,elem", [(2, 8, 2, R.ELEM_Q2Q1), (3, 6, 2, R.ELEM_Q2Q1), (2, 8, 3, R.ELEM_Q1Q1)],
                         ids=["q2q1-2d", "q2q1-3d", "q1q1-2d"])
def test_features_match_the_oracle(dim, N, nlev, elem):
    """Every feature of every subdomain on every smoothed level, graded cells
    and blob viscosity, against the oracle's features (pinned on CPU by closed
    forms); the GPU evaluates them in fp64 and stores fp32."""
    spec = _problem(dim, N, nlev, seed=11, s_max=3.0, aspect=4.0, nblobs=3)
    spec.update(element=elem, beta=0.02)
    mg = R.Multigrid(**spec)
    sm = R.Smoother(mg, R.RAV, R.F64, 0.5)
    orc = O.Oracle(dim, N, nlev, coords=spec["coords"], blobs=spec["blobs"], bc=O.BC_NOSLIP, element=elem,
                   beta=0.02)
    for lev in range(1, nlev):
        f = learned.features(sm, lev).cpu().numpy()
        want = orc.patch_features(lev)
        assert f.shape == want.shape
        assert np.abs(f - want).max() <= 1e-6 * max(1.0, np.abs(want).max()), lev


TRAIN_SET = [(101, 2, 32, 3, 4.0, 8.0), (102, 2, 48, 3, 2.0, 1.0), (103, 3, 8, 2, 4.0, 8.0), (104, 3, 12, 2, 2.0, 1.0),
             (105, 3, 16, 2, 3.0, 4.0), (106, 2, 64, 4, 3.0, 4.0), (107, 3, 16, 2, 1.0, 1.0), (108, 2, 64, 4, 1.0, 2.0)]


def test_trained_network_gains_over_fixed_damping_on_held_out_problems():
    """Train on line-search labels gathered from 2-D and 3-D runs (seeds 101-108,
    blob contrasts 1e1-1e4, aspect ratios 1-8), then solve held-out problems
    (seed 2103) to 1e-8 with the fixed damping 0.5 and with the learned one,
    installed as one predicted weight per level (shrink 0).  The network must
    cut the V-cycle count against 0.5 and match the best weight of a fixed-damping
    sweep (0.3 .. 0.9) to one FGMRES iteration; the oracle's residual checks the
    learned solutions."""
    Xs, ys = [], []
    for seed, dim, N, nlev, s_max, asp in TRAIN_SET:
        spec = _problem(dim, N, nlev, seed, s_max=s_max, aspect=asp)
        mg = R.Multigrid(**spec)
        sm = R.Smoother(mg, R.RAV, R.F64, 0.5)
        X, y = learned.collect(mg, sm, mg.initial_guess(), mg.rhs(R.F_SINKER), cycles=3)
        Xs.append(X)
        ys.append(y)
    P, losses = learned.train(torch.cat(Xs), torch.cat(ys), steps=1500, lr=3e-3)
    assert losses[-1][1] < 0.5 * losses[0][1]

    for dim, N, nlev, s_max, asp in [(3, 24, 3, 2.0, 1.0), (2, 64, 4, 2.0, 1.0)]:
        spec = _problem(dim, N, nlev, 2103, s_max=s_max, aspect=asp)
        mg = R.Multigrid(**spec)
        sm = R.Smoother(mg, R.RAV, R.F64, 0.5)
        b = mg.rhs(R.F_SINKER)
        it_fixed, _, rc1 = mg.solve(sm, mg.initial_guess(), b, tol=1e-8, maxit=200)
        learned.install(sm, P, shrink=0.0)
        x = mg.initial_guess()
        info = {}
        it_learn, _, rc2 = mg.solve(sm, x, b, tol=1e-8, maxit=200, fallback_rho=1.0, info_out=info)
        print(f"{dim}-D N={N}: cycles to 1e-8 fixed 0.5 -> {it_fixed}, learned -> {it_learn}")
        assert rc1 == 0 and rc2 == 0 and not info["fell_back"]
        assert it_learn < it_fixed
        # against the best fixed damping of a sweep 0.3 .. 0.9 (FGMRES(30) iterations):
        # one inference finds a weight per level as good as the sweep's best, to one iteration
        it_fg_learn, _, rc3 = mg.solve(sm, mg.initial_guess(), b, tol=1e-8, maxit=200, outer=1)
        sweep = {}
        for om in (0.3, 0.4, 0.5, 0.6, 0.7, 0.8, 0.9):
            sw = R.Smoother(mg, R.RAV, R.F64, om)
            it_om, _, rc_om = mg.solve(sw, mg.initial_guess(), b, tol=1e-8, maxit=200, outer=1, raise_on_error=False)
            sweep[om] = it_om if rc_om == 0 else 10 ** 6
            del sw
        print(f"  FGMRES: learned {it_fg_learn}, swept fixed {sweep}")
        assert rc3 == 0 and it_fg_learn <= min(sweep.values()) + 1
        orc = O.Oracle(dim, N, nlev, coords=spec["coords"], blobs=spec["blobs"], bc=O.BC_NOSLIP)
        bo = orc.rhs(O.F_SINKER)
        r0 = np.linalg.norm(orc.residual(nlev - 1, orc.initial_guess(), bo))
        r = np.linalg.norm(orc.residual(nlev - 1, x.cpu().numpy(), bo))
        assert r <= 2e-8 * r0


def test_fallback_restores_fixed_damping():
    """A damping that makes the cycle diverge is replaced by the fixed one."""
    spec = _problem(2, 32, 3, 2103, s_max=1.0, aspect=1.0)
    mg = R.Multigrid(**spec)
    sm = R.Smoother(mg, R.RAV, R.F64, 0.5)
    b = mg.rhs(R.F_SINKER)
    for lev in (1, 2):
        sm.set_omega(lev, torch.full((mg.counts(lev)["n_p"],), 1.5, device="cuda"))
    info = {}
    it, hist, rc = mg.solve(sm, mg.initial_guess(), b, tol=1e-8, maxit=200, fallback_rho=1.0, info_out=info)
    assert rc == 0 and info["fell_back"]


@pytest.mark.slow
def test_full_size_40cube_features_follow_their_definition():
    """The learned-damping benchmark's configuration (3-D 40^3, 4 levels, 20
    blobs of contrast up to 1e4, z-graded cells of aspect 8, seed 2103): the
    features of sampled fine-level subdomains equal their definition computed
    with numpy (viscosity at the 3^3 Gauss points of the cells around the
    vertex, cell aspects and diagonals, level, size and Dirichlet shares)."""
    N, nlev = 40, 4
    coords = inputs.graded_coordinates(N, 8.0, 3)
    blobs = inputs.viscosity_blobs(inputs.BASE_SEED, k=20, s_max=4.0)
    mg = R.Multigrid(3, N, nlev, coords=coords, blobs=blobs, bc=R.BC_NOSLIP)
    sm = R.Smoother(mg, R.RAV, R.F64, 0.5)
    f = learned.features(sm, nlev - 1).cpu().numpy()
    orc = O.Oracle(3, 4, 1, blobs=blobs)  # viscosity only
    xg, _ = np.polynomial.legendre.leggauss(3)
    xg = 0.5 * (xg + 1)
    N1 = N + 1
    samples = [0, N, N1 * N1 - 1, N1 ** 3 - 1] + (inputs.uniform(78, 12) * N1 ** 3).astype(int).tolist()
    for p in samples:
        v = (p % N1, (p // N1) % N1, p // (N1 * N1))
        cells = [(i, j, k) for i in (v[0] - 1, v[0]) for j in (v[1] - 1, v[1]) for k in (v[2] - 1, v[2])
                 if 0 <= i < N and 0 <= j < N and 0 <= k < N]
        etas, asp, diag = [], [], []
        for i, j, k in cells:
            h = [coords[0][i + 1] - coords[0][i], coords[1][j + 1] - coords[1][j], coords[2][k + 1] - coords[2][k]]
            asp.append(max(h) / min(h))
            diag.append(np.sqrt(sum(t * t for t in h)))
            for a in xg:
                for bq in xg:
                    for cq in xg:
                        etas.append(orc.viscosity(np.array([coords[0][i] + h[0] * a, coords[1][j] + h[1] * bq,
                                                            coords[2][k] + h[2] * cq])))
        etas = np.array(etas)
        box = [(2 * v[0] - 2 + a, 2 * v[1] - 2 + b2, 2 * v[2] - 2 + c) for a in range(5) for b2 in range(5)
               for c in range(5)]
        inside = [t for t in box if all(0 <= q <= 2 * N for q in t)]
        bnd = [t for t in inside if any(q in (0, 2 * N) for q in t)]
        nvalid = len(inside) - len(bnd)
        want = [np.log10(etas.max() / etas.min()), np.log10(etas).mean(), np.log10(max(asp)), np.log10(min(asp)),
                1.0, (3 * nvalid + 1) / (3 * 125 + 1), len(bnd) / len(inside), np.log10(np.mean(diag))]
        for q in range(8):
            assert abs(f[p, q] - want[q]) <= 1e-5 * max(1.0, abs(want[q])), (p, q, f[p, q], want[q])
