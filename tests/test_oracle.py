"""Pins of the FP64 oracle against facts that do not come from the oracle itself:
closed-form solutions, textbook operator forms built with numpy.linalg,
library routines, invariants and the paper's stated counts.

Paper references: Saberi, Meschke, Vogel, "A restricted additive Vanka smoother
for geometric multigrid" (Sec. 2 Eqs. 5-8, Sec. 3 Eqs. 9-13, Sec. 4, Sec. 4.3 Eq. 15).
"""
import os

import numpy as np
import pytest

import oracle as O
from oracle_helpers import (dense, free_residual, interpolate, node_coords, rav_matrix, vertex_coords,
                            vertex_index)
from paper_2103_10127_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def quad_u(dim):
    if dim == 2:
        return lambda X, c: X[:, 1] ** 2 if c == 0 else X[:, 0] ** 2
    return lambda X, c: [X[:, 1] ** 2, X[:, 2] ** 2, X[:, 0] ** 2][c]


def read_golden(name):
    rows = {}
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.split("#")[0].strip()
            if line:
                k, v = line.split("=")
                rows[k.strip()] = float(v)
    return rows


# --------------------------------------------------------------------------- counting
def test_dof_counting_convention():
    """n_DoF counts every DoF incl. Dirichlet ones, as in the paper's Table 1
    (Omega^1: 64 elements -> 243 = 3 * 81 DoFs for Q1-Q1); the 16x16 Q2-Q1
    cavity has 2178 velocity + 289 pressure DoFs."""
    g = read_golden("dof_counts.txt")
    o = O.Oracle(2, 8, 1)
    n_vertices = o.sizes(0)["n_p"]
    assert 3 * n_vertices == g["table1_omega1_q1q1_dofs"]
    assert 8 * 8 == g["table1_omega1_elements"]
    o16 = O.Oracle(2, 16, 3)
    s = o16.sizes(2)
    assert s["n_u"] == g["q2q1_16x16_velocity"] and s["n_p"] == g["q2q1_16x16_pressure"]
    assert s["n"] == 2467
    o3 = O.Oracle(3, 4, 1)
    assert o3.sizes(0)["n_u"] == 3 * 9 ** 3 and o3.sizes(0)["n_p"] == 5 ** 3


# --------------------------------------------------------------------------- assembly
@pytest.mark.parametrize("dim,N,nlev,graded", [(2, 8, 3, False), (2, 8, 2, True), (3, 4, 2, False)])
def test_manufactured_quadratic_solution_is_reproduced(dim, N, nlev, graded):
    """u = (y^2, x^2) [(y^2, z^2, x^2)], p = sum x - d/2 lies in the Q2-Q1 space,
    so the discrete solution equals its interpolant (closed form)."""
    coords = inputs.graded_coordinates(N, 3.0, dim) if graded else None
    o = O.Oracle(dim, N, nlev, coords=coords, bc=O.BC_QUADRATIC)
    o.setup_smoother(O.RAV, 0.5)
    b = o.rhs(O.F_QUADRATIC)
    x, it, hist = o.solve(o.initial_guess(), b, tol=1e-13, maxit=400)
    assert it > 0
    ex = interpolate(dim, N, quad_u(dim), lambda V: V.sum(1) - dim / 2.0, coords)
    nu = o.sizes(nlev - 1)["n_u"]
    assert np.abs(x[:nu] - ex[:nu]).max() < 1e-10
    p, pe = x[nu:], ex[nu:]
    assert np.abs((p - p.mean()) - (pe - pe.mean())).max() < 1e-8


def test_energy_with_variable_viscosity_matches_gauss_legendre():
    """u^T A u = int eta |grad u|^2 for a biquadratic u vanishing on the boundary,
    integrated here with numpy's Gauss-Legendre rule and the blob viscosity."""
    dim, N = 2, 4
    coords = inputs.graded_coordinates(N, 2.0, dim)
    blobs = inputs.viscosity_blobs(7, k=3, s_max=2.0)
    o = O.Oracle(dim, N, 1, coords=coords, blobs=blobs, bc=O.BC_NOSLIP)
    L = dense(o, 0)
    m, _ = o.dirichlet(0)
    f = lambda X, c: X[:, 0] * (1 - X[:, 0]) * X[:, 1] * (1 - X[:, 1])
    u = interpolate(dim, N, f, None, coords)
    nu = o.sizes(0)["n_u"]
    free = ~m[:nu]
    uf = u[:nu][free]
    energy = uf @ L[:nu, :nu][np.ix_(free, free)] @ uf
    xg, wg = np.polynomial.legendre.leggauss(3)
    xg, wg = 0.5 * (xg + 1), 0.5 * wg
    ref = 0.0
    for i in range(N):
        for j in range(N):
            x0, x1 = coords[0][i], coords[0][i + 1]
            y0, y1 = coords[1][j], coords[1][j + 1]
            for a in range(3):
                for bq in range(3):
                    X = x0 + (x1 - x0) * xg[a]
                    Y = y0 + (y1 - y0) * xg[bq]
                    g1 = (1 - 2 * X) * Y * (1 - Y)
                    g2 = X * (1 - X) * (1 - 2 * Y)
                    eta = o.viscosity(np.array([X, Y, 0.0]))
                    ref += wg[a] * wg[bq] * (x1 - x0) * (y1 - y0) * eta * 2 * (g1 * g1 + g2 * g2)
    assert abs(energy - ref) < 1e-12 * ref


def test_blob_viscosity_range():
    """eta in [eta0, eta0 * 10^max s] and eta0 * 10^s_k at blob centres far from others."""
    blobs = np.array([[0.3, 0.3, 0.5, 0.05, 2.0]])
    o = O.Oracle(3, 2, 1, blobs=blobs, eta0=2.0)
    assert abs(o.viscosity(np.array([0.3, 0.3, 0.5])) - 200.0) < 1e-9
    assert abs(o.viscosity(np.array([0.9, 0.9, 0.9])) - 2.0) < 1e-12


@pytest.mark.parametrize("dim,N", [(2, 4), (3, 2)])
def test_saddle_point_structure(dim, N):
    """L_FF symmetric; constant velocity and constant pressure are in the kernel
    of the free rows (grad of a constant and the integral of div v, v in V_0)."""
    blobs = inputs.viscosity_blobs(3, k=4)
    o = O.Oracle(dim, N, 1, blobs=blobs, bc=O.BC_CAVITY)
    L = dense(o, 0)
    m, _ = o.dirichlet(0)
    F = ~m
    LFF = L[np.ix_(F, F)]
    assert np.abs(LFF - LFF.T).max() <= 1e-14 * np.abs(LFF).max()
    nu = o.sizes(0)["n_u"]
    one_u = np.concatenate([np.ones(nu), np.zeros(L.shape[0] - nu)])
    one_p = np.concatenate([np.zeros(nu), np.ones(L.shape[0] - nu)])
    sc = np.abs(L).max()
    assert np.abs((L @ one_u)[F]).max() < 1e-12 * sc
    assert np.abs((L @ one_p)[F]).max() < 1e-12 * sc
    # B^T applied to the interpolant of a divergence-free quadratic vanishes
    u = interpolate(dim, N, quad_u(dim), None)
    assert np.abs((L @ u)[nu:]).max() < 1e-12 * sc


# --------------------------------------------------------------------------- subdomains
@pytest.mark.parametrize("dim,N", [(2, 6), (3, 4)])
def test_subdomains_follow_the_algebraic_definition(dim, N):
    """S_i = {p_i} + the free DoFs in the nonzero pattern of row i of B^T (Sec. 3)."""
    o = O.Oracle(dim, N, 1, bc=O.BC_CAVITY)
    o.build_patches(0)
    off, dofs, own = o.patches(0)
    rp, ci, va = o.csr(0)
    m, _ = o.dirichlet(0)
    nu = o.sizes(0)["n_u"]
    for i in range(o.sizes(0)["n_p"]):
        row = ci[rp[nu + i]:rp[nu + i + 1]]
        want = np.sort(np.concatenate([row[~m[row]], [nu + i]]))
        assert np.array_equal(dofs[off[i]:off[i + 1]], want)
    sizes = np.diff(off)
    assert sizes.max() == (51 if dim == 2 else 376)


@pytest.mark.parametrize("dim,N", [(2, 6), (3, 3)])
def test_ownership_is_a_partition_of_unity(dim, N):
    """sum_i G_i = I on the free DoFs; owned sets inside their subdomain; the
    vertex DoFs belong to their own vertex (Eq. 13's restricted set); interior
    subdomains own 2^d d + 1 DoFs."""
    o = O.Oracle(dim, N, 1, bc=O.BC_CAVITY)
    o.build_patches(0)
    off, dofs, own = o.patches(0)
    m, _ = o.dirichlet(0)
    assert np.all(own[m] == -1) and np.all(own[~m] >= 0)
    count = np.zeros(len(own), int)
    for i in range(len(off) - 1):
        s = dofs[off[i]:off[i + 1]]
        mine = s[own[s] == i]
        count[mine] += 1
    assert np.all(count[~m] == 1) and np.all(count[m] == 0)
    nu = o.sizes(0)["n_u"]
    M = 2 * N + 1
    vidx = vertex_index(dim, N)
    for i, v in enumerate(vidx):
        nid = sum(int(2 * v[a]) * M ** a for a in range(dim))
        for c in range(dim):
            dof = dim * nid + c
            if not m[dof]:
                assert own[dof] == i
        assert own[nu + i] == i
        if np.all((v > 0) & (v < N - 1)):
            s = dofs[off[i]:off[i + 1]]
            assert (own[s] == i).sum() == 2 ** dim * dim + 1


# --------------------------------------------------------------------------- smoothers
def _problem(dim, N, bc=O.BC_CAVITY, seed=11):
    blobs = inputs.viscosity_blobs(seed, k=3, s_max=1.0)
    return O.Oracle(dim, N, 2, blobs=blobs, bc=bc)


@pytest.mark.parametrize("dim,N", [(2, 4), (2, 6), (3, 4)])
def test_rav_step_equals_assembled_operator(dim, N):
    """x + S_RAV (b - L x), S_RAV = sum_i Rt_i^T w_i L_i^{-1} R_i (Eq. 13), built with numpy.linalg.inv."""
    o = _problem(dim, N)
    o.setup_smoother(O.RAV, 0.7)
    lev = 1
    off, dofs, own = o.patches(lev)
    w = 0.3 + 0.6 * inputs.uniform(5, len(off) - 1)
    o.set_omega(lev, w)
    L = dense(o, lev)
    m, _ = o.dirichlet(lev)
    S = rav_matrix(L, off, dofs, own, w, restricted=True)
    rng = np.random.default_rng(1)
    x, b = rng.standard_normal(L.shape[0]), rng.standard_normal(L.shape[0])
    want = x + S @ free_residual(L, x, b, m)
    got = o.smooth(lev, x, b)
    assert np.abs(got - want).max() <= 1e-12 * np.abs(want).max()


@pytest.mark.parametrize("dim,N", [(2, 4), (3, 4)])
def test_av_step_equals_assembled_operator(dim, N):
    """x + S_AV (b - L x), S_AV = sum_i R_i^T w L_i^{-1} R_i (Eq. 12)."""
    o = _problem(dim, N)
    o.setup_smoother(O.AV, 0.1)
    off, dofs, own = o.patches(1)
    L = dense(o, 1)
    m, _ = o.dirichlet(1)
    S = rav_matrix(L, off, dofs, own, 0.1, restricted=False)
    rng = np.random.default_rng(2)
    x, b = rng.standard_normal(L.shape[0]), rng.standard_normal(L.shape[0])
    want = x + S @ free_residual(L, x, b, m)
    got = o.smooth(1, x, b)
    assert np.abs(got - want).max() <= 1e-12 * np.abs(want).max()


@pytest.mark.parametrize("kind", [O.MV, O.MV_COLOURED])
def test_mv_step_is_the_product_of_subdomain_corrections(kind):
    """Multiplicative Vanka: the error propagates as prod_i (I - w R_i^T L_i^{-1} R_i L)
    in the sweep order (Eq. 11 as a multiplicative Schwarz method); lexicographic,
    or coloured by (v mod 4) with colours ascending."""
    dim, N = 2, 4
    o = _problem(dim, N)
    o.setup_smoother(kind, 0.66)
    off, dofs, own = o.patches(1)
    L = dense(o, 1)
    m, g = o.dirichlet(1)
    n = L.shape[0]
    order = np.arange(len(off) - 1)
    if kind == O.MV_COLOURED:
        v = vertex_index(dim, N)
        col = (v[:, 0] % 4) + 4 * (v[:, 1] % 4)
        order = np.argsort(col, kind="stable")
    E = np.eye(n)
    for p in order:
        s = dofs[off[p]:off[p + 1]]
        Pi = np.zeros((n, n))
        Pi[np.ix_(s, np.arange(n))] = np.linalg.solve(L[np.ix_(s, s)], L[s, :])
        E = (np.eye(n) - 0.66 * Pi) @ E
    rng = np.random.default_rng(3)
    xs = rng.standard_normal(n)
    b = L @ xs
    b[m] = xs[m]
    e0 = rng.standard_normal(n)
    e0[m] = 0.0
    got = o.smooth(1, xs + e0, b) - xs
    want = E @ e0
    assert np.abs(got - want).max() <= 1e-11 * np.abs(e0).max()


def test_single_global_subdomain_solves_exactly():
    """One subdomain holding every free DoF but one pressure (which fixes the
    constant) makes R_sd = Rt_sd = I there, and one step with w = 1 is an exact
    solve for all three variants."""
    dim, N = 2, 4
    for kind in (O.RAV, O.AV, O.MV):
        o = _problem(dim, N, bc=O.BC_CAVITY)
        o.setup_smoother(kind, 1.0)
        L = dense(o, 1)
        m, g = o.dirichlet(1)
        n = L.shape[0]
        nu = o.sizes(1)["n_u"]
        dofs = np.array([i for i in range(n) if not m[i] and i != nu])
        owner = np.full(n, -1)
        owner[dofs] = 0
        o.set_patches(1, np.array([0, len(dofs)]), dofs, owner, 1.0)
        rng = np.random.default_rng(4)
        xs = rng.standard_normal(n)
        xs[m] = g[m]
        b = L @ xs
        b[m] = g[m]
        x0 = g.copy()
        x1 = o.smooth(1, x0, b)
        r = free_residual(L, x1, b, m)
        assert np.linalg.norm(r) <= 1e-12 * np.linalg.norm(b)


def test_disjoint_subdomains_make_rav_and_av_block_jacobi():
    """With pairwise disjoint subdomains every DoF is owned by its only
    subdomain, so Rt_i = R_i and Eq. 13 equals Eq. 12: both are block Jacobi.
    The disjoint blocks used are the owned sets of the vertices that own a
    velocity DoF."""
    dim, N = 2, 4
    ref = _problem(dim, N)
    ref.build_patches(1)
    _, _, own0 = ref.patches(1)
    nu = ref.sizes(1)["n_u"]
    chunks = []
    for v in range(ref.sizes(1)["n_p"]):
        c = np.flatnonzero(own0 == v)
        if (c < nu).any():
            chunks.append(c)
    res = {}
    for kind in (O.RAV, O.AV):
        o = _problem(dim, N)
        o.setup_smoother(kind, 0.8)
        L = dense(o, 1)
        m, _ = o.dirichlet(1)
        off = np.concatenate([[0], np.cumsum([len(c) for c in chunks])])
        owner = np.full(L.shape[0], -1)
        for k, c in enumerate(chunks):
            owner[c] = k
        o.set_patches(1, off, np.concatenate(chunks), owner, 0.8)
        rng = np.random.default_rng(5)
        x, b = rng.standard_normal(L.shape[0]), rng.standard_normal(L.shape[0])
        res[kind] = o.smooth(1, x, b)
        r = free_residual(L, x, b, m)
        want = x.copy()
        for c in chunks:
            want[c] += 0.8 * np.linalg.solve(L[np.ix_(c, c)], r[c])
        assert np.abs(res[kind] - want).max() <= 1e-11 * np.abs(want).max()
    assert np.abs(res[O.RAV] - res[O.AV]).max() <= 1e-12 * np.abs(res[O.AV]).max()


# --------------------------------------------------------------------------- transfers
@pytest.mark.parametrize("dim,graded", [(2, False), (2, True), (3, False), (3, True)])
def test_prolongation_reproduces_coarse_polynomials(dim, graded):
    """P maps the coarse interpolant of a random tensor-quadratic velocity and a
    multilinear pressure to the fine interpolant (nested Q2/Q1 spaces)."""
    N = 8 if dim == 2 else 4
    coords = inputs.graded_coordinates(N, 3.0, dim) if graded else None
    o = O.Oracle(dim, N, 2, coords=coords, bc=O.BC_NOSLIP)
    rng = np.random.default_rng(6)
    cu = rng.standard_normal((dim,) + (3,) * dim)
    cp = rng.standard_normal((2,) * dim)

    def poly(X, coef):
        out = np.zeros(len(X))
        for idx in np.ndindex(coef.shape):
            out += coef[idx] * np.prod([X[:, a] ** idx[a] for a in range(dim)], axis=0)
        return out

    uf = lambda X, c: poly(X, cu[c])
    pf = lambda V: poly(V, cp)
    ccoords = None if coords is None else coords[:, ::2]
    xc = interpolate(dim, N // 2, uf, pf, ccoords)
    xf = interpolate(dim, N, uf, pf, coords)
    m, _ = o.dirichlet(1)
    got = o.prolong_add(1, xc, np.zeros_like(xf))
    assert np.abs(got[~m] - xf[~m]).max() < 1e-12 * np.abs(xf).max()
    assert np.all(got[m] == 0.0)


def test_restriction_is_the_adjoint_of_prolongation():
    o = O.Oracle(2, 8, 2, bc=O.BC_CAVITY)
    rng = np.random.default_rng(7)
    mf, _ = o.dirichlet(1)
    mc, _ = o.dirichlet(0)
    rf = rng.standard_normal(len(mf))
    rf[mf] = 0
    xc = rng.standard_normal(len(mc))
    xc[mc] = 0
    lhs = o.prolong_add(1, xc, np.zeros(len(mf))) @ rf
    rhs = xc @ o.restrict(1, rf)
    assert abs(lhs - rhs) < 1e-12 * abs(lhs)


def test_coarse_solve_matches_numpy_on_bordered_system():
    """Coarse LU solve (Sec. 2) of [L e_p; e_p^T 0] checked with numpy.linalg.solve."""
    o = O.Oracle(2, 4, 1, bc=O.BC_CAVITY)
    L = dense(o, 0)
    m, _ = o.dirichlet(0)
    n, nu = L.shape[0], o.sizes(0)["n_u"]
    Mb = np.zeros((n + 1, n + 1))
    Mb[:n, :n] = L
    Mb[nu:n, n] = 1
    Mb[n, nu:n] = 1
    rng = np.random.default_rng(8)
    b = rng.standard_normal(n)
    b[m] = 0
    want = np.linalg.solve(Mb, np.concatenate([b, [0]]))[:n]
    got = o.coarse_solve(b)
    assert np.abs(got - want).max() < 1e-11 * np.abs(want).max()
    assert abs(got[nu:].sum()) < 1e-10 * np.abs(got).max()


def test_two_grid_cycle_error_propagation():
    """V(2,2) on two levels propagates the error as
    (I - S L)^2 (I - P C R L) (I - S L)^2 with C the bordered coarse inverse."""
    dim, N = 2, 4
    o = _problem(dim, N)
    o.setup_smoother(O.RAV, 0.6)
    Lf, Lc = dense(o, 1), dense(o, 0)
    mf, gf = o.dirichlet(1)
    mc, _ = o.dirichlet(0)
    off, dofs, own = o.patches(1)
    S = rav_matrix(Lf, off, dofs, own, 0.6)
    P = o.prolongation(1).toarray()
    nc, nuc = Lc.shape[0], o.sizes(0)["n_u"]
    Mb = np.zeros((nc + 1, nc + 1))
    Mb[:nc, :nc] = Lc
    Mb[nuc:nc, nc] = 1
    Mb[nc, nuc:nc] = 1
    C = np.linalg.inv(Mb)[:nc, :nc] @ np.diag((~mc).astype(float))
    Df = np.diag((~mf).astype(float))
    Dc = np.diag((~mc).astype(float))
    n = Lf.shape[0]
    Es = np.eye(n) - S @ Df @ Lf
    Ec = np.eye(n) - P @ C @ Dc @ P.T @ Df @ Lf
    E = Es @ Es @ Ec @ Es @ Es
    rng = np.random.default_rng(9)
    xs = rng.standard_normal(n)
    xs[mf] = gf[mf]
    b = Lf @ xs
    b[mf] = gf[mf]
    e0 = rng.standard_normal(n)
    e0[mf] = 0
    got = o.vcycle(xs + e0, b, 2, 2) - xs
    assert np.abs(got - E @ e0).max() < 1e-10 * np.abs(e0).max()


# --------------------------------------------------------------------------- solvers
def test_fgmres_and_stationary_mg_reach_the_direct_solution():
    import scipy.sparse as sp
    import scipy.sparse.linalg as spla
    o = O.Oracle(2, 8, 2, blobs=inputs.viscosity_blobs(4, k=5), bc=O.BC_CAVITY)
    o.setup_smoother(O.RAV, 0.5)
    b = o.rhs(O.F_NONE)
    L = o.matrix(1)
    n, nu = L.shape[0], o.sizes(1)["n_u"]
    e = sp.csr_matrix((np.ones(n - nu), (np.arange(nu, n), np.zeros(n - nu))), shape=(n, 1))
    Mb = sp.bmat([[L, e], [e.T, None]]).tocsc()
    xd = spla.spsolve(Mb, np.concatenate([b, [0]]))[:n]
    for method in ("fgmres", "solve"):
        x, it, hist = getattr(o, method)(o.initial_guess(), b, tol=1e-11, maxit=300)
        assert it > 0 and hist[-1] <= 1e-11
        assert np.abs(x[:nu] - xd[:nu]).max() < 1e-8
        p, pd = x[nu:] - x[nu:].mean(), xd[nu:] - xd[nu:].mean()
        assert np.abs(p - pd).max() < 1e-6 * max(1.0, np.abs(pd).max())
        if method == "fgmres":
            assert np.all(np.diff(hist[1:]) <= 1e-12)


def test_manufactured_stream_function_converges_at_textbook_rates():
    """u = curl(sin^2(pi x) sin^2(pi y)), p = cos(pi x) cos(pi y): nodal errors of
    the Q2-Q1 solution fall at least like h^3 (u) and h^2 (p)."""
    eu, ep = [], []
    for N in (8, 16, 32):
        o = O.Oracle(2, N, 2, bc=O.BC_NOSLIP)
        o.setup_smoother(O.RAV, 0.5)
        b = o.rhs(O.F_PSI)
        x, it, _ = o.solve(o.initial_guess(), b, tol=1e-11, maxit=300)
        assert it > 0
        pi = np.pi
        uf = lambda X, c: (pi * np.sin(pi * X[:, 0]) ** 2 * np.sin(2 * pi * X[:, 1]) if c == 0
                           else -pi * np.sin(2 * pi * X[:, 0]) * np.sin(pi * X[:, 1]) ** 2)
        ex = interpolate(2, N, uf, lambda V: np.cos(pi * V[:, 0]) * np.cos(pi * V[:, 1]))
        nu = o.sizes(1)["n_u"]
        eu.append(np.abs(x[:nu] - ex[:nu]).max())
        p, pe = x[nu:] - x[nu:].mean(), ex[nu:] - ex[nu:].mean()
        ep.append(np.abs(p - pe).max())
    ru = np.log2(np.array(eu[:-1]) / np.array(eu[1:]))
    rp = np.log2(np.array(ep[:-1]) / np.array(ep[1:]))
    assert ru.min() > 2.7, (eu, ru)
    assert rp.min() > 1.7, (ep, rp)


def test_rav_multigrid_converges_on_the_cavity():
    """Stationary MG with RAV(0.5) V(2,2) on the 16x16 Q2-Q1 cavity reaches 1e-8."""
    o = O.Oracle(2, 16, 3, bc=O.BC_CAVITY)
    o.setup_smoother(O.RAV, 0.5)
    b = o.rhs(O.F_NONE)
    x, it, hist = o.solve(o.initial_guess(), b, tol=1e-8, maxit=100)
    assert 0 < it < 60 and hist[-1] <= 1e-8


# --------------------------------------------------------------------------- precision
def test_round_format_matches_library_casts():
    """RNE into fp32 equals numpy's cast; bf16 and fp8 e4m3 equal torch's casts of
    fp32-representable values; fp8 saturates at 448."""
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(10)
    v = rng.standard_normal(20000) * np.exp(rng.uniform(-30, 30, 20000))
    assert np.array_equal(O.round_format(O.F32, v), v.astype(np.float32).astype(np.float64))
    v32 = v.astype(np.float32).astype(np.float64)
    tb = torch.from_numpy(v32.astype(np.float32)).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(O.round_format(O.BF16, v32), tb)
    w = (rng.standard_normal(20000) * np.exp(rng.uniform(-12, 5, 20000))).astype(np.float32).astype(np.float64)
    w = w[np.abs(w) < 448]
    t8 = torch.from_numpy(w.astype(np.float32)).to(torch.float8_e4m3fn).to(torch.float64).numpy()
    assert np.array_equal(O.round_format(O.FP8, w), t8)
    assert np.array_equal(O.round_format(O.FP8, np.array([1e6, -1e6, 464.0])), np.array([448.0, -448.0, 448.0]))


@pytest.mark.parametrize("prec,bound", [(O.F32, 1e-6), (O.BF16, 2e-2), (O.FP8, 2e-1)])
def test_reduced_precision_step_error_is_bounded(prec, bound):
    """The quantised rows equal the fp64 rows rounded (fp32: numpy's cast), and
    one RAV step moves by at most ~unit roundoff of the format times a modest factor."""
    o = _problem(2, 8)
    o.setup_smoother(O.RAV, 0.5, prec)
    rows = o.inverse(1, 12)
    q, s = o.inverse(1, 12, quantised=True)
    if prec == O.F32:
        assert np.array_equal(q, rows.astype(np.float32).astype(np.float64))
    rel = np.abs(q * s[:, None] - rows).max() / np.abs(rows).max()
    assert rel <= {O.F32: 6e-8, O.BF16: 4e-3, O.FP8: 7e-2}[prec]
    o64 = _problem(2, 8)
    o64.setup_smoother(O.RAV, 0.5)
    rng = np.random.default_rng(12)
    n = o.sizes(1)["n"]
    x, b = rng.standard_normal(n), rng.standard_normal(n)
    d64 = o64.smooth(1, x, b) - x
    dq = o.smooth(1, x, b) - x
    assert np.linalg.norm(dq - d64) <= bound * np.linalg.norm(d64)


@pytest.mark.parametrize("dim,N", [(2, 8), (3, 4)])
def test_factored_storage_rebuilds_the_inverse(dim, N):
    """Rows rebuilt from A^{-1}, w = A^{-1} b and 1/s (block inverse of the
    saddle-point local system) equal the rows of L_i^{-1} from the LU of L_i^T
    up to the format's rounding: a wrong sign, index or dropped rank-one term
    would leave an O(1) error.  fp32 rounding of the stored values is exactly
    numpy's cast, so fp32 stays near 2^-24 and bf16 near 2^-8."""
    blobs = inputs.viscosity_blobs(3, k=6, s_max=3.0)
    exact = O.Oracle(dim, N, 2, blobs=blobs, bc=O.BC_NOSLIP)
    exact.setup_smoother(O.RAV, 0.5)
    for prec, bound in ((O.F32_FACT, 2.0 ** -23), (O.BF16_FACT, 2.0 ** -7)):
        o = O.Oracle(dim, N, 2, blobs=blobs, bc=O.BC_NOSLIP)
        o.setup_smoother(O.RAV, 0.5, prec)
        worst = 0.0
        for p in range((N + 1) ** dim):
            rows = exact.inverse(1, p)
            q, s = o.inverse(1, p, quantised=True)
            assert np.array_equal(s, np.ones(len(s)))
            assert q.shape == rows.shape
            worst = max(worst, np.abs(q - rows).max() / np.abs(rows).max())
        assert worst <= bound, (prec, worst)
        assert worst > 0.0  # the rounding did happen


def test_factored_storage_step_error_is_bounded():
    """One RAV step with fp32 / bf16 factored storage moves within the format's
    roundoff of the fp64 step (the rows are applied in fp64)."""
    o64 = _problem(2, 8)
    o64.setup_smoother(O.RAV, 0.5)
    rng = np.random.default_rng(13)
    n = o64.sizes(1)["n"]
    x, b = rng.standard_normal(n), rng.standard_normal(n)
    d64 = o64.smooth(1, x, b) - x
    for prec, bound in ((O.F32_FACT, 1e-6), (O.BF16_FACT, 2e-2)):
        o = _problem(2, 8)
        o.setup_smoother(O.RAV, 0.5, prec)
        dq = o.smooth(1, x, b) - x
        err = np.linalg.norm(dq - d64) / np.linalg.norm(d64)
        assert 0.0 < err <= bound, (prec, err)


# --------------------------------------------------------------------------- learned damping
def _mlp_params(seed, scale=0.3):
    return scale * inputs.normal(seed, O.mlp_nparam())


def test_mlp_forward_special_cases():
    """All weights zero but b3: omega = 1.5 sigmoid(b3); a single path through the
    first unit of each layer: omega = 1.5 sigmoid(max(f0, 0))."""
    n = O.mlp_nparam()
    assert n == 8 * 64 + 64 + 64 * 64 + 64 + 64 + 1 == 4801
    X = inputs.normal(1, 40).reshape(5, 8)
    P = np.zeros(n)
    P[-1] = 0.7
    assert np.allclose(O.mlp_forward(P, X), 1.5 / (1 + np.exp(-0.7)), rtol=0, atol=1e-15)
    P = np.zeros(n)
    P[0] = 1.0                      # W1[0][0]
    P[8 * 64 + 64] = 1.0            # W2[0][0]
    P[8 * 64 + 64 + 64 * 64 + 64] = 1.0  # W3[0]
    want = 1.5 / (1 + np.exp(-np.maximum(X[:, 0], 0.0)))
    assert np.abs(O.mlp_forward(P, X) - want).max() < 1e-15


def test_mlp_gradient_matches_central_differences():
    """Backpropagation against central finite differences of the fp64 loss."""
    P = _mlp_params(2)
    X = inputs.normal(3, 8 * 12).reshape(12, 8)
    y = 1.5 * inputs.uniform(4, 12)
    loss, g = O.mlp_loss_grad(P, X, y)
    idx = np.concatenate([np.arange(0, 4801, 97), [4800, 4799, 4736]])
    h = 1e-6
    for i in idx:
        Pp, Pm = P.copy(), P.copy()
        Pp[i] += h
        Pm[i] -= h
        fd = (O.mlp_loss_grad(Pp, X, y)[0] - O.mlp_loss_grad(Pm, X, y)[0]) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1e-3, np.abs(g).max()), (i, fd, g[i])


def test_labels_are_coordinate_line_search_minimisers():
    """omega*_i minimises ||r - L (s + (w - omega_i) c_i)||_2 over w (unclipped
    cases): c_i the subdomain's own restricted correction and s = sum_j omega_j c_j
    the whole RAV step, both built here with numpy.linalg.inv."""
    o = _problem(2, 4)
    o.build_patches(1)
    off, dofs, own = o.patches(1)
    L = dense(o, 1)
    m, _ = o.dirichlet(1)
    rng = np.random.default_rng(13)
    r = rng.standard_normal(L.shape[0])
    r[m] = 0.0
    omega = 0.3 + 0.4 * inputs.uniform(14, len(off) - 1)
    lab = o.labels(1, r, omega)
    cs = []
    for p in range(len(off) - 1):
        s_ = dofs[off[p]:off[p + 1]]
        keep = own[s_] == p
        c = np.zeros(L.shape[0])
        c[s_[keep]] = (np.linalg.inv(L[np.ix_(s_, s_)]) @ r[s_])[keep]
        cs.append(c)
    step = sum(w * c for w, c in zip(omega, cs))
    checked = 0
    for p, c in enumerate(cs):
        def f(w):
            res = r - L @ (step + (w - omega[p]) * c)
            res[m] = 0.0
            return np.sum(res ** 2)
        w = lab[p]
        assert 0.0 <= w <= 1.5
        if 0.0 < w < 1.5:
            checked += 1
            assert f(w) <= f(w + 1e-3) and f(w) <= f(w - 1e-3)
        elif w == 0.0:
            assert f(0.0) <= f(1e-3)
        else:
            assert f(1.5) <= f(1.5 - 1e-3)
    assert checked >= 5


@pytest.mark.parametrize("kind,prec", [(O.RAV, O.F64), (O.RAV, O.F32_FACT), (O.AV, O.F64)])
def test_thread_count_does_not_change_the_oracle(kind, prec):
    """The oracle's subdomain loops (local inverses, RAV corrections) may run
    on several threads; each subdomain's arithmetic is the same and RAV writes
    disjoint owned DoFs, so set-up, steps and V-cycles are bit-identical for
    any thread count."""
    rng = np.random.default_rng(3)
    coords = inputs.graded_coordinates(12, 3.0, 2)
    blobs = inputs.viscosity_blobs(17, k=5, s_max=2.0)
    outs = []
    try:
        for threads in (1, 4):
            O.set_threads(threads)
            orc = O.Oracle(2, 12, 2, coords=coords, blobs=blobs, bc=O.BC_NOSLIP)
            orc.setup_smoother(kind, 0.5 if kind == O.RAV else 0.1, prec)
            n = orc.sizes(1)["n"]
            x, b = rng.standard_normal(n), rng.standard_normal(n)
            outs.append((orc.smooth(1, x, b, 2), orc.vcycle(x, b, 2, 2),
                         orc.inverse(1, 5), orc.inverse(1, 40, quantised=prec != O.F64)))
            rng = np.random.default_rng(3)
    finally:
        O.set_threads(1)
    for a, b in zip(*outs):
        a, b = (a[0], b[0]) if isinstance(a, tuple) else (a, b)
        assert np.array_equal(a, b)


@pytest.mark.parametrize("dim,N,elem", [(2, 8, O.ELEM_Q2Q1), (3, 4, O.ELEM_Q2Q1), (2, 8, O.ELEM_Q1Q1)])
def test_patch_features_closed_forms_on_a_uniform_grid(dim, N, elem):
    """Constant viscosity eta0 on a uniform grid: no contrast, mean log10 eta0,
    aspect 1, level share, log10 of the cell diagonal h sqrt(d); the size and
    boundary shares of interior, corner and edge subdomains counted by hand
    from the box (5^d nodes on Q2-Q1, 3^d on Q1-Q1)."""
    orc = O.Oracle(dim, N, 2, eta0=2.5, bc=O.BC_NOSLIP, element=elem, beta=0.02)
    q = 1 if elem == O.ELEM_Q1Q1 else 2
    ext = 2 * q + 1
    for lev in (0, 1):
        Nl = N // 2 ** (1 - lev)
        f = orc.patch_features(lev)
        assert f.shape == ((Nl + 1) ** dim, 8)
        assert np.allclose(f[:, 0], 0.0, atol=1e-14)
        assert np.allclose(f[:, 1], np.log10(2.5), atol=1e-14)
        assert np.allclose(f[:, 2:4], 0.0, atol=1e-14)
        assert np.allclose(f[:, 4], lev)
        assert np.allclose(f[:, 7], np.log10(np.sqrt(dim) / Nl), atol=1e-14)
        M = q * Nl + 1

        def shares(v):
            axes = [[q * vv - q + a for a in range(ext)] for vv in v]
            inside = [J for J in np.array(np.meshgrid(*axes)).reshape(dim, -1).T if np.all((J >= 0) & (J < M))]
            bnd = [J for J in inside if np.any((J == 0) | (J == M - 1))]
            free = len(inside) - len(bnd)
            return (dim * free + 1) / (dim * ext ** dim + 1), len(bnd) / len(inside)

        for v in [(0,) * dim, (Nl // 2,) * dim, (1,) + (Nl // 2,) * (dim - 1), (Nl,) * dim]:
            p = sum(vv * (Nl + 1) ** a for a, vv in enumerate(v))
            want5, want6 = shares(v)
            assert abs(f[p, 5] - want5) < 1e-15 and abs(f[p, 6] - want6) < 1e-15, v
        if Nl >= 4:  # a vertex whose whole box is free
            inner = (Nl // 2,) * dim
            p = sum(vv * (Nl + 1) ** a for a, vv in enumerate(inner))
            assert f[p, 5] == 1.0 and f[p, 6] == 0.0


def test_patch_features_on_graded_cells_and_blobs():
    """Graded coordinates: the largest and smallest aspect ratios of the cells
    around a vertex are their side ratios; blob viscosity: the contrast is
    positive and grows with the blob strength, vanishes for strength 0, and
    the mean of log10 eta lies between log10 of the extremes."""
    N = 8
    coords = inputs.graded_coordinates(N, 4.0, 2)
    orc = O.Oracle(2, N, 1, coords=coords, bc=O.BC_NOSLIP)
    f = orc.patch_features(0)
    for v in [(0, 0), (3, 5), (8, 8), (4, 0)]:
        ratios = []
        for i in (v[0] - 1, v[0]):
            for j in (v[1] - 1, v[1]):
                if 0 <= i < N and 0 <= j < N:
                    hx, hy = coords[0][i + 1] - coords[0][i], coords[1][j + 1] - coords[1][j]
                    ratios.append(max(hx, hy) / min(hx, hy))
        p = v[0] + (N + 1) * v[1]
        assert abs(f[p, 2] - np.log10(max(ratios))) < 1e-13 and abs(f[p, 3] - np.log10(min(ratios))) < 1e-13
    blob = np.array([[0.5, 0.5, 0.0, 0.15, 0.0]])
    prev = None
    for s_ in (0.0, 1.0, 2.0):
        blob[0, 4] = s_
        fb = O.Oracle(2, N, 1, blobs=blob, bc=O.BC_NOSLIP).patch_features(0)
        p = 4 + (N + 1) * 4  # the vertex under the blob centre
        if s_ == 0.0:
            assert np.allclose(fb[:, 0], 0.0) and np.allclose(fb[:, 1], 0.0)
        else:
            assert fb[p, 0] > 0.0 and fb[p, 0] > prev
            assert 0.0 <= fb[p, 1] <= s_
        prev = fb[p, 0]
