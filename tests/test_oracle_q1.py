"""Pins of the oracle's stabilised Q1-Q1 discretisation (Sec. 2, Eqs. 7-8) and of
its Vanka subdomains (Sec. 3), against facts that do not come from the oracle:
operators rebuilt as tensor products of closed-form 1-D element matrices,
integration-by-parts identities for linear fields, a textbook convergence rate,
numpy.linalg inverses and scipy's sparse direct solver.

On Q1-Q1 velocity and pressure share the vertices: x holds the velocity
interleaved per vertex (d * id + c), then the pressure per vertex.
"""
import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as sla

import oracle as O
from oracle_helpers import dense, free_residual, rav_matrix, vertex_coords, vertex_index
from paper_2103_10127_gb300 import inputs

BETA = 0.02


def q1_oracle(dim, N, nlev=1, coords=None, eta0=1.0, blobs=None, bc=O.BC_CAVITY, beta=BETA):
    return O.Oracle(dim, N, nlev, coords=coords, eta0=eta0, blobs=blobs, bc=bc, element=O.ELEM_Q1Q1,
                    beta=beta)


def one_d(xv, weighted=False):
    """1-D linear-element matrices on vertices xv: stiffness S_ij = int phi_i' phi_j',
    mass M_ij = int phi_i phi_j, D_ij = int phi_i phi_j'; each cell's share times
    its length squared when weighted."""
    n = len(xv)
    S, M, D = np.zeros((n, n)), np.zeros((n, n)), np.zeros((n, n))
    for k in range(n - 1):
        h = xv[k + 1] - xv[k]
        f = h * h if weighted else 1.0
        ix = np.ix_([k, k + 1], [k, k + 1])
        S[ix] += f * np.array([[1.0, -1.0], [-1.0, 1.0]]) / h
        M[ix] += f * h * np.array([[2.0, 1.0], [1.0, 2.0]]) / 6.0
        D[ix] += f * np.array([[-0.5, 0.5], [-0.5, 0.5]])
    return S, M, D


def kron_axes(mats):
    """Operator on the vertex numbering id = i_0 + (N+1)(i_1 + (N+1) i_2) from
    per-axis factors (axis 0 fastest)."""
    out = mats[0]
    for m in mats[1:]:
        out = np.kron(m, out)
    return out


def tensor_operator(dim, xv, eta, beta, dirmask):
    """Dense L = [A B^T; B C] of Eqs. 7-8 for constant eta from 1-D factors:
    A = eta sum_a (S on axis a, M elsewhere) per component; B_c = -(D on axis c,
    M elsewhere); C = -beta sum_b sum_a (S on axis a, M elsewhere) with axis b's
    factor weighted by h_b^2, since h_e^2 = sum_b h_b^2 on a box cell."""
    one = [one_d(x) for x in xv]
    onew = [one_d(x, True) for x in xv]
    A = sum(kron_axes([one[m][0] if m == a else one[m][1] for m in range(dim)]) for a in range(dim))
    B = [-kron_axes([one[m][2] if m == c else one[m][1] for m in range(dim)]) for c in range(dim)]
    C = np.zeros_like(A)
    for b in range(dim):
        for a in range(dim):
            f = []
            for m in range(dim):
                src = onew if m == b else one
                f.append(src[m][0] if m == a else src[m][1])
            C -= beta * kron_axes(f)
    nv = A.shape[0]
    nu = dim * nv
    L = np.zeros((nu + nv, nu + nv))
    for c in range(dim):
        L[c:nu:dim, c:nu:dim] = eta * A
        L[c:nu:dim, nu:] = B[c].T
        L[nu:, c:nu:dim] = B[c]
    L[nu:, nu:] = C
    for i in np.nonzero(dirmask)[0]:
        L[i, :] = 0.0
        L[i, i] = 1.0
    return L


@pytest.mark.parametrize("dim,graded", [(2, False), (2, True), (3, True)])
def test_operator_equals_tensor_product_forms(dim, graded):
    """Every entry of the assembled Q1-Q1 operator (A scaled by eta, B and its
    transpose, the stabilisation C with the squared cell diameter) equals the
    tensor-product form; a dropped term, a wrong sign, a transposed block or a
    side length in place of the diameter fails it."""
    N = 6 if dim == 2 else 3
    coords = inputs.graded_coordinates(N, 3.0, dim) if graded else None
    o = q1_oracle(dim, N, coords=coords, eta0=1.7, beta=0.3)
    m, _ = o.dirichlet(0)
    xv = [np.linspace(0, 1, N + 1) if coords is None else coords[a] for a in range(dim)]
    want = tensor_operator(dim, xv, 1.7, 0.3, m)
    got = dense(o, 0)
    assert got.shape == want.shape
    assert np.abs(got - want).max() <= 1e-13 * np.abs(want).max()


@pytest.mark.parametrize("dim", [2, 3])
def test_linear_fields(dim):
    """Integration by parts on the discrete space: a linear divergence-free
    velocity with constant pressure leaves no residual on the free rows; a linear
    pressure g.x with zero velocity gives B^T p = g_c int phi_v on interior
    velocity rows (sign and scale of B), and C p = 0 on interior pressure rows
    of a uniform grid."""
    N = 6 if dim == 2 else 4
    o = q1_oracle(dim, N, bc=O.BC_NOSLIP, beta=0.3)
    L = dense(o, 0)
    m, _ = o.dirichlet(0)
    V = vertex_coords(dim, N)
    nv = len(V)
    nu = dim * nv
    G = np.array([[0.3, 1.1, -0.4], [0.7, -0.9, 2.0], [1.5, 0.2, 0.6]])[:dim, :dim]
    G[-1, -1] = -np.trace(G[:-1, :-1])  # divergence free
    x = np.zeros(nu + nv)
    x[:nu] = (V @ G.T).reshape(-1)
    x[nu:] = 0.25
    r = L @ x
    assert np.abs(r[:nu][~m[:nu]]).max() < 1e-12
    assert np.abs(r[nu:]).max() < 1e-12

    g = np.array([0.8, -1.3, 0.5])[:dim]
    x = np.zeros(nu + nv)
    x[nu:] = V @ g
    r = L @ x
    h = 1.0 / N
    vidx = vertex_index(dim, N)
    interior = np.all((vidx > 0) & (vidx < N), axis=1)
    for c in range(dim):
        rows = dim * np.nonzero(interior)[0] + c
        assert np.allclose(r[rows], g[c] * h ** dim, rtol=0, atol=1e-14)
    assert np.abs(r[nu:][interior]).max() < 1e-13


def _bordered_solve(L, b, nu):
    n = L.shape[0]
    e = np.zeros((n, 1))
    e[nu:] = 1.0
    K = sp.bmat([[sp.csr_matrix(L), sp.csr_matrix(e)], [sp.csr_matrix(e.T), None]]).tocsc()
    return sla.spsolve(K, np.concatenate([b, [0.0]]))[:n]


def test_quadratic_solution_converges_at_textbook_rates():
    """u = (y^2, x^2), p = x + y - 1 (forcing and boundary data of the quadratic
    solution): with the pressure stabilisation the nodal velocity error falls
    like h^2 and the pressure error like h (the stabilisation is not consistent
    for a non-constant pressure gradient)."""
    errs = []
    for N in (8, 16, 32):
        o = q1_oracle(2, N, bc=O.BC_QUADRATIC)
        L = o.matrix(0)
        nu = o.sizes(0)["n_u"]
        x = _bordered_solve(L, o.rhs(3), nu)
        V = vertex_coords(2, N)
        u = x[:nu].reshape(-1, 2)
        ue = np.stack([V[:, 1] ** 2, V[:, 0] ** 2], 1)
        p, pe = x[nu:] - x[nu:].mean(), V.sum(1) - 1.0
        pe -= pe.mean()
        errs.append((np.abs(u - ue).max(), np.abs(p - pe).max()))
    for (eu0, ep0), (eu1, ep1) in zip(errs, errs[1:]):
        assert 3.5 < eu0 / eu1 < 4.5
        assert 1.7 < ep0 / ep1 < 2.3
    assert errs[-1][0] < 1e-4


def test_without_stabilisation_the_pair_is_unstable():
    """beta = 0 leaves the spurious pressure modes of the equal-order pair (the
    reason for Eq. 8): the bordered system is singular or its pressure is far
    off, while any beta > 0 gives an O(h) pressure."""
    N = 8
    o = q1_oracle(2, N, bc=O.BC_QUADRATIC, beta=0.0)
    L = o.matrix(0).toarray()
    nu = o.sizes(0)["n_u"]
    m, _ = o.dirichlet(0)
    free = np.concatenate([~m[:nu], np.ones(L.shape[0] - nu, bool)])
    Lf = L[np.ix_(free, free)]
    sv = np.linalg.svd(Lf, compute_uv=False)
    assert (sv < 1e-10 * sv[0]).sum() >= 2  # constant + checkerboard pressure modes
    o = q1_oracle(2, N, bc=O.BC_QUADRATIC, beta=BETA)
    L = o.matrix(0).toarray()
    sv = np.linalg.svd(L[np.ix_(free, free)], compute_uv=False)
    assert (sv < 1e-10 * sv[0]).sum() == 1  # the constant pressure only


@pytest.mark.parametrize("dim,N", [(2, 5), (3, 4)])
def test_subdomains_and_ownership(dim, N):
    """S_i = {p_i} + the free velocity DoFs of row i of B (Sec. 3); interior
    subdomains hold 3^d d + 1 DoFs; the owned (restricted) set is exactly the
    velocity DoFs of vertex i and p_i (Eq. 13), a partition of the free DoFs."""
    o = q1_oracle(dim, N)
    o.build_patches(0)
    off, dofs, own = o.patches(0)
    rp, ci, va = o.csr(0)
    m, _ = o.dirichlet(0)
    nu = o.sizes(0)["n_u"]
    for i in range((N + 1) ** dim):
        row = ci[rp[nu + i]:rp[nu + i + 1]]
        row = row[row < nu]
        want = np.sort(np.concatenate([row[~m[row]], [nu + i]]))
        assert np.array_equal(dofs[off[i]:off[i + 1]], want)
        s = dofs[off[i]:off[i + 1]]
        mine = s[own[s] == i]
        vel = [dim * i + c for c in range(dim) if not m[dim * i + c]]
        assert np.array_equal(mine, np.array(vel + [nu + i], np.int64))
    assert np.diff(off).max() == 3 ** dim * dim + 1
    count = np.zeros(len(own), int)
    for i in range(len(off) - 1):
        s = dofs[off[i]:off[i + 1]]
        count[s[own[s] == i]] += 1
    assert np.all(count[~m] == 1) and np.all(count[m] == 0)


@pytest.mark.parametrize("dim,N", [(2, 4), (2, 6), (3, 4)])
def test_rav_step_equals_assembled_operator(dim, N):
    """x + S_RAV (b - L x), S_RAV = sum_i Rt_i^T w_i L_i^{-1} R_i (Eq. 13) on the
    stabilised Q1-Q1 operator, with numpy.linalg.inv and per-subdomain damping."""
    blobs = inputs.viscosity_blobs(11, k=3, s_max=1.0)
    o = q1_oracle(dim, N, nlev=2, blobs=blobs)
    o.setup_smoother(O.RAV, 0.66)
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


@pytest.mark.parametrize("dim,graded", [(2, False), (2, True), (3, True)])
def test_prolongation_reproduces_coarse_multilinear_fields(dim, graded):
    """P maps the coarse interpolant of random multilinear velocity and pressure
    fields to the fine interpolant (nested Q1 spaces); fine Dirichlet rows are empty."""
    N = 8 if dim == 2 else 4
    coords = inputs.graded_coordinates(N, 3.0, dim) if graded else None
    o = q1_oracle(dim, N, nlev=2, coords=coords, bc=O.BC_NOSLIP)
    rng = np.random.default_rng(6)
    cu = rng.standard_normal((dim,) + (2,) * dim)
    cp = rng.standard_normal((2,) * dim)

    def poly(X, coef):
        out = np.zeros(len(X))
        for idx in np.ndindex(coef.shape):
            out += coef[idx] * np.prod([X[:, a] ** idx[a] for a in range(dim)], axis=0)
        return out

    def field(n, cds):
        V = vertex_coords(dim, n, cds)
        u = np.stack([poly(V, cu[c]) for c in range(dim)], -1).reshape(-1)
        return np.concatenate([u, poly(V, cp)])

    xc = field(N // 2, None if coords is None else coords[:, ::2])
    xf = field(N, coords)
    m, _ = o.dirichlet(1)
    got = o.prolong_add(1, xc, np.zeros_like(xf))
    assert np.abs(got[~m] - xf[~m]).max() < 1e-12 * np.abs(xf).max()
    assert np.all(got[m] == 0.0)
    # restriction is the adjoint on the free DoFs
    mc, _ = o.dirichlet(0)
    xc[mc] = 0.0
    rf = rng.standard_normal(len(xf))
    rf[m] = 0.0
    lhs = o.prolong_add(1, xc, np.zeros_like(xf)) @ rf
    assert abs(lhs - xc @ o.restrict(1, rf)) < 1e-12 * abs(lhs)


@pytest.mark.parametrize("dim,N", [(2, 8), (3, 4)])
def test_factored_storage_with_a_pressure_block(dim, N):
    """The factored rows (A^{-1}, w = A^{-1} b, 1/s with s = c - b^T w, c the
    stabilisation's diagonal entry) rebuild the owned rows of L_i^{-1} up to
    the format's rounding; leaving c out of s would leave an O(1) error."""
    blobs = inputs.viscosity_blobs(3, k=6, s_max=2.0)
    exact = q1_oracle(dim, N, nlev=2, blobs=blobs, bc=O.BC_NOSLIP, beta=0.3)
    exact.setup_smoother(O.RAV, 0.66)
    for prec, bound in ((O.F32_FACT, 2.0 ** -23), (O.BF16_FACT, 2.0 ** -7)):
        o = q1_oracle(dim, N, nlev=2, blobs=blobs, bc=O.BC_NOSLIP, beta=0.3)
        o.setup_smoother(O.RAV, 0.66, prec)
        worst = 0.0
        for p in range((N + 1) ** dim):
            rows = exact.inverse(1, p)
            q, _ = o.inverse(1, p, quantised=True)
            worst = max(worst, np.abs(q - rows).max() / np.abs(rows).max())
        assert 0.0 < worst <= bound, (prec, worst)


def test_rav_multigrid_converges_on_the_cavity():
    """RAV(omega = 0.66, the paper's damping for Q1-Q1) V(2,2)-cycles reach the
    1e-8 reduction on the 2-D cavity, as stationary iteration and as FGMRES
    preconditioner, and the result solves the bordered system."""
    o = q1_oracle(2, 32, nlev=4)
    o.check_coarse()
    o.setup_smoother(O.RAV, 0.66)
    b, x0 = o.rhs(0), o.initial_guess()
    x, it, hist = o.solve(x0, b, tol=1e-8, maxit=40)
    assert 0 < it <= 20 and hist[-1] <= 1e-8
    x2, it2, _ = o.fgmres(x0, b, tol=1e-8, maxit=40)
    assert 0 < it2 <= it
    nu = o.sizes(3)["n_u"]
    ref = _bordered_solve(o.matrix(3), b, nu)
    for y in (x, x2):
        du = np.abs(y[:nu] - ref[:nu]).max()
        dp = np.abs((y[nu:] - y[nu:].mean()) - (ref[nu:] - ref[nu:].mean())).max()
        assert du < 1e-6 and dp < 1e-5


@pytest.mark.parametrize("dim,N", [(2, 4), (3, 3)])
def test_av_step_equals_assembled_operator(dim, N):
    """x + S_AV (b - L x), S_AV = sum_i R_i^T w L_i^{-1} R_i (Eq. 12), on the
    stabilised Q1-Q1 subdomains."""
    blobs = inputs.viscosity_blobs(17, k=3, s_max=1.0)
    o = q1_oracle(dim, N, nlev=2, blobs=blobs)
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
    """Multiplicative Vanka on Q1-Q1: the error propagates as
    prod_i (I - w R_i^T L_i^{-1} R_i L) in the sweep order (lexicographic, or
    coloured by (v mod 4) with colours ascending)."""
    dim, N = 2, 4
    o = q1_oracle(dim, N, nlev=2, blobs=inputs.viscosity_blobs(18, k=3, s_max=1.0))
    o.setup_smoother(kind, 0.66)
    off, dofs, own = o.patches(1)
    L = dense(o, 1)
    m, _ = o.dirichlet(1)
    n = L.shape[0]
    order = np.arange(len(off) - 1)
    if kind == O.MV_COLOURED:
        v = vertex_index(dim, N)
        order = np.argsort((v[:, 0] % 4) + 4 * (v[:, 1] % 4), kind="stable")
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
    assert np.abs(got - E @ e0).max() <= 1e-11 * np.abs(e0).max()


def test_single_global_subdomain_solves_exactly():
    """One subdomain holding every free DoF but one pressure (which fixes the
    constant-pressure kernel of the all-Dirichlet problem), owning all of them,
    with unit damping: one RAV step solves L x = b on those DoFs exactly."""
    N = 4
    o = q1_oracle(2, N, nlev=2)
    o.setup_smoother(O.RAV, 1.0)
    L = dense(o, 1)
    m, g = o.dirichlet(1)
    n = L.shape[0]
    nu = o.sizes(1)["n_u"]
    free = np.nonzero(~m)[0]
    keep = free[free != nu]  # pin p_0
    off = np.array([0, len(keep)], np.int64)
    owner = np.full(n, -1, np.int64)
    owner[keep] = 0
    o.set_patches(1, off, keep.astype(np.int64), owner, 1.0)
    rng = np.random.default_rng(9)
    xs = rng.standard_normal(n)
    xs[m] = g[m]
    xs[nu] = 0.0
    b = L @ xs
    b[m] = g[m]
    x0 = np.zeros(n)
    x0[m] = g[m]
    got = o.smooth(1, x0, b)
    assert np.abs(got - xs).max() <= 1e-10 * np.abs(xs).max()


def test_dof_count_equals_the_papers_table():
    """The paper's Table 1 row Omega_h^1 (64 elements, 243 DoFs) is a uniform
    8x8 Q1-Q1 grid counted with every DoF: the oracle's Q1-Q1 hierarchy on it
    has exactly 243 DoFs (162 velocity + 81 pressure)."""
    from test_oracle import read_golden
    g = read_golden("dof_counts.txt")
    o = q1_oracle(2, 8)
    s = o.sizes(0)
    assert 8 * 8 == g["table1_omega1_elements"]
    assert s["n"] == g["table1_omega1_q1q1_dofs"] and s["n_u"] == 162 and s["n_p"] == 81
