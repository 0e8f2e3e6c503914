"""Pins of the CPU oracle against facts the paper and mathematics fix (no GPU).

Each test ties an oracle function to something other than itself: closed-form
textbook values, exactness/invariance properties, the Kronecker forms of
Section 3.1, the additive-Schwarz bounds of Section 3.2, the manufactured
solution order, and the paper's printed iteration counts (Table 3).
"""
import os

import numpy as np
import pytest
import scipy.linalg as sla
import scipy.sparse.linalg as spla

from oracle import basis, cg, krylov, lor
from oracle.mesh import Mesh
from paper_1908_07071_gb300.synthetic import make_mesh, splitmix64, uniform01, normal

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ------------------------------------------------------------------ generator
def test_splitmix64_published_vectors():
    # SplitMix64 reference outputs (Steele-Lea-Flood; Vigna's splitmix64.c)
    assert int(splitmix64(0, 1)[0]) == 0xE220A8397B1DCDAF
    assert int(splitmix64(0, 2)[1]) == 0x6E789E6AA1B965F4
    assert int(splitmix64(1234567, 1)[0]) == 6457827717110365317


def test_generator_distributions():
    u = uniform01(5, 200000)
    assert 0.0 <= u.min() and u.max() < 1.0 and abs(u.mean() - 0.5) < 5e-3
    z = normal(9, 200000)
    assert abs(z.mean()) < 1e-2 and abs(z.std() - 1.0) < 1e-2


# ---------------------------------------------------------------------- basis
def _golden_gll():
    out = {}
    for line in open(os.path.join(GOLDEN, "gll_closed_forms.txt")):
        if line.startswith("#") or not line.strip():
            continue
        p, xs, ws = line.split("|")
        ev = lambda s: float(eval(s, {"sqrt": np.sqrt}))  # noqa: E731
        out[int(p)] = (np.array([ev(s) for s in xs.split()]), np.array([ev(s) for s in ws.split()]))
    return out


@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_gll_closed_forms(p):
    x, w = basis.gll(p)
    xr, wr = _golden_gll()[p]
    np.testing.assert_allclose(2 * x - 1, xr, atol=1e-15)
    np.testing.assert_allclose(2 * w, wr, rtol=1e-14)


@pytest.mark.parametrize("p", range(1, 11))
def test_gll_exactness(p):
    x, w = basis.gll(p)
    for k in range(2 * p):
        assert abs(w @ x ** k - 1.0 / (k + 1)) < 1e-14
    # GLL with p+1 points is not exact for degree 2p
    assert abs(w @ x ** (2 * p) - 1.0 / (2 * p + 1)) > 1e-12


@pytest.mark.parametrize("q", range(1, 11))
def test_gauss_exactness(q):
    x, w = basis.gauss_legendre(q)
    for k in range(2 * q):
        assert abs(w @ x ** k - 1.0 / (k + 1)) < 1e-14


@pytest.mark.parametrize("p", [1, 3, 6, 8])
def test_lagrange(p):
    xg = basis.gll(p)[0]
    B, D = basis.lagrange(xg, xg)
    np.testing.assert_allclose(B, np.eye(p + 1), atol=1e-14)
    t = np.linspace(0, 1, 7)
    B, D = basis.lagrange(xg, t)
    for k in range(p + 1):
        np.testing.assert_allclose(B @ xg ** k, t ** k, atol=1e-12)
        np.testing.assert_allclose(D @ xg ** k, k * t ** max(k - 1, 0) if k else 0 * t, atol=1e-10)


# ----------------------------------------------------------------- operators
def _textbook_p2(h):
    """1D quadratic FE stiffness and mass on [0,h] with nodes 0, h/2, h."""
    K = np.array([[7, -8, 1], [-8, 16, -8], [1, -8, 7]]) / (3.0 * h)
    M = np.array([[4, 2, -1], [2, 16, 2], [-1, 2, 4]]) * h / 30.0
    return K, M


def test_element_stiffness_kronecker_2d():
    # Section 3.1: K_p = sum_j (x)_i G_i^j on a tensor (affine) element
    hx, hy = 0.3, 0.7
    corners = np.array([[0, 0], [hx, 0], [0, hy], [hx, hy]], dtype=float)
    Kx, Mx = _textbook_p2(hx)
    Ky, My = _textbook_p2(hy)
    Kref = np.kron(My, Kx) + np.kron(Ky, Mx)
    np.testing.assert_allclose(cg.element_stiffness(corners, 1.0, 2), Kref, rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(cg.element_stiffness(corners, 2.5, 2), 2.5 * Kref, rtol=1e-12, atol=1e-12)


def test_element_stiffness_kronecker_3d():
    h = (0.2, 0.5, 0.9)
    corners = np.array([[(c & 1) * h[0], ((c >> 1) & 1) * h[1], ((c >> 2) & 1) * h[2]]
                        for c in range(8)], dtype=float)
    K = [_textbook_p2(v) for v in h]
    Kref = (np.kron(K[2][1], np.kron(K[1][1], K[0][0])) + np.kron(K[2][1], np.kron(K[1][0], K[0][1]))
            + np.kron(K[2][0], np.kron(K[1][1], K[0][1])))
    np.testing.assert_allclose(cg.element_stiffness(corners, 1.0, 2), Kref, rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("dim,n,p", [(2, 3, 4), (3, 2, 3)])
def test_linear_patch_test_and_constants(dim, n, p):
    """Linear functions are in Q_p on multilinear elements: K u = 0 on interior rows (b=1),
    and constants are in the kernel for any b (no Dirichlet)."""
    v, k = make_mesh(dim, n, seed=3, perturb=0.15, kappa_const=1.0)
    m = Mesh(v, k)
    N = cg.node_shape(m.n, p)
    X = cg.node_coordinates(m, p)
    interior = ~cg.boundary_mask(N)
    a = np.array([0.3, -1.1, 0.7][:dim])
    u = X @ a + 0.25
    for K in (cg.assemble_stiffness(m, p), lor.assemble_lor(m, p)):
        r = K @ u
        assert np.max(np.abs(r[interior])) < 1e-12 * np.max(np.abs(K.diagonal()))
    v, k = make_mesh(dim, n, seed=3, perturb=0.15)
    m = Mesh(v, k)
    for K in (cg.assemble_stiffness(m, p), lor.assemble_lor(m, p)):
        assert np.max(np.abs(K @ np.ones(K.shape[0]))) < 1e-12 * np.max(np.abs(K.diagonal()))
        assert abs(K - K.T).max() < 1e-13 * np.max(np.abs(K.diagonal()))


@pytest.mark.parametrize("dim", [2, 3])
def test_spd_after_dirichlet(dim):
    v, k = make_mesh(dim, 2, seed=1, perturb=0.15)
    m = Mesh(v, k)
    p = 3
    N = cg.node_shape(m.n, p)
    mask = ~cg.boundary_mask(N)
    for K in (cg.assemble_stiffness(m, p), lor.assemble_lor(m, p)):
        sla.cholesky(K[mask][:, mask].toarray())   # raises if not SPD


def test_apply_rows_matches_assembled():
    v, k = make_mesh(3, 2, seed=2, perturb=0.15)
    m = Mesh(v, k)
    p = 3
    N = cg.node_shape(m.n, p)
    K = cg.assemble_stiffness(m, p)
    x = np.random.default_rng(0).standard_normal(K.shape[0])
    y = cg.apply_A(K, N, x)
    rows = np.array([0, 5, 40, 100, 171, 342])
    np.testing.assert_allclose(cg.apply_A_rows(m, p, x, rows), y[rows], rtol=1e-12, atol=1e-12)


def test_manufactured_solution_order():
    """Eq. (poisson) with u = sin(pi x) sin(pi y): L2 error decays like h^(p+1)."""
    exact = lambda X: np.sin(np.pi * X[:, 0]) * np.sin(np.pi * X[:, 1])  # noqa: E731
    f = lambda X: 2 * np.pi ** 2 * exact(X)  # noqa: E731
    for p in (2, 3):
        errs = []
        for n in (2, 4, 8):
            v, k = make_mesh(2, n, seed=0, perturb=0.0, kappa_const=1.0)
            m = Mesh(v, k)
            N = cg.node_shape(m.n, p)
            K = cg.assemble_stiffness(m, p)
            b = cg.load_vector(m, p, f)
            mask = ~cg.boundary_mask(N)
            u = np.zeros(K.shape[0])
            u[mask] = spla.spsolve(K[mask][:, mask].tocsc(), b[mask])
            errs.append(cg.l2_error(m, p, u, exact))
        rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
        assert rates[-1] > p + 1 - 0.25, (p, rates)


# ----------------------------------------------------------------------- LOR
def _lin1d(pts):
    """Textbook 1D linear FE stiffness/mass on the (non-uniform) points."""
    m = len(pts)
    K = np.zeros((m, m))
    M = np.zeros((m, m))
    for i in range(m - 1):
        h = pts[i + 1] - pts[i]
        K[i:i + 2, i:i + 2] += np.array([[1, -1], [-1, 1]]) / h
        M[i:i + 2, i:i + 2] += np.array([[2, 1], [1, 2]]) * h / 6
    return K, M


def _cartesian_pts(n, p, sel):
    xg = basis.gll(p)[0]
    return np.concatenate([[0.0]] + [(e + xg[sel[1:]]) / n for e in range(n)])


@pytest.mark.parametrize("dim,p", [(2, 4), (3, 3)])
def test_lor_kronecker_and_galerkin_levels(dim, p):
    """K_h on a Cartesian grid is the Kronecker sum of 1D linear FE matrices on GLL points,
    and each Galerkin level equals the rediscretisation on the kept GLL subset."""
    n = 2
    v, k = make_mesh(dim, n, seed=0, perturb=0.0, kappa_const=1.0)
    m = Mesh(v, k)
    B = lor.LORPreconditioner(m, p)
    for l, sel in enumerate(B.sels):
        K1, M1 = _lin1d(_cartesian_pts(n, p, sel))
        if dim == 2:
            ref = np.kron(M1, K1) + np.kron(K1, M1)
        else:
            ref = (np.kron(M1, np.kron(M1, K1)) + np.kron(M1, np.kron(K1, M1))
                   + np.kron(K1, np.kron(M1, M1)))
        np.testing.assert_allclose(B.A[l].toarray(), ref, atol=1e-12)


def test_level_selections():
    sub = lambda p: [len(s) - 1 for s in lor.level_selections(p)]  # noqa: E731
    assert sub(2) == [2, 1]
    assert sub(3) == [3, 2, 1]
    assert sub(4) == [4, 2, 1]
    assert sub(6) == [6, 3, 2, 1]
    assert sub(7) == [7, 4, 2, 1]
    assert sub(8) == [8, 4, 2, 1]
    assert [len(s) - 1 for s in lor.level_selections(4, 2)] == [4, 1]


def test_fem_sem_equivalence_p_robust():
    """Proposition (fem-sem): the spectrum of K_h^{-1} K_p stays in a p-independent band.

    In 1D the stiffness ratio lies in [1, pi^2/4] and the exact-mass to linear-mass
    ratio in (1/2, 3); on a tensor grid the d-dimensional ratio is bounded by the
    products of these limits, whatever p is."""
    his, los = [], []
    for p in (2, 4, 8, 12):
        v, k = make_mesh(2, 2, seed=0, perturb=0.0, kappa_const=1.0)
        m = Mesh(v, k)
        N = cg.node_shape(m.n, p)
        mask = ~cg.boundary_mask(N)
        Kp = cg.assemble_stiffness(m, p)[mask][:, mask].toarray()
        Kh = lor.assemble_lor(m, p)[mask][:, mask].toarray()
        ev = sla.eigvalsh(Kp, Kh)
        los.append(ev[0])
        his.append(ev[-1])
    assert min(los) > 0.5 and max(his) < (np.pi ** 2 / 4) * 3.0, (los, his)
    # growth per unit of p slows down after the pre-asymptotic range
    slope = np.diff(his) / np.diff([2, 4, 8, 12])
    assert slope[-1] < 0.6 * slope[0], his


# --------------------------------------------------------------------- ILU(0)
def test_ilu0_properties():
    v, k = make_mesh(2, 2, seed=4, perturb=0.15)
    m = Mesh(v, k)
    B = lor.LORPreconditioner(m, 4)
    lev = B.patches[4]["levels"][0]          # interior vertex patch: 7x7
    A = lev["A"]
    pat = lor.box_pattern(lev["ranges"])
    L, U = lor.ilu0(A, pat)
    LU = L @ U
    np.testing.assert_allclose(LU[pat], A[pat], atol=1e-12 * np.abs(A).max())
    assert np.abs(LU - A)[~pat].max() > 0      # fill is dropped, so M != A
    D = np.diag(np.diag(U))
    np.testing.assert_allclose(U, D @ L.T, atol=1e-12 * np.abs(A).max())   # symmetric A
    # no fill (tridiagonal): ILU(0) is the exact LU
    T = np.diag(np.full(9, 2.0)) - np.diag(np.ones(8), 1) - np.diag(np.ones(8), -1)
    Lt, Ut = lor.ilu0(T, np.abs(T) > 0)
    np.testing.assert_allclose(Lt @ Ut, T, atol=1e-14)


def test_ilu0_breakdown():
    A = np.array([[1.0, 2.0], [2.0, 1.0]])
    with pytest.raises(FloatingPointError):
        lor.ilu0(A, np.ones((2, 2), dtype=bool))


# ---------------------------------------------------------- additive Schwarz
def _dense_B(B, mask, **kw):
    idx = np.nonzero(mask)[0]
    out = np.zeros((len(idx), len(idx)))
    e = np.zeros(len(mask))
    for c, i in enumerate(idx):
        e[:] = 0
        e[i] = 1
        out[:, c] = B.apply(e, **kw)[mask]
    return out


@pytest.mark.parametrize("dim,n,p", [(2, 3, 3), (3, 2, 2)])
def test_as_bounds_exact_solves(dim, n, p):
    """Section 3.2: with exact R_j and R_0, lambda_max(B K_h) <= 2^d + 1."""
    v, k = make_mesh(dim, n, seed=0, perturb=0.15)
    m = Mesh(v, k)
    B = lor.LORPreconditioner(m, p, exact_local=True, exact_coarse=True)
    mask = ~cg.boundary_mask(cg.node_shape(m.n, p))
    Bm = _dense_B(B, mask)
    Kh = B.K_h[mask][:, mask].toarray()
    ev = np.linalg.eigvals(Bm @ Kh).real
    assert ev.max() <= 2 ** dim + 1 + 1e-9
    assert ev.min() > 0.1
    np.testing.assert_allclose(Bm, Bm.T, atol=1e-12)
    # patches alone (no coarse space): at most 2^d overlapping patches per point
    Bp = _dense_B(B, mask, parts=("patches",))
    assert np.linalg.eigvals(Bp @ Kh).real.max() <= 2 ** dim + 1e-9


@pytest.mark.parametrize("dim,n,p,mg", [(2, 3, 4, 0), (2, 3, 4, 2), (3, 2, 3, 0)])
def test_vcycle_preconditioner_symmetric_spd(dim, n, p, mg):
    v, k = make_mesh(dim, n, seed=1, perturb=0.15)
    m = Mesh(v, k)
    B = lor.LORPreconditioner(m, p, mg_levels=mg)
    mask = ~cg.boundary_mask(cg.node_shape(m.n, p))
    Bm = _dense_B(B, mask)
    np.testing.assert_allclose(Bm, Bm.T, atol=1e-11 * np.abs(Bm).max())
    assert np.linalg.eigvalsh(0.5 * (Bm + Bm.T)).min() > 0
    # every patch V-cycle is a convergent iteration for its A_j
    for pt in B.patches:
        lev = pt["levels"][0]
        A = lev["A"]
        if A.shape[0] == 0:
            continue
        V = np.column_stack([B.vcycle(pt["levels"], 0, col) for col in np.eye(A.shape[0])])
        rho = np.abs(np.linalg.eigvals(np.eye(A.shape[0]) - V @ A)).max()
        assert rho < 0.6, rho


def test_coarse_vcycle_convergent():
    v, k = make_mesh(3, 10, seed=2, perturb=0.15)
    m = Mesh(v, k)
    B = lor.LORPreconditioner(m, 1)
    assert len(B.cA) >= 2                       # 729 > 343 unknowns: one V-cycle level
    A = B.cA[0].toarray()
    V = np.column_stack([B.coarse_solve(c) for c in np.eye(A.shape[0])])
    np.testing.assert_allclose(V, V.T, atol=1e-12 * np.abs(V).max())
    rho = np.abs(np.linalg.eigvals(np.eye(A.shape[0]) - V @ A)).max()
    assert rho < 0.7, rho


# ---------------------------------------------------------------- PCG solves
def test_pcg_matches_direct_solve():
    v, k = make_mesh(3, 2, seed=0, perturb=0.15)
    m = Mesh(v, k)
    p = 3
    N = cg.node_shape(m.n, p)
    K = cg.assemble_stiffness(m, p)
    b = cg.load_vector(m, p, lambda X: np.ones(len(X)))
    B = lor.LORPreconditioner(m, p)
    x, it, hist, _ = krylov.pcg(lambda u: cg.apply_A(K, N, u), B.apply, b, rtol=1e-12)
    mask = ~cg.boundary_mask(N)
    xd = np.zeros_like(b)
    xd[mask] = spla.spsolve(K[mask][:, mask].tocsc(), b[mask])
    assert np.linalg.norm(x - xd) / np.linalg.norm(xd) < 1e-10
    assert hist[-1] <= 1e-12 * np.linalg.norm(b)


def _paper_table3():
    t = {}
    for line in open(os.path.join(GOLDEN, "table3_vertex_patches.txt")):
        if line.startswith("#") or not line.strip():
            continue
        vals = [int(s) for s in line.split()]
        for c, nx in enumerate([2, 4, 8, 16, 32]):
            t[(vals[0], nx)] = vals[c + 1]
    return t


@pytest.mark.parametrize("p,nx", [(2, 2), (2, 4), (4, 2), (4, 4), (4, 8), (6, 4)])
def test_iteration_counts_vs_table3(p, nx):
    """Table 3 (Section 4.1): vertex-patch counts on the Cartesian grid.  Ordering and R_0
    differ (lexicographic ILU, own coarse V-cycle) and the paper does not state its
    right-hand side (the manufactured sin(pi x) sin(pi y) one is used), so only the
    magnitude is pinned."""
    paper = _paper_table3()[(p, nx)]
    v, k = make_mesh(2, nx, seed=0, perturb=0.0, kappa_const=1.0)
    m = Mesh(v, k)
    N = cg.node_shape(m.n, p)
    K = cg.assemble_stiffness(m, p)
    f = lambda X: 2 * np.pi ** 2 * np.sin(np.pi * X[:, 0]) * np.sin(np.pi * X[:, 1])  # noqa: E731
    b = cg.load_vector(m, p, f)
    B = lor.LORPreconditioner(m, p)
    _, it, _, _ = krylov.pcg(lambda u: cg.apply_A(K, N, u), B.apply, b, rtol=1e-8)
    assert 0.5 * paper <= it <= 2.0 * paper, (it, paper)


def test_iterations_bounded_in_h_and_p():
    """Corollary (as): counts stay bounded under h- and p-refinement (2D, perturbed, log-normal b)."""
    its = {}
    for p in (2, 4, 6):
        for nx in (2, 4, 8):
            v, k = make_mesh(2, nx, seed=0, perturb=0.15)
            m = Mesh(v, k)
            N = cg.node_shape(m.n, p)
            K = cg.assemble_stiffness(m, p)
            b = cg.load_vector(m, p, lambda X: np.ones(len(X)))
            B = lor.LORPreconditioner(m, p)
            its[(p, nx)] = krylov.pcg(lambda u: cg.apply_A(K, N, u), B.apply, b, rtol=1e-8)[1]
    assert max(its.values()) <= 45, its
    for p in (2, 4, 6):                       # h-refinement adds little
        assert its[(p, 8)] <= 1.35 * its[(p, 4)], its
    for nx in (4, 8):                         # p-refinement growth flattens
        assert its[(6, nx)] - its[(4, nx)] <= its[(4, nx)] - its[(2, nx)] + 2, its
