"""Pins of the oracle's element-structured patch hierarchy and V(1,1) cycle (Section 3.3).

Three facts fixed by the mathematics, each checked on interior, edge and corner
patches of distorted 2D and 3D meshes:

* the 1D prolongation interpolates linearly in the element reference coordinate, so
  it reproduces constants and the reference coordinate itself;
* the patch blocks of the global Galerkin levels are Galerkin on the patch: a coarse
  hat function of an interior patch node vanishes on the patch boundary, so
  P_j^T A_j^l P_j = A_j^{l+1} with P_j the patch block of the global prolongation;
* the coarse-space basis P_0 (Section 3.2) is Q1 on each element of T_p evaluated at
  the GLL nodes, and each coordinate of the multilinear element map is such a Q1
  function, so P_0 maps the vertex coordinates onto the node coordinates;
* the V(1,1) cycle with ILU(0) smoother M_l = L_l U_l and an exact solve on the
  vertex level has the textbook error propagation
  I - V_l A_l = (I - M_l^{-1} A_l)(I - P_l V_{l+1} P_l^T A_l)(I - M_l^{-1} A_l),
  V_last = A_last^{-1}; a dropped residual update, a restriction by P instead of
  P^T or a missing coarse correction all break it.
"""
import numpy as np
import pytest

from oracle import basis, cg, lor
from oracle.mesh import Mesh
from paper_1908_07071_gb300.synthetic import make_mesh


def _patches(dim, n, p, seed, mg=0):
    v, k = make_mesh(dim, n, seed=seed, perturb=0.15)
    B = lor.LORPreconditioner(Mesh(v, k), p, mg_levels=mg, coarse=False)
    return B


@pytest.mark.parametrize("p", [2, 3, 5, 8])
def test_prolongation_reproduces_linears_in_reference_coordinate(p):
    xg = basis.gll(p)[0]          # GLL points mapped to [0, 1]
    sels = lor.level_selections(p)
    nel = 3
    for l in range(len(sels) - 1):
        P = lor.prolong_1d(nel, p, sels[l], sels[l + 1])
        # reference coordinate (element index + local GLL point) on both grids
        xf = np.concatenate([[0.0]] + [e + xg[sels[l][1:]] for e in range(nel)])
        xc = np.concatenate([[0.0]] + [e + xg[sels[l + 1][1:]] for e in range(nel)])
        np.testing.assert_allclose(P @ np.ones(len(xc)), 1.0, atol=1e-14)
        np.testing.assert_allclose(P @ xc, xf, atol=1e-13)
        # kept points are injected, so every column has a unit entry
        assert np.all(np.isclose(P, 1.0).sum(axis=0) == 1)


@pytest.mark.parametrize("dim,n,p", [(2, 3, 6), (3, 2, 4), (3, 3, 3)])
def test_patch_levels_are_galerkin_on_the_patch(dim, n, p):
    B = _patches(dim, n, p, seed=3)
    checked = 0
    for pt in B.patches:
        lv = pt["levels"]
        for l in range(len(lv) - 1):
            A, P, Ac = lv[l]["A"], lv[l]["P"], lv[l + 1]["A"]
            if Ac.shape[0] == 0:
                continue
            scale = np.abs(A).max()
            np.testing.assert_allclose(P.T @ A @ P, Ac, atol=1e-12 * scale)
            checked += 1
    assert checked >= len(B.patches)


def _vcycle_matrix(B, levels, l):
    m = levels[l]["A"].shape[0]
    return np.column_stack([B.vcycle(levels, l, c) for c in np.eye(m)]) if m else np.zeros((0, 0))


@pytest.mark.parametrize("dim,n,p,mg", [(2, 3, 8, 0), (2, 2, 4, 2), (3, 2, 4, 0), (3, 2, 6, 0)])
def test_vcycle_error_propagation_is_the_textbook_product(dim, n, p, mg):
    B = _patches(dim, n, p, seed=5, mg=mg)
    corner = tuple([0] * dim)
    interior = tuple([1] * dim)
    for pt in B.patches:
        if pt["v"] not in (corner, interior):
            continue
        lv = pt["levels"]
        L = len(lv)
        A_last = lv[L - 1]["A"]
        V_next = np.linalg.inv(A_last) if A_last.shape[0] else np.zeros((0, 0))
        for l in range(L - 2, -1, -1):
            A, P = lv[l]["A"], lv[l]["P"]
            m = A.shape[0]
            Lf, Uf = lv[l]["LU"]
            S = np.eye(m) - np.linalg.solve(Lf @ Uf, A)
            C = np.eye(m) - P @ V_next @ P.T @ A
            E = S @ C @ S
            V = _vcycle_matrix(B, lv, l)
            np.testing.assert_allclose(np.eye(m) - V @ A, E, atol=1e-10)
            V_next = V
        # vertex level: an interior patch keeps its own vertex; the patch of a corner
        # vertex keeps none (its vertex is a Dirichlet node), so it has no coarse correction
        assert A_last.shape == ((1, 1) if pt["v"] == interior else (0, 0))


def test_vcycle_without_level0_post_smoothing_drops_the_last_factor():
    """post_smooth0=False (the cycle the learned correction's replace variant
    completes): the level-0 error propagation is (I - P V_1 P^T A)(I - M^{-1} A), the
    textbook product without its last factor, and the coarser levels are unchanged."""
    v, k = make_mesh(3, 2, seed=5, perturb=0.15)
    full = lor.LORPreconditioner(Mesh(v, k), 4, coarse=False)
    cut = lor.LORPreconditioner(Mesh(v, k), 4, coarse=False, post_smooth0=False)
    lv = [pt for pt in cut.patches if pt["v"] == (1, 1, 1)][0]["levels"]
    A, P = lv[0]["A"], lv[0]["P"]
    m = A.shape[0]
    Lf, Uf = lv[0]["LU"]
    S = np.eye(m) - np.linalg.solve(Lf @ Uf, A)
    V1 = _vcycle_matrix(full, lv, 1)
    np.testing.assert_allclose(_vcycle_matrix(cut, lv, 1), V1, atol=1e-12)
    E = (np.eye(m) - P @ V1 @ P.T @ A) @ S
    np.testing.assert_allclose(np.eye(m) - _vcycle_matrix(cut, lv, 0) @ A, E, atol=1e-10)
    assert np.abs(_vcycle_matrix(full, lv, 0) - _vcycle_matrix(cut, lv, 0)).max() > 1e-3


@pytest.mark.parametrize("dim,n,p", [(2, 3, 5), (3, 2, 4)])
def test_coarse_basis_maps_vertex_coordinates_to_node_coordinates(dim, n, p):
    v, k = make_mesh(dim, n, seed=7, perturb=0.2)
    m = Mesh(v, k)
    B = lor.LORPreconditioner(m, p, patch_subset=[])
    X = cg.node_coordinates(m, p)
    for a in range(dim):
        np.testing.assert_allclose(B.P0 @ m.vertices[a].ravel(), X[:, a], atol=1e-13)
    np.testing.assert_allclose(B.P0 @ np.ones(B.P0.shape[1]), 1.0, atol=1e-14)
    # without Dirichlet rows the coarse operator keeps the constants in its kernel
    A0 = (B.P0.T @ B.K_h @ B.P0).toarray()
    assert np.abs(A0 @ np.ones(A0.shape[0])).max() <= 1e-12 * np.abs(A0).max()


def _textbook_coarse(B, sweeps):
    """Error propagation I - V_l A_l of the coarse V-cycle (R_0, Section 3.2 with the
    l1-Jacobi reading), level by level from the coarsest: `sweeps` l1-Jacobi sweeps
    S = I - D^{-1} A with D the l1 row sums (D_ii = sum_j |A_ij|), the Galerkin coarse
    correction, `sweeps` more sweeps; the coarsest level solved exactly.  Returns
    the list of (A_l, E_l) from level 0 up."""
    out = []
    A_last = B.cA[-1].toarray()
    V_next = np.linalg.inv(A_last)
    for l in range(len(B.cA) - 2, -1, -1):
        A = B.cA[l].toarray()
        P = B.cP[l].toarray()
        m = A.shape[0]
        D = np.abs(A).sum(axis=1)
        S = np.eye(m) - A / D[:, None]
        C = np.eye(m) - P @ V_next @ P.T @ A
        Sk = np.linalg.matrix_power(S, sweeps)
        E = Sk @ C @ Sk
        out.append((A, E))
        V_next = np.linalg.solve(A, (np.eye(m) - E).T).T    # V = (I - E) A^{-1}
    return out[::-1]


def _coarse_vcycle_matrix(B, l):
    m = B.cA[l].shape[0]
    return np.column_stack([B.coarse_vcycle(l, c) for c in np.eye(m)])


@pytest.mark.parametrize("dim,n", [(2, 24), (3, 10)])
def test_coarse_vcycle_error_propagation_is_the_textbook_product(dim, n):
    """R_0 (Section 3.2, own V-cycle reading): on a vertex grid too large for the direct
    solve, the coarse levels are Galerkin (P^T A_l P = A_{l+1}), P interpolates linearly
    in the vertex index (constants and the index itself are reproduced on interior
    points), the coarsest level is small enough for the dense inverse while the level
    above it is not, and I - V_l A_l = S^2 (I - P V_{l+1} P^T A_l) S^2 with the l1-Jacobi
    S = I - D^{-1} A_l on every level."""
    v, k = make_mesh(dim, n, seed=11, perturb=0.15)
    B = lor.LORPreconditioner(Mesh(v, k), 2, patch_subset=[])
    assert len(B.cA) >= 2
    assert B.cA[-1].shape[0] <= lor.COARSE_DIRECT_MAX < B.cA[-2].shape[0]
    for l in range(len(B.cA) - 1):
        A, P, Ac = B.cA[l].toarray(), B.cP[l].toarray(), B.cA[l + 1].toarray()
        np.testing.assert_allclose(P.T @ A @ P, Ac, atol=1e-12 * np.abs(A).max())
    textbook = _textbook_coarse(B, sweeps=2)
    for l, (A, E) in enumerate(textbook):
        V = _coarse_vcycle_matrix(B, l)
        np.testing.assert_allclose(np.eye(A.shape[0]) - V @ A, E, atol=1e-10)


def test_coarse_prolongation_is_linear_interpolation_in_the_vertex_index():
    v, k = make_mesh(2, 24, seed=11, perturb=0.15)
    B = lor.LORPreconditioner(Mesh(v, k), 2, patch_subset=[])
    P = B.cP[0].toarray()
    # interior vertex indices of the fine (25 x 25) and coarse (13 x 13) vertex grids
    fi = np.arange(1, 24)
    ci = np.arange(1, 12)
    Xf = np.stack(np.meshgrid(fi, fi, indexing="xy"), -1).reshape(-1, 2).astype(float)
    Xc = 2.0 * np.stack(np.meshgrid(ci, ci, indexing="xy"), -1).reshape(-1, 2).astype(float)
    # a linear function of the vertex index that vanishes on the boundary of the coarse
    # grid's interior support is reproduced where all its coarse neighbours are interior
    inner = np.all((Xf >= 2) & (Xf <= 22), axis=1)
    for a in range(2):
        np.testing.assert_allclose((P @ Xc[:, a])[inner], Xf[inner, a], atol=1e-12)
    np.testing.assert_allclose((P @ np.ones(len(Xc)))[inner], 1.0, atol=1e-14)


def test_coarse_vcycle_pin_catches_planted_mistakes(monkeypatch):
    """The textbook product above fails for a cycle with one sweep instead of two, and for
    one that smooths with the plain diagonal instead of the l1 row sums."""
    v, k = make_mesh(2, 24, seed=11, perturb=0.15)
    B = lor.LORPreconditioner(Mesh(v, k), 2, patch_subset=[])
    (A, E), = _textbook_coarse(B, sweeps=2)[:1]
    monkeypatch.setattr(lor, "COARSE_SWEEPS", 1)
    V = _coarse_vcycle_matrix(B, 0)
    assert np.abs(np.eye(A.shape[0]) - V @ A - E).max() > 1e-3
    monkeypatch.setattr(lor, "COARSE_SWEEPS", 2)
    B.cDl1 = [Ai.diagonal().copy() for Ai in B.cA]
    V = _coarse_vcycle_matrix(B, 0)
    assert np.abs(np.eye(A.shape[0]) - V @ A - E).max() > 1e-3
