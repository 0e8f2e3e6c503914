"""Pins of the oracle's single-patch preconditioner B(1) (Section 4.1): the whole
domain as one patch, i.e. one element-structured V(1,1) cycle on K_h with ILU(0)
smoothing and R_0 at the vertex level."""
import os

import numpy as np
import pytest

from oracle import cg, krylov, lor as olor
from oracle.mesh import Mesh
from oracle.single_patch import SinglePatchPreconditioner, grid_pattern, ilu0_csr
from paper_1908_07071_gb300.synthetic import make_mesh

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _paper_table2():
    t = {}
    for line in open(os.path.join(GOLDEN, "table2_single_patch.txt")):
        if line.startswith("#") or not line.strip():
            continue
        vals = [int(s) for s in line.split()]
        for c, nx in enumerate([2, 4, 8, 16, 32]):
            t[(vals[0], nx)] = vals[c + 1]
    return t


def _cartesian(nx, p):
    v, k = make_mesh(2, nx, seed=0, perturb=0.0, kappa_const=1.0)
    m = Mesh(v, k)
    N = cg.node_shape(m.n, p)
    K = cg.assemble_stiffness(m, p)
    f = lambda X: 2 * np.pi ** 2 * np.sin(np.pi * X[:, 0]) * np.sin(np.pi * X[:, 1])  # noqa: E731
    return m, N, K, cg.load_vector(m, p, f)


@pytest.mark.parametrize("p,nx", [(4, 2), (4, 4), (4, 8), (6, 2), (6, 4), (6, 8), (8, 2), (8, 4), (8, 8)])
def test_single_patch_counts_match_table2(p, nx):
    """Table 2 (Section 4.1): within one iteration of the paper's counts, although the
    ordering (lexicographic vs MDF) and R_0 (own V-cycle vs BoomerAMG) differ."""
    paper = _paper_table2()[(p, nx)]
    m, N, K, b = _cartesian(nx, p)
    B = SinglePatchPreconditioner(m, p)
    it = krylov.pcg(lambda u: cg.apply_A(K, N, u), B.apply, b, rtol=1e-8)[1]
    assert abs(it - paper) <= 1, (it, paper)


@pytest.mark.parametrize("nx", [2, 4, 8])
def test_single_patch_p2_magnitude(nx):
    paper = _paper_table2()[(2, nx)]
    m, N, K, b = _cartesian(nx, 2)
    it = krylov.pcg(lambda u: cg.apply_A(K, N, u), SinglePatchPreconditioner(m, 2).apply, b, rtol=1e-8)[1]
    assert 0.5 * paper <= it <= 2.0 * paper, (it, paper)


def test_vertex_patches_need_more_iterations_than_one_patch():
    """Section 4.1: with vertex patches the counts grow (about twice those of one
    patch per domain in the paper's tables)."""
    for p, nx in ((4, 4), (6, 4), (8, 4)):
        m, N, K, b = _cartesian(nx, p)
        A = lambda u: cg.apply_A(K, N, u)  # noqa: E731
        it1 = krylov.pcg(A, SinglePatchPreconditioner(m, p).apply, b, rtol=1e-8)[1]
        itv = krylov.pcg(A, olor.LORPreconditioner(m, p).apply, b, rtol=1e-8)[1]
        assert 1.2 * it1 <= itv <= 2.5 * it1, (p, it1, itv)


def test_single_patch_is_symmetric_positive_definite():
    v, k = make_mesh(2, 3, seed=1, perturb=0.15)
    m = Mesh(v, k)
    p = 3
    B = SinglePatchPreconditioner(m, p)
    N = cg.node_shape(m.n, p)
    inner = ~cg.boundary_mask(N).ravel()
    n = inner.sum()
    E = np.zeros((len(inner), n))
    E[np.nonzero(inner)[0], np.arange(n)] = 1.0
    M = np.column_stack([B.apply(E[:, c])[inner] for c in range(n)])
    assert np.abs(M - M.T).max() <= 1e-12 * np.abs(M).max()
    assert np.linalg.eigvalsh(0.5 * (M + M.T)).min() > 0


def test_sparse_ilu0_matches_the_dense_ilu0_of_a_patch():
    v, k = make_mesh(3, 2, seed=2, perturb=0.15)
    m = Mesh(v, k)
    B = olor.LORPreconditioner(m, 3, coarse=False, patch_subset=[(1, 1, 1)])
    lev = B.patches[0]["levels"][0]
    A, pat = lev["A"], olor.box_pattern(lev["ranges"])
    Ld, Ud = olor.ilu0(A, pat)
    Ls, Us = ilu0_csr(A, pat)
    assert np.allclose(Ls.toarray(), Ld, atol=1e-13) and np.allclose(Us.toarray(), Ud, atol=1e-13 * np.abs(A).max())


def test_grid_pattern_is_the_3d_point_stencil():
    P = grid_pattern((4, 3, 5)).toarray()
    idx = np.array([(i, j, k) for k in range(5) for j in range(3) for i in range(4)])
    ref = np.all(np.abs(idx[:, None, :] - idx[None, :, :]) <= 1, axis=2)
    assert np.array_equal(P, ref)


def test_hybrid_schwarz_is_spd_and_close_to_additive():
    """Coarse correction applied multiplicatively (symmetric hybrid form): symmetric
    positive definite without damping, and about as effective as the additive form."""
    v, k = make_mesh(2, 3, seed=1, perturb=0.15)
    m = Mesh(v, k)
    p = 3
    B = olor.LORPreconditioner(m, p)
    N = cg.node_shape(m.n, p)
    inner = ~cg.boundary_mask(N)
    n = inner.sum()
    E = np.zeros((len(inner), n))
    E[np.nonzero(inner)[0], np.arange(n)] = 1.0
    M = np.column_stack([B.apply_hybrid(E[:, c])[inner] for c in range(n)])
    assert np.abs(M - M.T).max() <= 1e-12 * np.abs(M).max()
    assert np.linalg.eigvalsh(0.5 * (M + M.T)).min() > 0
    for nx, p in ((4, 4), (6, 4)):
        v, k = make_mesh(2, nx, seed=0, perturb=0.15)
        m = Mesh(v, k)
        N = cg.node_shape(m.n, p)
        K = cg.assemble_stiffness(m, p)
        b = cg.load_vector(m, p, lambda X: np.ones(len(X)))
        B = olor.LORPreconditioner(m, p)
        A = lambda u: cg.apply_A(K, N, u)  # noqa: E731
        ita = krylov.pcg(A, B.apply, b, rtol=1e-8)[1]
        ith = krylov.pcg(A, B.apply_hybrid, b, rtol=1e-8)[1]
        assert abs(ith - ita) <= 0.15 * ita, (ita, ith)


@pytest.mark.parametrize("dim,n,p", [(2, 3, 4), (3, 2, 3), (3, 3, 2)])
def test_count_weights_closed_form(dim, n, p):
    """The patch count of a node is 2 per axis along which it lies strictly inside an
    element and 1 per axis on a vertex plane (the form the GPU kernel evaluates),
    checked against the oracle's enumeration of the patches."""
    v, k = make_mesh(dim, n, seed=0, perturb=0.15)
    B = olor.LORPreconditioner(Mesh(v, k), p, weighting="count", coarse=False)
    N = cg.node_shape(B.mesh.n, p)
    idx = np.array(np.unravel_index(np.arange(int(np.prod(N))), tuple(reversed(N)))[::-1]).T
    c = np.sum(idx % p != 0, axis=1)
    inner = ~cg.boundary_mask(N)
    closed = np.where(inner, 1.0 / np.sqrt(2.0 ** c), 0.0)
    assert np.allclose(B.count_weights(), closed, atol=1e-15)


def test_count_weighting_is_spd_and_reduces_iterations():
    """Counting-matrix weighting (D^{-1/2} on both sides of the patch sum): SPD, and
    far fewer iterations than unit weights on a perturbed 3D mesh with log-normal b."""
    v, k = make_mesh(3, 3, seed=0, perturb=0.15)
    m = Mesh(v, k)
    p = 3
    N = cg.node_shape(m.n, p)
    K = cg.assemble_stiffness(m, p)
    b = cg.load_vector(m, p, lambda X: np.ones(len(X)))
    A = lambda u: cg.apply_A(K, N, u)  # noqa: E731
    it1 = krylov.pcg(A, olor.LORPreconditioner(m, p).apply, b, rtol=1e-8)[1]
    Bw = olor.LORPreconditioner(m, p, weighting="count")
    itw = krylov.pcg(A, Bw.apply, b, rtol=1e-8)[1]
    assert itw <= 0.6 * it1, (it1, itw)
    v2, k2 = make_mesh(2, 3, seed=1, perturb=0.15)
    m2 = Mesh(v2, k2)
    B2 = olor.LORPreconditioner(m2, 3, weighting="count")
    N2 = cg.node_shape(m2.n, 3)
    inner = ~cg.boundary_mask(N2)
    n = inner.sum()
    E = np.zeros((len(inner), n))
    E[np.nonzero(inner)[0], np.arange(n)] = 1.0
    M = np.column_stack([B2.apply(E[:, c])[inner] for c in range(n)])
    assert np.abs(M - M.T).max() <= 1e-12 * np.abs(M).max()
    assert np.linalg.eigvalsh(0.5 * (M + M.T)).min() > 0


def test_count_weighting_gain_reverses_at_high_degree_in_2d():
    """The counting-weight gain shrinks with p: on a Cartesian 4 x 4 mesh it helps at p = 4
    and costs iterations at p = 16 (the weighted decomposition is not p-robust)."""
    v, k = make_mesh(2, 4, seed=0, perturb=0.0, kappa_const=1.0)
    m = Mesh(v, k)
    its = {}
    for p in (4, 16):
        N = cg.node_shape(m.n, p)
        K = cg.assemble_stiffness(m, p)
        b = cg.load_vector(m, p, lambda X: np.ones(len(X)))
        A = lambda u: cg.apply_A(K, N, u)  # noqa: E731
        for w in ("none", "count"):
            its[p, w] = krylov.pcg(A, olor.LORPreconditioner(m, p, weighting=w).apply, b, rtol=1e-8)[1]
    assert its[4, "count"] <= 0.75 * its[4, "none"], its
    assert its[16, "count"] > its[16, "none"], its


@pytest.mark.parametrize("dim,n,p", [(2, 3, 4), (3, 2, 3)])
def test_pou_weights_are_a_partition_of_unity_and_b_is_spd(dim, n, p):
    """weighting="pou": sum_j W_j^2 = 1 at every interior node (the Q1 vertex functions
    sum to one and vanish on each patch boundary); B stays symmetric positive definite."""
    v, k = make_mesh(dim, n, seed=0, perturb=0.15)
    m = Mesh(v, k)
    B = olor.LORPreconditioner(m, p, weighting="pou")
    s = np.zeros(int(np.prod(B.Ns[0])))
    for j, pt in enumerate(B.patches):
        idx = pt["levels"][0]["idx"]
        if len(idx):
            w = B.pou_weights(j)
            assert np.all(w > 0)
            s[idx] += w ** 2
    inner = ~cg.boundary_mask(B.Ns[0])
    np.testing.assert_allclose(s[inner], 1.0, atol=1e-14)
    if dim == 2:
        idx = np.nonzero(inner)[0]
        E = np.zeros((len(inner), len(idx)))
        E[idx, np.arange(len(idx))] = 1.0
        M = np.column_stack([B.apply(E[:, c])[inner] for c in range(len(idx))])
        assert np.abs(M - M.T).max() <= 1e-12 * np.abs(M).max()
        assert np.linalg.eigvalsh(0.5 * (M + M.T)).min() > 0


def test_pou_weighting_is_p_robust_in_2d_and_beats_counting_weights_in_3d():
    """Measured: Cartesian 4 x 4, p = 4 / 16: unit 25 / 39, counting 16 / 47, pou 16 / 23;
    perturbed 3D Q4 on 3^3 with log-normal b: unit 66, counting 29, pou 27."""
    v, k = make_mesh(2, 4, seed=0, perturb=0.0, kappa_const=1.0)
    m = Mesh(v, k)
    its = {}
    for p in (4, 16):
        N = cg.node_shape(m.n, p)
        K = cg.assemble_stiffness(m, p)
        b = cg.load_vector(m, p, lambda X: np.ones(len(X)))
        A = lambda u: cg.apply_A(K, N, u)  # noqa: E731
        its[p] = krylov.pcg(A, olor.LORPreconditioner(m, p, weighting="pou").apply, b, rtol=1e-8)[1]
    assert its[16] <= 1.6 * its[4], its
    v, k = make_mesh(3, 3, seed=0, perturb=0.15)
    m = Mesh(v, k)
    p = 4
    N = cg.node_shape(m.n, p)
    K = cg.assemble_stiffness(m, p)
    b = cg.load_vector(m, p, lambda X: np.ones(len(X)))
    A = lambda u: cg.apply_A(K, N, u)  # noqa: E731
    got = {w: krylov.pcg(A, olor.LORPreconditioner(m, p, weighting=w).apply, b, rtol=1e-8)[1]
           for w in ("none", "count", "pou")}
    assert got["pou"] <= got["count"] and got["pou"] <= 0.5 * got["none"], got


@pytest.mark.parametrize("dim,n,p", [(2, (3, 4), 4), (3, 2, 3), (3, (2, 3, 2), 1)])
def test_pou_weight_table_indexing(dim, n, p):
    """The patch kernel evaluates the partition-of-unity weight of node I in the patch of
    vertex v as sqrt(prod_a hat[(2 - v_a) p + I_a]), where hat is the coarse-space table
    of the library: hat[p + t] is the vertex function at position t = 1 .. 2p-1 of the
    two elements around a vertex (x_t rising, then 1 - x_{t-p} falling).  That index
    arithmetic, written out here, must give the oracle's pou_weights on every patch."""
    from oracle.basis import gll
    v, k = make_mesh(dim, n, seed=0, perturb=0.15)
    B = olor.LORPreconditioner(Mesh(v, k), p, weighting="pou", coarse=False)
    x = gll(p)[0]
    hat = np.zeros(3 * p)
    hat[:p + 1] = x
    for t in range(1, 2 * p):
        hat[p + t] = x[t] if t <= p else 1.0 - x[t - p]
    for j, pt in enumerate(B.patches):
        ranges = pt["levels"][0]["ranges"]
        if not all(len(r) for r in ranges):
            continue
        idx = [(2 - pt["v"][a]) * p + ranges[a] for a in range(dim)]
        assert all(ix.min() >= p + 1 and ix.max() <= 3 * p - 1 for ix in idx)
        grids = np.meshgrid(*[hat[ix] for ix in reversed(idx)], indexing="ij")
        w = np.sqrt(np.prod([g.ravel() for g in grids], axis=0))
        np.testing.assert_allclose(w, B.pou_weights(j), atol=1e-15)


@pytest.mark.parametrize("dim,n,p", [(2, (3, 4), 5), (3, 2, 4)])
def test_pou_weights_are_square_roots_of_the_coarse_basis(dim, n, p):
    """theta_j is the vertex function of patch j, i.e. column j of P_0 (built separately,
    by tensor linear interpolation), so W_j = sqrt(P_0[idx_j, j])."""
    v, k = make_mesh(dim, n, seed=2, perturb=0.15)
    B = olor.LORPreconditioner(Mesh(v, k), p, weighting="pou")
    P0 = B.P0.toarray()
    for j, pt in enumerate(B.patches):
        idx = pt["levels"][0]["idx"]
        if len(idx):
            np.testing.assert_allclose(B.pou_weights(j), np.sqrt(P0[idx, j]), atol=1e-14)


def test_pou_weighted_vertex_patches_close_the_gap_to_one_patch():
    """Section 4.1 reports vertex patches needing about twice the iterations of one patch
    B(1).  Measured (Cartesian 4 x 4, Q4): B(1) 15, vertex patches with unit weights 25,
    with partition-of-unity weights 16: the gap is the unit-weight overlap sum."""
    v, k = make_mesh(2, 4, seed=0, perturb=0.0, kappa_const=1.0)
    m = Mesh(v, k)
    p = 4
    K = cg.assemble_stiffness(m, p)
    N = cg.node_shape(m.n, p)
    b = cg.load_vector(m, p, lambda X: np.ones(len(X)))
    A = lambda u: cg.apply_A(K, N, u)  # noqa: E731
    one = krylov.pcg(A, SinglePatchPreconditioner(m, p).apply, b, rtol=1e-8)[1]
    unit = krylov.pcg(A, olor.LORPreconditioner(m, p).apply, b, rtol=1e-8)[1]
    pou = krylov.pcg(A, olor.LORPreconditioner(m, p, weighting="pou").apply, b, rtol=1e-8)[1]
    assert unit >= 1.5 * one and pou <= 1.2 * one, (one, unit, pou)


def test_smoother_comparison_on_the_gll_refined_mesh():
    """Section 3.4: pointwise smoothers degrade on the anisotropic GLL-refined mesh as p
    grows, ordered ILU(0) does not.  Measured (B(1), Cartesian 4 x 4), p = 4 / 12: ILU 15 / 19,
    Jacobi 15 / 32, Gauss-Seidel 17 / 26, line Jacobi 16 / 28, line Gauss-Seidel 16 / 23."""
    from oracle.single_patch import SMOOTHERS
    v, k = make_mesh(2, 4, seed=0, perturb=0.0, kappa_const=1.0)
    m = Mesh(v, k)
    its = {}
    for p in (4, 12):
        N = cg.node_shape(m.n, p)
        K = cg.assemble_stiffness(m, p)
        b = cg.load_vector(m, p, lambda X: np.ones(len(X)))
        A = lambda u: cg.apply_A(K, N, u)  # noqa: E731
        for s in SMOOTHERS:
            its[s, p] = krylov.pcg(A, SinglePatchPreconditioner(m, p, smoother=s).apply, b, rtol=1e-8)[1]
    assert all(its["ilu", 12] <= its[s, 12] for s in SMOOTHERS), its
    assert its["jacobi", 12] >= 1.8 * its["jacobi", 4] and its["ilu", 12] <= 1.4 * its["ilu", 4], its
