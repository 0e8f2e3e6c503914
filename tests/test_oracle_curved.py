"""Curved (isoparametric) elements in the oracle (the curved mesh of Section 4.2).

The element map is the degree-p interpolant of warp(multilinear(xi)) at the GLL points.
Pins: with an affine warp it is the (warped) multilinear map exactly; on one quarter of
the square-with-a-hole domain the mesh area converges to 1 - pi/64 and the boundary
nodes lie on the arc and on the outer square; linear functions pass the patch test
(in 2D the (p+1)-point Gauss rule integrates the isoparametric stiffness of a linear
function exactly); a manufactured solution that vanishes on the whole boundary
converges at order p+1 in L2; and the CG counts of the single patch and the vertex
patches have the magnitudes of Table 5 (golden file; the paper's mesh (b) is the full
unstructured square with a hole, the stand-in is one structured quarter of it, so this
is a magnitude check, not parity).
"""
import os

import numpy as np
import pytest
import scipy.sparse.linalg as spla

from oracle import cg, dg, krylov, lor
from oracle.basis import gauss_legendre
from oracle.mesh import Mesh, multilinear
from oracle.single_patch import SinglePatchPreconditioner
from paper_1908_07071_gb300.synthetic import make_mesh, make_quarter_hole_mesh, two_valued_kappa

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
R = 0.25


@pytest.mark.parametrize("dim,p", [(2, 3), (3, 2)])
def test_affine_warp_gives_the_warped_multilinear_map(dim, p):
    v, k = make_mesh(dim, 2, seed=1, perturb=0.15)
    rng = np.random.default_rng(0)
    A = np.eye(dim) + 0.3 * rng.standard_normal((dim, dim))
    c = rng.standard_normal(dim)
    m = Mesh(v, k, warp=lambda X: X @ A.T + c)
    xi = rng.random((7, dim))
    for e in m.elements():
        X, J = m.element_map(e, xi, p)
        X0, J0 = multilinear(m.corners(e), xi)
        np.testing.assert_allclose(X, X0 @ A.T + c, atol=1e-13)
        np.testing.assert_allclose(J, np.einsum("ab,qbc->qac", A, J0), atol=1e-12)


def _area(m, p):
    x1, w1 = gauss_legendre(p + 1)
    pts, w = cg.tensor_points(2, x1, w1)
    return sum(np.sum(w * np.abs(np.linalg.det(m.element_map(e, pts, p)[1]))) for e in m.elements())


def test_quarter_hole_area_and_boundary_nodes():
    exact = 1.0 - np.pi * R * R / 4
    errs = []
    for n in (2, 4, 8):
        v, k, w = make_quarter_hole_mesh(n)
        errs.append(abs(_area(Mesh(v, k, warp=w), 2) - exact))
    rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(rates > 3.0), rates
    v, k, w = make_quarter_hole_mesh(4)
    m = Mesh(v, k, warp=w)
    assert abs(_area(m, 4) - exact) < 1e-10
    p = 4
    N = cg.node_shape(m.n, p)
    X = cg.node_coordinates(m, p).reshape(N[1], N[0], 2)
    np.testing.assert_allclose(np.hypot(X[0, :, 0], X[0, :, 1]), R, atol=1e-14)      # t = 0: the arc
    np.testing.assert_allclose(np.max(X[-1], axis=1), 1.0, atol=1e-14)              # t = 1: x = 1 or y = 1
    np.testing.assert_allclose(X[:, 0, 0], 0.0, atol=1e-14)                         # s = 0: x = 0
    np.testing.assert_allclose(X[:, -1, 1], 0.0, atol=1e-14)                        # s = 1: y = 0


def test_quarter_hole_map_keeps_orientation_and_inverted_maps_are_refused():
    """Section 2: every element is the image of the unit square under an orientation-
    keeping map.  The quarter-hole stand-in has det J > 0 at every quadrature point;
    its mirror image (angle increasing with s, a clockwise parametrisation) has det J < 0
    everywhere, and the oracle refuses it instead of integrating |det J|."""
    v, k, w = make_quarter_hole_mesh(4)
    m = Mesh(v, k, warp=w)
    x1, w1 = gauss_legendre(5)
    pts, _ = cg.tensor_points(2, x1, w1)
    for e in m.elements():
        assert np.all(np.linalg.det(m.element_map(e, pts, 4)[1]) > 0)
    mirrored = Mesh(v, k, warp=lambda X: w(X)[:, ::-1])
    for e in mirrored.elements():
        assert np.all(np.linalg.det(mirrored.element_map(e, pts, 4)[1]) < 0)
    with pytest.raises(ValueError, match="inverted"):
        cg.assemble_stiffness(mirrored, 2)
    with pytest.raises(ValueError, match="inverted"):
        lor.assemble_lor(mirrored, 2)
    with pytest.raises(ValueError, match="inverted"):
        cg.load_vector(mirrored, 2, lambda X: np.ones(len(X)))
    # a multilinear element turned inside out by one swapped vertex pair is refused too
    v2, k2 = make_mesh(2, 2, perturb=0.0)
    v2 = v2.copy()
    v2[0, :, [0, 1]] = v2[0, :, [1, 0]]
    with pytest.raises(ValueError, match="inverted"):
        cg.assemble_stiffness(Mesh(v2, k2), 2)
    with pytest.raises(ValueError, match="inverted"):
        dg.assemble_dg(Mesh(v2, k2), 2, 10.0, "ip")


def test_linear_patch_test_on_curved_elements():
    v, k, w = make_quarter_hole_mesh(4)
    m = Mesh(v, k, warp=w)
    for p in (2, 5):
        N = cg.node_shape(m.n, p)
        inner = ~cg.boundary_mask(N)
        X = cg.node_coordinates(m, p)
        u = X @ np.array([0.3, -1.1]) + 0.25
        for K in (cg.assemble_stiffness(m, p), lor.assemble_lor(m, p)):
            scale = np.abs(K.diagonal()).max()
            assert np.abs((K @ u)[inner]).max() <= 1e-13 * scale
            assert np.abs(K @ np.ones(K.shape[0])).max() <= 1e-12 * scale


def _u(X):
    x, y = X[:, 0], X[:, 1]
    return (x * x + y * y - R * R) * x * y * (1 - x) * (1 - y)


def _minus_laplacian_u(X):
    """-Laplace(u) for u = g h, g = x^2 + y^2 - R^2, h = x y (1-x)(1-y), written out."""
    x, y = X[:, 0], X[:, 1]
    g = x * x + y * y - R * R
    h = x * y * (1 - x) * (1 - y)
    hx, hy = y * (1 - y) * (1 - 2 * x), x * (1 - x) * (1 - 2 * y)
    return -(4 * h + 2 * (2 * x * hx + 2 * y * hy) + g * (-2 * y * (1 - y) - 2 * x * (1 - x)))


@pytest.mark.parametrize("p", [2, 3])
def test_manufactured_order_on_the_curved_domain(p):
    errs = []
    for n in (4, 8, 16):
        v, k, w = make_quarter_hole_mesh(n)
        m = Mesh(v, k, warp=w)
        K = cg.assemble_stiffness(m, p)
        inner = ~cg.boundary_mask(cg.node_shape(m.n, p))
        b = cg.load_vector(m, p, _minus_laplacian_u)
        uh = np.zeros(len(b))
        uh[inner] = spla.spsolve(K[inner][:, inner].tocsc(), b[inner])
        errs.append(cg.l2_error(m, p, uh, _u))
    rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert rates[-1] > p + 0.5 and rates[-1] > rates[0], rates


def test_dg_oracle_refuses_curved_elements():
    v, k, w = make_quarter_hole_mesh(2)
    with pytest.raises(NotImplementedError):
        dg.assemble_dg(Mesh(v, k, warp=w), 2, 10.0)


COEF = {
    "b1": lambda X: 1e4 * (1 - X[:, 0] ** 2) * (1 - X[:, 1] ** 2),
    "b2": lambda X: 100 * X[:, 0] ** 2 + X[:, 1] ** 2 + 1,
    "b3": lambda X: (1 + X[:, 0] ** 2 + X[:, 1] ** 2) ** 4,
}


def _paper_table5():
    out = {}
    for line in open(os.path.join(GOLDEN, "table5_curved_mesh.txt")):
        if line.startswith("#") or not line.strip():
            continue
        v = [int(x) for x in line.split()]
        for c, name in enumerate(["b1", "b2", "b3", "b4"]):
            out[(v[0], name)] = (v[1 + c], v[5 + c])
    return out


@pytest.mark.parametrize("p", [2, 4])
def test_iteration_counts_vs_table5(p):
    n = 8
    paper = _paper_table5()
    for name in ("b1", "b2", "b3", "b4"):
        v, k, w = make_quarter_hole_mesh(n)
        m = Mesh(v, two_valued_kappa((n, n), seed=0) if name == "b4" else k, warp=w)
        coef = COEF.get(name)
        K = cg.assemble_stiffness(m, p, coef=coef)
        Kh = lor.assemble_lor(m, p, coef=coef)
        N = cg.node_shape(m.n, p)
        b = cg.load_vector(m, p, lambda X: np.ones(len(X)))
        A = lambda z: cg.apply_A(K, N, z)  # noqa: E731
        single = krylov.pcg(A, SinglePatchPreconditioner(m, p, K_h=Kh).apply, b, rtol=1e-8)[1]
        vertex = krylov.pcg(A, lor.LORPreconditioner(m, p, K_h=Kh).apply, b, rtol=1e-8)[1]
        ps, pv = paper[(p, name)]
        assert abs(single - ps) <= max(2, 0.15 * ps), (name, single, ps)
        assert 0.8 * pv <= vertex <= 1.3 * pv, (name, vertex, pv)
