"""Anisotropic strip meshes and vertex patches enlarged for isotropic overlap (Section 4.5).

Pins: the strip mesh has the stated element sizes; the enlargement rule is the
vertex patch itself on shape-regular meshes and covers the thin strip on strip
meshes; enlarged patches keep the hierarchy Galerkin and the V(1,1) error
propagation textbook; with exact local and coarse solves the patch sum obeys the
colouring bound of additive Schwarz (patches of one colour share no coupling, so
their corrections are A-orthogonal projections); and the iteration counts behave as
Section 4.5 reports: flat in the aspect ratio with enlarged patches, growing without.
"""
import numpy as np
import pytest

from oracle import cg, krylov, lor
from oracle.mesh import Mesh
from paper_1908_07071_gb300.synthetic import make_mesh, make_strip_mesh


def test_strip_mesh_element_sizes():
    n, ar, layers = 12, 150.0, 4
    v, k = make_strip_mesh(n, ar, layers=layers, perturb=0.1, seed=3)
    ys = v[1][:, 0]
    assert np.allclose(v[1], ys[:, None])                  # rows are straight lines y = const
    xs = v[0][0]
    assert np.allclose(v[0], xs[None, :])                  # columns are straight lines x = const
    assert xs[0] == 0.0 and xs[-1] == 1.0 and ys[0] == 0.0 and ys[-1] == 1.0
    dy = np.diff(ys)
    nb = (n - layers) // 2
    np.testing.assert_allclose(dy[nb:nb + layers], 1.0 / (n * ar), rtol=1e-12)
    assert np.all(dy[:nb] > 0.1) and np.all(dy[nb + layers:] > 0.1)
    assert np.all(np.diff(xs) > 0) and np.allclose(k, 1.0)


@pytest.mark.parametrize("dim", [2, 3])
def test_enlargement_is_the_vertex_patch_on_shape_regular_meshes(dim):
    v, k = make_mesh(dim, 4, seed=0, perturb=0.15)
    spans = lor.isotropic_overlap_spans(Mesh(v, k))
    assert all(s == [(1, 1)] * dim for s in spans.values())


def test_enlarged_patches_cover_the_strip():
    n, layers = 12, 4
    nb = (n - layers) // 2
    v, k = make_strip_mesh(n, 150.0, layers=layers, perturb=0.1)
    spans = lor.isotropic_overlap_spans(Mesh(v, k))
    for (i, j), s in spans.items():
        assert s[0] == (1, 1)                                # no enlargement along the strip
        if nb <= j <= nb + layers:
            lo, hi = s[1]
            assert j - lo <= max(nb - 1, 0) and j + hi >= min(nb + layers + 1, n)
        else:
            assert s[1] == (1, 1)


def _strip_preconditioner(n, p, ar, layers, **kw):
    v, k = make_strip_mesh(n, ar, layers=layers, perturb=0.1, seed=1)
    m = Mesh(v, k)
    return m, lor.LORPreconditioner(m, p, patch_spans=lor.isotropic_overlap_spans(m), **kw)


def test_enlarged_patch_hierarchy_and_vcycle():
    m, B = _strip_preconditioner(8, 4, 150.0, 2, coarse=False)
    centre = [pt for pt in B.patches if pt["v"] == (4, 4)][0]
    lv = centre["levels"]
    assert lv[-1]["A"].shape[0] > 1                         # several vertices on the coarsest level
    V_next = np.linalg.inv(lv[-1]["A"])
    for l in range(len(lv) - 2, -1, -1):
        A, P = lv[l]["A"], lv[l]["P"]
        np.testing.assert_allclose(P.T @ A @ P, lv[l + 1]["A"], atol=1e-12 * np.abs(A).max())
        Lf, Uf = lv[l]["LU"]
        I = np.eye(A.shape[0])
        S = I - np.linalg.solve(Lf @ Uf, A)
        V = np.column_stack([B.vcycle(lv, l, c) for c in I])
        np.testing.assert_allclose(I - V @ A, S @ (I - P @ V_next @ P.T @ A) @ S, atol=1e-9)
        V_next = V


def _colouring(B, K):
    """Greedy colouring of the patches: one colour never holds two patches whose unknowns
    share a node or a matrix coupling of K."""
    sets = [set(pt["levels"][0]["idx"].tolist()) for pt in B.patches]
    reach = [set(K[list(s)].indices.tolist()) if s else set() for s in sets]
    colour = []
    for j in range(len(sets)):
        used = {colour[i] for i in range(j) if sets[i] & reach[j]}
        c = 0
        while c in used:
            c += 1
        colour.append(c)
    return max(colour) + 1


def test_enlarged_patches_obey_the_colouring_bound():
    m, B = _strip_preconditioner(6, 2, 150.0, 2, exact_local=True, exact_coarse=True)
    mask = ~cg.boundary_mask(cg.node_shape(m.n, 2))
    idx = np.nonzero(mask)[0]
    Kh = B.K_h[mask][:, mask].toarray()
    cols = []
    e = np.zeros(len(mask))
    for i in idx:
        e[:] = 0.0
        e[i] = 1.0
        cols.append(B.apply(e, parts=("patches",))[mask])
    Bp = np.column_stack(cols)
    np.testing.assert_allclose(Bp, Bp.T, atol=1e-10 * np.abs(Bp).max())
    lam = np.linalg.eigvals(Bp @ Kh).real
    chi = _colouring(B, B.K_h.tocsr())
    assert lam.max() <= chi + 1e-8, (lam.max(), chi)
    assert lam.min() > 0


def test_iterations_flat_in_aspect_ratio_with_enlarged_patches():
    """Section 4.5: with isotropic overlap the CG counts stay constant in the aspect ratio
    of the strip; plain vertex patches degrade.  Q3 on 8 x 8 elements, a 2-layer strip."""
    p = 3
    its = {}
    for ar in (15.0, 1500.0):
        v, k = make_strip_mesh(8, ar, layers=2, perturb=0.1)
        m = Mesh(v, k)
        K = cg.assemble_stiffness(m, p)
        N = cg.node_shape(m.n, p)
        b = cg.load_vector(m, p, lambda X: np.ones(len(X)))
        spans = lor.isotropic_overlap_spans(m)
        for name, kw in (("vertex", {}), ("enlarged", {"patch_spans": spans}),
                         ("enlarged+count", {"patch_spans": spans, "weighting": "count"})):
            B = lor.LORPreconditioner(m, p, **kw)
            its[name, ar] = krylov.pcg(lambda z: cg.apply_A(K, N, z), B.apply, b, rtol=1e-8)[1]
    assert its["enlarged", 1500.0] <= 1.1 * its["enlarged", 15.0], its
    assert abs(its["enlarged+count", 1500.0] - its["enlarged+count", 15.0]) <= 2, its
    assert its["vertex", 1500.0] >= 3 * its["enlarged", 1500.0], its
    assert its["vertex", 1500.0] >= 2 * its["vertex", 15.0], its


def test_pou_weights_on_enlarged_patches():
    """weighting="pou" with enlarged patches: normalised tents in physical coordinates,
    sum_j W_j^2 = 1 at every interior node, and counts flat in the aspect ratio (measured on
    8 x 8, 2-layer strip, Q3: 16 / 16 at aspect 15 / 1500; vertex patches 51 / 172)."""
    p = 3
    its = {}
    for ar in (15.0, 1500.0):
        v, k = make_strip_mesh(8, ar, layers=2, perturb=0.1)
        m = Mesh(v, k)
        B = lor.LORPreconditioner(m, p, patch_spans=lor.isotropic_overlap_spans(m), weighting="pou")
        s = np.zeros(int(np.prod(B.Ns[0])))
        for j, pt in enumerate(B.patches):
            idx = pt["levels"][0]["idx"]
            if len(idx):
                w = B.pou_weights(j)
                assert np.all(w > 0)
                s[idx] += w ** 2
        inner = ~cg.boundary_mask(B.Ns[0])
        np.testing.assert_allclose(s[inner], 1.0, atol=1e-14)
        K = cg.assemble_stiffness(m, p)
        N = cg.node_shape(m.n, p)
        b = cg.load_vector(m, p, lambda X: np.ones(len(X)))
        its[ar] = krylov.pcg(lambda z: cg.apply_A(K, N, z), B.apply, b, rtol=1e-8)[1]
    assert abs(its[1500.0] - its[15.0]) <= 2 and its[1500.0] <= 25, its
