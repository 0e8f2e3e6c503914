"""Pins of the unstructured-mesh oracle (`oracle.unstructured`, Section 4.2 meshes).

* A structured grid given as an unstructured mesh reproduces the structured oracle's
  K_p, K_h, P_0 and (with exact patch and coarse solves) B exactly, after matching
  nodes by their coordinates: the general numbering and patch extraction are checked
  against independent code.
* On the split-triangle mesh (interior vertices with 3, 4 or 8 elements, edges run in
  opposite directions by their two elements) the numbering is conforming, linear
  functions pass the patch test, the patch hierarchy is Galerkin and the V(1,1) cycle
  has the textbook error propagation, the additive Schwarz sum with exact solves obeys
  the colouring bound, and the CG counts stay bounded in h (Section 4.2: iteration
  counts remain bounded on unstructured meshes).
"""
import numpy as np
import pytest

from oracle import cg, krylov, lor, unstructured as un
from oracle.mesh import Mesh
from paper_1908_07071_gb300.synthetic import make_mesh, make_split_triangle_mesh


def _grid_as_quads(n, seed):
    v, k = make_mesh(2, n, seed=seed, perturb=0.15)
    verts = np.stack([v[0].ravel(), v[1].ravel()], axis=1)
    vid = lambda i, j: j * (n + 1) + i  # noqa: E731
    quads = [(vid(i, j), vid(i + 1, j), vid(i, j + 1), vid(i + 1, j + 1)) for j in range(n) for i in range(n)]
    return Mesh(v, k), un.QuadMesh(verts, quads, k.ravel())


def _match(Xa, Xb):
    """perm with Xb[perm[i]] == Xa[i]."""
    d = np.linalg.norm(Xa[:, None, :] - Xb[None, :, :], axis=2)
    perm = d.argmin(axis=1)
    assert np.all(d[np.arange(len(Xa)), perm] < 1e-12) and len(set(perm.tolist())) == len(Xa)
    return perm


@pytest.mark.parametrize("p", [2, 3])
def test_structured_grid_reproduces_the_structured_oracle(p):
    n = 3
    sm, um = _grid_as_quads(n, seed=4)
    L0 = un.Level(um, p, list(range(p + 1)))
    perm = _match(L0.X, cg.node_coordinates(sm, p))
    Ks = cg.assemble_stiffness(sm, p).toarray()
    np.testing.assert_allclose(un.assemble_stiffness(um, p, L0).toarray(), Ks[np.ix_(perm, perm)],
                               atol=1e-12 * np.abs(Ks).max())
    Khs = lor.assemble_lor(sm, p).toarray()
    np.testing.assert_allclose(un.assemble_lor(um, L0).toarray(), Khs[np.ix_(perm, perm)],
                               atol=1e-12 * np.abs(Khs).max())
    Bs = lor.LORPreconditioner(sm, p, exact_local=True, exact_coarse=True)
    Bu = un.UnstructuredLOR(um, p, local="exact")
    np.testing.assert_allclose(Bu.P0.toarray(), Bs.P0.toarray()[perm], atol=1e-14)
    assert np.array_equal(L0.boundary, cg.boundary_mask(cg.node_shape(sm.n, p))[perm])
    rng = np.random.default_rng(1)
    for _ in range(3):
        r = rng.standard_normal(L0.ntot)
        rs = np.empty_like(r)
        rs[perm] = r
        np.testing.assert_allclose(Bu.apply(r), Bs.apply(rs)[perm], atol=1e-12 * np.abs(Bs.apply(rs)).max())


def _unstructured(n=2, seed=0):
    v, q, k = make_split_triangle_mesh(n, seed=seed)
    return un.QuadMesh(v, q, k)


def test_split_triangle_mesh_is_unstructured_and_numbering_conforming():
    m = _unstructured(3)
    valence = np.bincount(m.quads.ravel(), minlength=m.nv)
    inner = [v for v in range(m.nv) if v not in m.boundary_vertices]
    assert {3, 4, 8} <= set(valence[inner].tolist())
    # some shared edge is run in opposite directions by its two elements
    runs = {}
    for q in m.quads:
        for a, b in m.local_edges:
            runs.setdefault((min(q[a], q[b]), max(q[a], q[b])), set()).add(q[a] < q[b])
    assert any(len(s) == 2 for s in runs.values())
    p = 4
    for sel in lor.level_selections(p):
        lev = un.Level(m, p, sel)
        # every global node gets the same position from each element that holds it
        from oracle.basis import gll
        from oracle.mesh import multilinear
        xg = gll(p)[0][sel]
        pts, _ = cg.tensor_points(2, xg, np.ones(len(sel)))
        for e, q in enumerate(m.quads):
            np.testing.assert_allclose(multilinear(m.vertices[q], pts)[0], lev.X[lev.local[e]], atol=1e-14)
        assert len(np.unique(lev.local)) == lev.ntot


@pytest.mark.parametrize("p", [2, 5])
def test_linear_patch_test_on_the_unstructured_mesh(p):
    m = _unstructured(2, seed=3)
    L0 = un.Level(m, p, list(range(p + 1)))
    u = L0.X @ np.array([0.3, -1.1]) + 0.25
    inner = ~L0.boundary
    for K in (un.assemble_stiffness(m, p, L0), un.assemble_lor(m, L0)):
        scale = np.abs(K.diagonal()).max()
        assert np.abs((K @ u)[inner]).max() <= 1e-12 * scale
        assert np.abs(K @ np.ones(K.shape[0])).max() <= 1e-12 * scale
        assert abs(K - K.T).max() <= 1e-13 * scale


def test_odd_degrees_refuse_the_hierarchy():
    with pytest.raises(NotImplementedError):
        un.UnstructuredLOR(_unstructured(2), 3)


def test_patch_hierarchy_and_vcycle_on_unstructured_patches():
    m = _unstructured(2, seed=1)
    B = un.UnstructuredLOR(m, 4)
    valence = np.bincount(m.quads.ravel(), minlength=m.nv)
    picked = [pt for pt in B.patches if pt["v"] not in m.boundary_vertices and valence[pt["v"]] in (3, 8)]
    assert {valence[pt["v"]] for pt in picked} == {3, 8}
    for pt in picked:
        lv = pt["levels"]
        V_next = np.linalg.inv(lv[-1]["A"])
        for l in range(len(lv) - 2, -1, -1):
            A, P = lv[l]["A"], lv[l]["P"]
            np.testing.assert_allclose(P.T @ A @ P, lv[l + 1]["A"], atol=1e-12 * np.abs(A).max())
            I = np.eye(A.shape[0])
            S = I - B.smooth(lv[l], A)
            V = np.column_stack([B.vcycle(lv, l, c) for c in I])
            np.testing.assert_allclose(I - V @ A, S @ (I - P @ V_next @ P.T @ A) @ S, atol=1e-9)
            V_next = V


def test_exact_solves_obey_the_colouring_bound():
    m = _unstructured(2, seed=2)
    p = 2
    B = un.UnstructuredLOR(m, p, local="exact")
    inner = np.nonzero(~B.levels[0].boundary)[0]
    Kh = B.K_h.toarray()[np.ix_(inner, inner)]
    cols = []
    for i in inner:
        e = np.zeros(B.levels[0].ntot)
        e[i] = 1.0
        cols.append(B.apply(e, parts=("patches",))[inner])
    Bp = np.column_stack(cols)
    np.testing.assert_allclose(Bp, Bp.T, atol=1e-10 * np.abs(Bp).max())
    lam = np.linalg.eigvals(Bp @ Kh).real
    # greedy colouring: one colour never holds two patches that share a node or a K_h coupling
    sets = [set(pt["levels"][0]["idx"].tolist()) for pt in B.patches]
    K = B.K_h.tocsr()
    reach = [set(K[list(s)].indices.tolist()) if s else set() for s in sets]
    colour = []
    for j in range(len(sets)):
        used = {colour[i] for i in range(j) if sets[i] & reach[j]}
        c = 0
        while c in used:
            c += 1
        colour.append(c)
    assert 0 < lam.min() and lam.max() <= max(colour) + 1 + 1e-8, (lam.max(), max(colour) + 1)


def test_iterations_bounded_in_h_on_unstructured_meshes():
    its = {}
    for p in (2, 4):
        for n in (2, 4):
            m = _unstructured(n, seed=0)
            L0 = un.Level(m, p, list(range(p + 1)))
            K = un.assemble_stiffness(m, p, L0)
            inner = ~L0.boundary
            b = np.where(inner, 1.0, 0.0)
            A = lambda z: np.where(inner, K @ np.where(inner, z, 0.0), 0.0)  # noqa: E731
            its[p, n] = krylov.pcg(A, un.UnstructuredLOR(m, p).apply, b, rtol=1e-8)[1]
    for p in (2, 4):
        assert its[p, 4] <= 1.25 * its[p, 2] + 2, its
    assert its[4, 4] <= 45, its


def test_pou_weights_on_unstructured_patches():
    """weighting="pou": W_j = sqrt(P_0[:, j]) on the patch; sum_j W_j^2 = 1 at every interior
    node, and fewer PCG iterations than unit weights (measured: p = 4, n = 2: 34 -> 21)."""
    m = _unstructured(2, seed=0)
    p = 4
    Bw = un.UnstructuredLOR(m, p, weighting="pou")
    s = np.zeros(Bw.levels[0].ntot)
    for pt in Bw.patches:
        idx = pt["levels"][0]["idx"]
        s[idx] += Bw.P0[idx, pt["v"]].toarray().ravel()
    inner = ~Bw.levels[0].boundary
    np.testing.assert_allclose(s[inner], 1.0, atol=1e-14)
    L0 = Bw.levels[0]
    K = un.assemble_stiffness(m, p, L0)
    b = np.where(inner, 1.0, 0.0)
    A = lambda z: np.where(inner, K @ np.where(inner, z, 0.0), 0.0)  # noqa: E731
    it_unit = krylov.pcg(A, un.UnstructuredLOR(m, p).apply, b, rtol=1e-8)[1]
    it_pou = krylov.pcg(A, Bw.apply, b, rtol=1e-8)[1]
    assert it_pou <= 0.75 * it_unit, (it_unit, it_pou)
