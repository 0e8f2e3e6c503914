"""Pins of the oracle's ILU(0) orderings (Section 3.4): MDF and RCM.

MDF is checked against a separate vectorized elimination that recomputes every
candidate's discarded fill from the dense rank-1 update at each step, and against
the case where the answer is known in closed form (a chain: no fill in natural
order, so MDF must return the natural order and ILU(0) must be the exact LU).
"""
import numpy as np
import pytest

from oracle import cg, krylov, lor as olor
from oracle.mesh import Mesh
from oracle.ordering import bandwidth, discarded_fill, mdf_order, order_for, rcm_order
from paper_1908_07071_gb300.synthetic import make_mesh


def _box_matrix(dims, seed):
    """SPD matrix on the 3^d-point pattern of a box: a K_h patch block of a real mesh."""
    dim = len(dims)
    v, k = make_mesh(dim, 2, seed=seed, perturb=0.15)
    m = Mesh(v, k)
    p = (dims[0] + 1) // 2
    B = olor.LORPreconditioner(m, p, coarse=False, patch_subset=[tuple([1] * dim)])
    lev = B.patches[0]["levels"][0]
    return lev["A"], olor.box_pattern(lev["ranges"])


def _mdf_reference(A, pattern):
    """Independent MDF: dense rank-1 updates; discarded fill of every remaining
    candidate from the masked outer product at every step."""
    a = np.array(A, dtype=np.float64)
    m = a.shape[0]
    alive = np.ones(m, dtype=bool)
    off = ~np.asarray(pattern, dtype=bool)
    order = []
    for _ in range(m):
        best, bi = None, None
        for i in np.nonzero(alive)[0]:
            rest = alive.copy()
            rest[i] = False
            nb = rest & np.asarray(pattern[i], dtype=bool)
            upd = np.outer(a[nb, i], a[i, nb]) / a[i, i]
            val = np.sqrt(np.sum((upd * off[np.ix_(nb, nb)]) ** 2))
            if best is None or val < best - 1e-14 * max(best, 1.0):
                best, bi = val, i
        order.append(bi)
        alive[bi] = False
        nb = alive & np.asarray(pattern[bi], dtype=bool)
        upd = np.outer(a[nb, bi], a[bi, nb]) / a[bi, bi]
        blk = np.ix_(nb, nb)
        a[blk] -= upd * (~off[blk])
    return np.array(order)


def test_mdf_of_a_chain_is_the_natural_order_and_ilu_is_exact():
    n = 12
    rng = np.random.default_rng(0)
    A = np.diag(2.0 + rng.random(n)) - np.diag(np.ones(n - 1), 1) - np.diag(np.ones(n - 1), -1)
    pat = np.abs(np.subtract.outer(np.arange(n), np.arange(n))) <= 1
    order = mdf_order(A, pat)
    assert order.tolist() == list(range(n))
    L, U = olor.ilu0(A, pat)
    assert np.allclose(L @ U, A, atol=1e-14)


@pytest.mark.parametrize("dims", [(5, 5), (3, 3, 3)])
def test_mdf_matches_an_independent_greedy_elimination(dims):
    A, pat = _box_matrix(dims, seed=2)
    assert mdf_order(A, pat).tolist() == _mdf_reference(A, pat).tolist()


def test_mdf_first_choice_minimises_discarded_fill():
    A, pat = _box_matrix((5, 5, 5), seed=3)
    m = A.shape[0]
    nbrs = [np.array([j for j in np.nonzero(pat[i])[0] if j != i]) for i in range(m)]
    alive = np.ones(m, dtype=bool)
    fills = np.array([discarded_fill(A, pat, alive, nbrs, i) for i in range(m)])
    first = mdf_order(A, pat)[0]
    assert fills[first] == fills.min()
    # a box corner has the fewest neighbours; the choice is one of the corners
    corners = {0, 4, 20, 24, 100, 104, 120, 124}
    assert first in corners


@pytest.mark.parametrize("kind", ["lex", "rcm", "mdf"])
def test_ordered_ilu_reproduces_A_on_the_pattern(kind):
    A, pat = _box_matrix((5, 5, 5), seed=4)
    perm = order_for(kind, A, pat)
    assert sorted(perm.tolist()) == list(range(A.shape[0]))
    Ap, Pp = A[np.ix_(perm, perm)], pat[np.ix_(perm, perm)]
    L, U = olor.ilu0(Ap, Pp)
    assert np.abs((L @ U - Ap)[Pp]).max() <= 1e-13 * np.abs(A).max()
    D = np.diag(np.diag(U))
    assert np.allclose(U, D @ L.T, atol=1e-13 * np.abs(A).max())   # symmetric A: U = D L^T


def test_rcm_is_a_breadth_first_order_from_a_peripheral_node():
    """Reversed, RCM is Cuthill-McKee: breadth-first from a pseudo-peripheral node,
    so graph distances from its first node never decrease along the order (checked
    with separately computed shortest paths); on a box that node is a corner whose
    eccentricity is the graph diameter."""
    import scipy.sparse as sp
    from scipy.sparse.csgraph import shortest_path
    _, pat = _box_matrix((7, 7, 7), seed=5)
    cm = rcm_order(pat)[::-1]
    dist = shortest_path(sp.csr_matrix(pat.astype(np.int8)), unweighted=True)
    d = dist[cm[0], cm]
    assert np.all(np.diff(d) >= 0)
    assert dist[cm[0]].max() == dist.max()
    assert bandwidth(pat, cm) == bandwidth(pat, rcm_order(pat))


def test_orderings_give_symmetric_preconditioners_and_comparable_iterations():
    """Section 3.4: MDF- and RCM-ordered ILU give comparable iteration counts."""
    v, k = make_mesh(2, 6, seed=0, perturb=0.15)
    m = Mesh(v, k)
    p = 4
    K = cg.assemble_stiffness(m, p)
    N = cg.node_shape(m.n, p)
    mask = cg.boundary_mask(N).ravel()
    b = cg.load_vector(m, p, lambda X: np.ones(len(X)))
    its = {}
    rng = np.random.default_rng(0)
    u, w = rng.standard_normal(len(b)), rng.standard_normal(len(b))
    u[mask], w[mask] = 0.0, 0.0
    for kind in ("lex", "rcm", "mdf"):
        B = olor.LORPreconditioner(m, p, ordering=kind)
        assert abs(u @ B.apply(w) - w @ B.apply(u)) <= 1e-12 * abs(u @ B.apply(w))
        its[kind] = krylov.pcg(lambda z: cg.apply_A(K, N, z), B.apply, b, rtol=1e-8)[1]
    assert abs(its["mdf"] - its["lex"]) <= 2 and abs(its["rcm"] - its["lex"]) <= 2, its
