"""The ILU(0) orderings of the library's host code (lor_box_ordering: reverse
Cuthill-McKee and minimum discarded fill, Section 3.4) against the oracle's, node for
node, on the patch matrices of small meshes (no GPU: host code of the C ABI)."""
import numpy as np
import pytest

from oracle import lor as olor
from oracle import ordering as ordo
from oracle.mesh import Mesh
from paper_1908_07071_gb300.synthetic import make_mesh


@pytest.fixture(scope="module")
def lor():
    from paper_1908_07071_gb300.build import build_library
    build_library()
    from paper_1908_07071_gb300 import lor as mod
    return mod


def _a27(Aj, dims, dim):
    """Stencil layout of a box matrix: per node its 3^d values in stencil-offset order."""
    A, B = dims[0], dims[1]
    C = dims[2] if dim == 3 else 1
    n = A * B * C
    NS = 27 if dim == 3 else 9
    out = np.zeros((n, NS))
    for i in range(n):
        x, y, z = i % A, (i // A) % B, i // (A * B)
        for o in range(NS):
            dx, dy, dz = o % 3 - 1, (o // 3) % 3 - 1, (o // 9 - 1 if dim == 3 else 0)
            X, Y, Z = x + dx, y + dy, z + dz
            if 0 <= X < A and 0 <= Y < B and 0 <= Z < C:
                out[i, o] = Aj[i, (Z * B + Y) * A + X]
    return out


@pytest.mark.parametrize("dim,n,p", [(2, 3, 4), (3, 2, 3), (3, 3, 2), (2, 4, 6)])
@pytest.mark.parametrize("kind,code", [("rcm", 1), ("mdf", 2)])
def test_box_orderings_equal_the_oracle(lor, dim, n, p, kind, code):
    v, k = make_mesh(dim, n, seed=1, perturb=0.15)
    B = olor.LORPreconditioner(Mesh(v, k), p, ordering=kind, coarse=False)
    checked = 0
    for P in B.patches:
        for lev in P["levels"][:-1]:
            if "perm" not in lev:
                continue
            dims = [len(r) for r in lev["ranges"]]
            a27 = _a27(lev["A"], dims, dim) if code == 2 else None
            perm = lor.box_ordering(dims, code, a27)
            np.testing.assert_array_equal(perm, lev["perm"])
            checked += 1
    assert checked > 0


def _box_matrix(dims, dim, kind, seed):
    """Dense symmetric matrix on the 3^d-point pattern of a box: equal couplings (every
    MDF step is decided by exact ties, broken by the smallest index) or random ones."""
    pat = olor.box_pattern([np.arange(d) for d in dims])
    m = pat.shape[0]
    rng = np.random.default_rng(seed)
    A = np.zeros((m, m))
    for r in range(m):
        for c in range(r + 1, m):
            if pat[r, c]:
                A[r, c] = A[c, r] = -1.0 if kind == "ties" else -rng.uniform(0.2, 1.0)
    A[np.arange(m), np.arange(m)] = np.abs(A).sum(axis=1) + 0.5
    return A, pat


@pytest.mark.parametrize("dims", [(3, 3, 3), (4, 3, 2), (2, 2, 2), (1, 4, 3), (6, 5), (7, 1), (4, 4, 4)])
@pytest.mark.parametrize("kind", ["ties", "random"])
def test_mdf_of_box_matrices_equals_the_oracle(lor, dims, kind):
    """MDF through lor_box_ordering against the oracle's greedy elimination on whole
    box matrices, node for node, including matrices whose every step is a tie."""
    dim = len(dims)
    A, pat = _box_matrix(dims, dim, kind, seed=len(dims) * 100 + dims[0])
    perm = lor.box_ordering(dims, 2, _a27(A, dims, dim))
    np.testing.assert_array_equal(perm, ordo.mdf_order(A, pat))


def _stencil_dense(lu, dims, dim, perm):
    """Dense factors, in elimination order, from the stencil layout of lor_box_ilu0."""
    A, B = dims[0], dims[1]
    C = dims[2] if dim == 3 else 1
    n = A * B * C
    NS = 27 if dim == 3 else 9
    pos = np.empty(n, dtype=np.int64)
    pos[perm] = np.arange(n)
    L, U = np.eye(n), np.zeros((n, n))
    for i in range(n):
        x, y, z = i % A, (i // A) % B, i // (A * B)
        for o in range(NS):
            dx, dy, dz = o % 3 - 1, (o // 3) % 3 - 1, (o // 9 - 1 if dim == 3 else 0)
            X, Y, Z = x + dx, y + dy, z + dz
            if not (0 <= X < A and 0 <= Y < B and 0 <= Z < C):
                assert lu[i, o] == 0.0
                continue
            k = (Z * B + Y) * A + X
            if pos[k] < pos[i]:
                L[pos[i], pos[k]] = lu[i, o]
            else:
                U[pos[i], pos[k]] = lu[i, o]
    return L, U, pos


@pytest.mark.parametrize("dims", [(3, 3, 3), (4, 3, 2), (1, 4, 3), (6, 5), (2, 7)])
@pytest.mark.parametrize("order", ["lex", "rcm", "mdf", "random"])
def test_ordered_ilu0_of_box_matrices_equals_the_oracle(lor, dims, order):
    """lor_box_ilu0 (the factorization lor_setup runs for RCM/MDF-ordered patches)
    against the oracle's IKJ ILU(0) of the permuted matrix: factors bit for bit (both
    sides round every product and difference alone, in the same order), and dependency
    levels equal to their definition (0 without earlier neighbours, else one more than
    the largest earlier neighbour's)."""
    dim = len(dims)
    A, pat = _box_matrix(dims, dim, "random", seed=sum(dims))
    a27 = _a27(A, dims, dim)
    n = A.shape[0]
    perm = {"lex": np.arange(n), "rcm": lor.box_ordering(dims, 1), "mdf": lor.box_ordering(dims, 2, a27),
            "random": np.random.default_rng(n).permutation(n)}[order]
    lu, level = lor.box_ilu0(dims, a27, perm)
    L, U, pos = _stencil_dense(lu, dims, dim, perm)
    Lo, Uo = olor.ilu0(A[np.ix_(perm, perm)], pat[np.ix_(perm, perm)])
    np.testing.assert_array_equal(L, Lo)
    np.testing.assert_array_equal(U, Uo)
    want = np.zeros(n, dtype=np.int64)
    for q in range(n):
        i = perm[q]
        earlier = [k for k in np.nonzero(pat[i])[0] if pos[k] < q]
        want[i] = 1 + max(want[k] for k in earlier) if earlier else 0
    np.testing.assert_array_equal(level, want)


def test_box_ilu0_rejects_bad_orders_and_reports_breakdown(lor):
    A, pat = _box_matrix((3, 2), 2, "random", seed=1)
    a27 = _a27(A, (3, 2), 2)
    with pytest.raises(lor.LorError) as err:
        lor.box_ilu0((3, 2), a27, [0, 1, 2, 3, 4, 4])      # not a permutation
    assert err.value.status == lor.LOR_EINVAL
    bad = a27.copy()
    bad[:, 4] = 0.05                                       # pivots too small: breakdown
    with pytest.raises(lor.LorError) as err:
        lor.box_ilu0((3, 2), bad, np.arange(6))
    assert err.value.status == lor.LOR_EBREAKDOWN


def test_box_ordering_rejects_bad_input_and_reports_breakdown(lor):
    with pytest.raises(lor.LorError) as err:
        lor.box_ordering((3, 3, 3), 3)
    assert err.value.status == lor.LOR_EINVAL
    with pytest.raises(lor.LorError):
        lor.box_ordering((3, 3, 3), 2)                  # MDF needs the matrix
    a27 = np.zeros((8, 9))
    a27[:, 4] = -1.0                                    # non-positive pivots
    with pytest.raises(lor.LorError) as err:
        lor.box_ordering((4, 2), 2, a27)
    assert err.value.status == lor.LOR_EBREAKDOWN
    np.testing.assert_array_equal(lor.box_ordering((4, 2), 0), np.arange(8))
    # RCM of a box is a permutation with the bandwidth scipy's routine reaches
    pat = np.ones((1, 1), dtype=bool)
    for dims in [(5, 4, 3), (6, 1, 1), (4, 4)]:
        perm = lor.box_ordering(dims, 1)
        assert sorted(perm.tolist()) == list(range(int(np.prod(dims))))
        ranges = [np.arange(d) for d in dims]
        pat = olor.box_pattern(ranges)
        assert ordo.bandwidth(pat, perm) == ordo.bandwidth(pat, ordo.rcm_order(pat))
