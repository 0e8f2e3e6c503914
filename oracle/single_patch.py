"""B(1): the whole domain as one additive-Schwarz patch.  TEST INFRASTRUCTURE ONLY.

Section 4.1 first studies the local multigrid solver with a single patch for the
entire domain: the high-order system is preconditioned by one element-structured
V-cycle (Section 3.3) on the low-order refined system K_h, with one ordered ILU(0)
sweep (forward and backward) as pre- and post-smoother at every level, coarsening
each element until its interior Gauss-Lobatto points are gone; the p=1 problem on the
coarse mesh that remains is solved by the coarse solver R_0.  Here the levels are the
Galerkin operators of `oracle.lor` restricted to interior (non-Dirichlet) nodes, the
ILU(0) is lexicographic on the structural 3^d-point pattern of each level grid, and
R_0 is the same vertex-grid V-cycle the vertex-patch preconditioner uses.  Because
each coarsening step interpolates linearly in the element reference coordinate, the
composition of the level prolongations down to the vertex level is the vertex basis
P_0, so the vertex-level operator is the coarse operator P_0^T K_h P_0 that R_0 was
built for.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from .cg import boundary_mask
from .lor import LORPreconditioner, kron_nd
from .mesh import Mesh


def grid_pattern(N):
    """Structural 3^d-point pattern (|di|, |dj|, |dk| <= 1) of a full grid N (x first), CSR."""
    tri = [sp.diags([1, 1, 1], [-1, 0, 1], shape=(n, n), dtype=np.int8, format="csr") for n in N]
    return kron_nd(tri).astype(bool).tocsr()


def ilu0_csr(A, pattern):
    """IKJ ILU(0) of sparse A on `pattern` (CSR, same shape); unit-lower L and upper U.

    A non-positive pivot is a breakdown (raises FloatingPointError)."""
    A = sp.csr_matrix(A)
    pattern = sp.csr_matrix(pattern)
    m = A.shape[0]
    rows = []
    for i in range(m):
        cols = pattern.indices[pattern.indptr[i]:pattern.indptr[i + 1]]
        vals = dict.fromkeys(cols.tolist(), 0.0)
        for c, v in zip(A.indices[A.indptr[i]:A.indptr[i + 1]], A.data[A.indptr[i]:A.indptr[i + 1]]):
            if c in vals:
                vals[int(c)] = float(v)
        rows.append(vals)
    diag = np.zeros(m)
    for i in range(m):
        ri = rows[i]
        for k in sorted(c for c in ri if c < i):
            ri[k] /= diag[k]
            lik = ri[k]
            for j, ukj in rows[k].items():
                if j > k and j in ri:
                    ri[j] -= lik * ukj
        if not ri.get(i, 0.0) > 0.0:
            raise FloatingPointError(f"ILU(0) breakdown: non-positive pivot at row {i}")
        diag[i] = ri[i]
    Li, Lj, Lv, Ui, Uj, Uv = [], [], [], [], [], []
    for i, ri in enumerate(rows):
        for j, v in ri.items():
            if j < i:
                Li.append(i); Lj.append(j); Lv.append(v)
            else:
                Ui.append(i); Uj.append(j); Uv.append(v)
    L = sp.csr_matrix((Lv, (Li, Lj)), shape=(m, m)) + sp.identity(m, format="csr")
    U = sp.csr_matrix((Uv, (Ui, Uj)), shape=(m, m))
    return L.tocsr(), U.tocsr()


def ilu_apply(L, U, r):
    """(L U)^{-1} r with the sparse factors (one ILU(0) smoothing, Section 3.4)."""
    w = spla.spsolve_triangular(L, r, lower=True, unit_diagonal=True)
    return spla.spsolve_triangular(U, w, lower=False)


SMOOTHERS = ("ilu", "jacobi", "gs", "line-jacobi", "line-gs")


def line_blocks(N, mask):
    """Interior unknowns grouped by x-line (fixed y[, z]), in the order of the masked grid."""
    ids = np.nonzero(mask)[0]
    pos = np.empty(len(mask), dtype=np.int64)
    pos[ids] = np.arange(len(ids))
    key = ids // N[0]
    return [pos[ids[key == k]] for k in np.unique(key)]


class SinglePatchPreconditioner:
    """B(1) r = one V(1,1) cycle of the element-structured hierarchy on the whole domain.

    smoother (Section 3.4 compares smoothers on the GLL-refined mesh): "ilu" (ordered
    ILU(0), the method), "jacobi" (damped point Jacobi, weight 2/3), "gs" (point
    Gauss-Seidel: forward sweep before, backward sweep after the coarse correction, so
    the cycle stays symmetric), "line-jacobi" (damped block Jacobi on x-lines, weight
    2/3) and "line-gs" (block Gauss-Seidel on x-lines, forward then backward)."""

    def __init__(self, mesh: Mesh, p: int, mg_levels: int = 0, K_h=None, smoother: str = "ilu"):
        if smoother not in SMOOTHERS:
            raise ValueError(smoother)
        self.smoother = smoother
        self.base = LORPreconditioner(mesh, p, mg_levels=mg_levels, patch_subset=[], K_h=K_h)
        b = self.base
        self.L = len(b.A)
        self.mask = [~boundary_mask(N).ravel() for N in b.Ns]
        self.A = [b.A[l][self.mask[l]][:, self.mask[l]].tocsr() for l in range(self.L)]
        self.P = []
        for l in range(self.L - 1):
            P = kron_nd(b.P1[l]).tocsr()
            self.P.append(P[self.mask[l]][:, self.mask[l + 1]].tocsr())
        self.LU = []
        self.lines = []
        for l in range(self.L - 1):
            if smoother == "ilu":
                pat = grid_pattern(b.Ns[l])[self.mask[l]][:, self.mask[l]]
                self.LU.append(ilu0_csr(self.A[l], pat))
            self.lines.append(line_blocks(b.Ns[l], self.mask[l]) if smoother.startswith("line") else None)

    def smooth(self, l, r, x, forward=True):
        """One smoothing step x <- x + M^{-1} (r - A x) on level l (pre: forward, post: backward)."""
        A = self.A[l]
        if self.smoother == "ilu":
            return x + ilu_apply(*self.LU[l], r - A @ x)
        if self.smoother == "jacobi":
            return x + (2.0 / 3.0) * (r - A @ x) / A.diagonal()
        if self.smoother == "gs":
            Ad = A.toarray()
            T = np.tril(Ad) if forward else np.triu(Ad)
            return x + spla.spsolve_triangular(sp.csr_matrix(T), r - A @ x, lower=forward)
        blocks = self.lines[l] if forward else self.lines[l][::-1]
        if self.smoother == "line-jacobi":
            res = r - A @ x
            y = x.copy()
            for blk in blocks:
                y[blk] += (2.0 / 3.0) * np.linalg.solve(A[blk][:, blk].toarray(), res[blk])
            return y
        y = x.copy()                                      # line Gauss-Seidel
        for blk in blocks:
            y[blk] += np.linalg.solve(A[blk][:, blk].toarray(), (r - A @ y)[blk])
        return y

    def vcycle(self, l, r):
        """V(1,1) on global level l (Section 3.3); R_0 on the vertex level."""
        if len(r) == 0:
            return r
        if l == self.L - 1:
            return self.base.coarse_solve(r)
        A = self.A[l]
        x = self.smooth(l, r, np.zeros_like(r), forward=True)
        P = self.P[l]
        if P.shape[1] > 0:
            x = x + P @ self.vcycle(l + 1, P.T @ (r - A @ x))
        return self.smooth(l, r, x, forward=False)

    def apply(self, r):
        """B(1) r on the full node grid; Dirichlet entries are ignored and returned as 0."""
        r = np.asarray(r, dtype=np.float64)
        z = np.zeros_like(r)
        z[self.mask[0]] = self.vcycle(0, r[self.mask[0]])
        return z
