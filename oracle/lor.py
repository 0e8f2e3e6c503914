"""Low-order-refined additive-Schwarz preconditioner (oracle; FP64).

Follows Section 3 step by step, with dense/sparse library primitives only:

* Section 3.1: T_h subdivides every element at its GLL points; K_h is the
  assembled multilinear (p=1) stiffness on T_h.  Reading: 2-point Gauss per
  direction on each sub-element, coefficient of the parent element.
* Section 3.3: element-structured hierarchy.  Each level keeps every other
  point of the previous level's 1D subgrid (positions 0, 2, 4, ... plus the
  last endpoint) until only the element vertices remain.  Prolongation is
  1D linear interpolation in the element's reference coordinate (tensor
  product in d dimensions); coarse operators are Galerkin P^T A P (reading).
  V(1,1): one pre- and one post-smoothing per level, exact solve on the
  coarsest (vertex) level.
* Section 3.4: smoothing by ILU(0) of the patch matrix on its structural
  (3^d-point) pattern, rows in patch-lexicographic order (x fastest).
* Section 3.2, Eq. (as) and Eq. (patch): B = sum_j R_j Q_j with one patch per
  coarse vertex, Omega_j = union of the elements touching the vertex, homogeneous
  Dirichlet on its boundary, plus the coarse space V_0 = Q1 on T_p.
  Reading (R_0): the paper uses one BoomerAMG V-cycle, a third-party system;
  here R_0 is one V-cycle on the coarse vertex grid: keep-even-plus-last 2x
  coarsening, index-space linear interpolation, Galerkin operators, two sweeps of
  l1-scaled Jacobi before and after (the relaxation BoomerAMG offers, Section 4.4),
  and an exact dense solve once at most 343 unknowns remain.
"""
from __future__ import annotations

import itertools

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp

from . import ordering
from .basis import gll
from .cg import boundary_mask, node_coordinates, node_shape
from .mesh import Mesh, multilinear, oriented_det

COARSE_DIRECT_MAX = 343
COARSE_SWEEPS = 2


# --------------------------------------------------------------------------- K_h
def q1_stiffness_batch(corners, kappa):
    """Q1 element stiffness for a batch of cells: corners (C, 2^d, d) -> (C, 2^d, 2^d).

    kappa: (C,) constants per cell, or a callable b(X) of physical points (C, d)
    evaluated at each cell's Gauss points (Section 4.2 coefficients)."""
    C, nc, d = corners.shape
    g = 0.5 - 0.5 / np.sqrt(3.0)
    g1 = np.array([g, 1.0 - g])
    K = np.zeros((C, nc, nc))
    for gp in itertools.product(range(2), repeat=d):
        xi = np.array([g1[gp[a]] for a in range(d)])
        w = 0.5 ** d
        # reference gradients of the 2^d corner functions at xi
        dN = np.zeros((nc, d))
        for c in range(nc):
            bits = [(c >> a) & 1 for a in range(d)]
            for b in range(d):
                v = 1.0
                for a in range(d):
                    f = xi[a] if bits[a] else 1.0 - xi[a]
                    df = 1.0 if bits[a] else -1.0
                    v *= df if a == b else f
                dN[c, b] = v
        J = np.einsum("Cca,cb->Cab", corners, dN)          # dX_a/dxi_b
        detJ = oriented_det(J)
        Jinv = np.linalg.inv(J)
        gphys = np.einsum("Cba,cb->Cca", Jinv, dN)         # J^{-T} dN
        if callable(kappa):
            Nc = np.array([np.prod([xi[a] if (c >> a) & 1 else 1.0 - xi[a] for a in range(d)])
                           for c in range(nc)])
            kq = np.asarray(kappa(np.einsum("Cca,c->Ca", corners, Nc)), dtype=np.float64)
        else:
            kq = kappa
        K += (w * detJ * kq)[:, None, None] * np.einsum("Cia,Cja->Cij", gphys, gphys)
    return K


def assemble_lor(mesh: Mesh, p: int, coef=None):
    """K_h over all nodes of the GLL-refined grid (no Dirichlet elimination), CSR.

    coef: optional callable b(X) replacing the parent element's kappa; reading: it is
    evaluated at the 2-point Gauss points of every LOR sub-cell, like the geometry."""
    d = mesh.dim
    N = node_shape(mesh.n, p)
    X = node_coordinates(mesh, p)
    cells = np.array(list(itertools.product(*[range(v - 1) for v in reversed(N)])))
    cells = cells[:, ::-1]                          # (C, d) as (I, J, K)
    strides = np.cumprod([1] + list(N[:-1]))
    corner_ids = np.zeros((len(cells), 2 ** d), dtype=np.int64)
    for c in range(2 ** d):
        off = np.array([(c >> a) & 1 for a in range(d)])
        corner_ids[:, c] = ((cells + off) * strides).sum(axis=1)
    elem = cells // p
    kap = mesh.kappa[tuple(elem[:, a] for a in reversed(range(d)))] if coef is None else coef
    Kc = q1_stiffness_batch(X[corner_ids], kap)
    rows = np.repeat(corner_ids, 2 ** d, axis=1).ravel()
    cols = np.tile(corner_ids, (1, 2 ** d)).ravel()
    ntot = int(np.prod(N))
    K = sp.coo_matrix((Kc.ravel(), (rows, cols)), shape=(ntot, ntot)).tocsr()
    K.sum_duplicates()
    return K


# --------------------------------------------------------------- hierarchy (3.3)
def level_selections(p: int, mg_levels: int = 0):
    """GLL-index subsets per level, finest first, ending with [0, p].

    mg_levels = 0 takes the full hierarchy; mg_levels = L >= 2 keeps its first
    L-1 levels and then jumps to the vertex level.
    """
    sels = [list(range(p + 1))]
    while len(sels[-1]) > 2:
        s = sels[-1]
        t = s[0::2]
        if t[-1] != s[-1]:
            t = t + [s[-1]]
        sels.append(t)
    if mg_levels and mg_levels < len(sels):
        sels = sels[: mg_levels - 1] + [sels[-1]]
    return sels


def prolong_1d(nel: int, p: int, sel_f, sel_c):
    """Global 1D prolongation (N_f x N_c): linear interpolation in reference coordinates."""
    xg = gll(p)[0]
    mf, mc = len(sel_f) - 1, len(sel_c) - 1
    P = np.zeros((nel * mf + 1, nel * mc + 1))
    for e in range(nel):
        for t, g in enumerate(sel_f):
            a = max(i for i in range(mc + 1) if sel_c[i] <= g)
            if sel_c[a] == g:
                P[e * mf + t, e * mc + a] = 1.0
                continue
            b = a + 1
            w = (xg[g] - xg[sel_c[a]]) / (xg[sel_c[b]] - xg[sel_c[a]])
            P[e * mf + t, e * mc + a] = 1.0 - w
            P[e * mf + t, e * mc + b] = w
    return P


def kron_nd(mats_xyz):
    """kron over axes given in x, y, z order with x fastest in the result."""
    out = sp.csr_matrix(mats_xyz[-1])
    for m in reversed(mats_xyz[:-1]):
        out = sp.kron(out, sp.csr_matrix(m), format="csr")
    return out


# ----------------------------------------------------------------- ILU(0) (3.4)
def ilu0(A, pattern):
    """IKJ ILU(0) on the structural ``pattern``; returns dense unit-L and U.

    A pivot that is not positive is a breakdown (raises FloatingPointError).
    """
    a = np.array(A, dtype=np.float64, copy=True)
    m = a.shape[0]
    if m and a[0, 0] <= 0:
        raise FloatingPointError("ILU(0) breakdown: non-positive pivot at row 0")
    for i in range(1, m):
        ks = np.nonzero(pattern[i, :i])[0]
        for k in ks:
            a[i, k] /= a[k, k]
            cols = np.nonzero(pattern[i, k + 1:])[0] + k + 1
            a[i, cols] -= a[i, k] * a[k, cols]
        if a[i, i] <= 0:
            raise FloatingPointError(f"ILU(0) breakdown: non-positive pivot at row {i}")
    L = np.tril(a, -1) + np.eye(m)
    U = np.triu(a)
    return L, U


def ilu_solve(L, U, r):
    """(L U)^{-1} r: forward then backward triangular solve (one ILU(0) smoothing, Section 3.4)."""
    w = sla.solve_triangular(L, r, lower=True, unit_diagonal=True)
    return sla.solve_triangular(U, w, lower=False)


# ------------------------------------------------------------- patches (3.2)
def patch_range_1d(v: int, nel: int, m: int, lo_k: int = 1, hi_k: int = 1):
    """Global level indices of the open interior of the patch of vertex v (one axis).

    The patch covers the elements v - lo_k, ..., v + hi_k - 1 of the axis (clamped to
    the mesh); lo_k = hi_k = 1 is the vertex patch of Eq. (patch)."""
    lo = max(v - lo_k, 0) * m
    hi = min(v + hi_k, nel) * m
    return np.arange(lo + 1, hi)


def isotropic_overlap_spans(mesh: Mesh, ratio: float = 0.5):
    """Element spans of vertex patches enlarged so that their overlap stays isotropic.

    Section 4.5 extends the patches that contain high-aspect-ratio elements so that the
    overlap no longer shrinks with the aspect ratio (the partition-of-unity argument
    behind the lemma on the local decomposition in Section 3.2 needs overlap of the
    size of the elements, not of their thin side).  The paper does not state the rule;
    reading: the isotropic size of vertex v is the longest mesh edge at v, and along
    each axis and side the patch takes whole elements until the vertex it reaches lies
    at least ratio x that size from v (or the boundary is reached).  On meshes whose
    edges at a vertex differ by less than 1/ratio this is the vertex patch itself.
    Returns {vertex multi-index: [(lo_k, hi_k) per axis]}.
    """
    d, n = mesh.dim, mesh.n

    def X(idx):
        return mesh.vertices[(slice(None),) + tuple(reversed(idx))]

    spans = {}
    for t in itertools.product(*[range(v + 1) for v in reversed(n)]):
        v = tuple(reversed(t))
        x0 = X(v)
        edges = []
        for a in range(d):
            for s in (-1, 1):
                w = list(v)
                w[a] += s
                if 0 <= w[a] <= n[a]:
                    edges.append(np.linalg.norm(X(w) - x0))
        target = ratio * max(edges)
        per_axis = []
        for a in range(d):
            ks = []
            for s in (-1, 1):
                k = 1
                while True:
                    w = list(v)
                    w[a] += s * k
                    if w[a] <= 0 or w[a] >= n[a] or np.linalg.norm(X(w) - x0) >= target:
                        break
                    k += 1
                ks.append(k)
            per_axis.append(tuple(ks))
        spans[v] = per_axis
    return spans


def box_indices(ranges, N):
    """Flattened global indices of the tensor box of 1D index ranges (x fastest)."""
    grids = np.meshgrid(*reversed(ranges), indexing="ij")
    idx = np.zeros(grids[0].shape, dtype=np.int64)
    stride = 1
    for a in range(len(ranges)):
        idx = idx + grids[len(ranges) - 1 - a] * stride
        stride *= N[a]
    return idx.ravel()


def box_pattern(ranges):
    """Structural 3^d-point pattern of a tensor box: |di|,|dj|,|dk| <= 1."""
    grids = np.meshgrid(*reversed(ranges), indexing="ij")
    coords = np.stack([g.ravel() for g in reversed(grids)], axis=1)
    diff = np.abs(coords[:, None, :] - coords[None, :, :])
    return np.all(diff <= 1, axis=2)


class LORPreconditioner:
    """B = P_0 R_0 P_0^T + sum_j R_j^T V_j R_j (Eq. (as)), with options for exact solves."""

    def __init__(self, mesh: Mesh, p: int, mg_levels: int = 0,
                 exact_local: bool = False, exact_coarse: bool = False, K_h=None,
                 patch_subset=None, coarse=True, ordering: str = "lex", weighting: str = "none",
                 patch_spans=None, post_smooth0: bool = True, patch_orders=None):
        """patch_subset: vertex multi-indices whose patches are built (default all);
        patch_spans: {vertex: [(lo_k, hi_k) per axis]} element spans of enlarged patches
        (`isotropic_overlap_spans`, Section 4.5); vertices not listed keep the vertex patch;
        coarse=False skips the coarse space (for checks of the patch part alone);
        ordering: ILU(0) ordering of every patch level, "lex" (patch-lexicographic),
        "mdf" or "rcm" (Section 3.4, `oracle.ordering`);
        weighting: "none" (unit weights, Eq. (as)), "count": the patch sum scaled on
        both sides by D^{-1/2}, D = number of patches containing each node (the counting
        matrix Section 4.1 names as future work), or "pou": each patch scaled on both
        sides by W_j = sqrt(theta_j), theta_j the Q1 vertex function of its vertex in
        the element reference coordinates at the level-0 nodes (`pou_weights`);
        post_smooth0=False leaves out the post-smoothing of the patch level 0 (the cycle
        the learned correction's replace variant completes);
        patch_orders: {(vertex, level): permutation} taken in place of the computed
        ordering for those patch levels (an order is not unique when the ordering's
        greedy choices tie, e.g. MDF on meshes with exact symmetries, so a check of
        another implementation's ILU(0) in its own order needs that order)."""
        self.patch_orders = patch_orders or {}
        self.post_smooth0 = post_smooth0
        self.ordering = ordering
        self.patch_spans = patch_spans or {}
        if weighting not in ("none", "count", "pou"):
            raise ValueError(f"unknown weighting {weighting!r}")
        self.weighting = weighting
        self.patch_subset = None if patch_subset is None else set(map(tuple, patch_subset))
        self.with_coarse = coarse
        self.mesh, self.p, self.dim = mesh, p, mesh.dim
        self.exact_local, self.exact_coarse = exact_local, exact_coarse
        n = mesh.n
        self.sels = level_selections(p, mg_levels)
        self.ms = [len(s) - 1 for s in self.sels]
        self.Ns = [tuple(v * m + 1 for v in n) for m in self.ms]
        self.K_h = assemble_lor(mesh, p) if K_h is None else K_h
        # global level operators A_l (Galerkin) and 1D/ND prolongations l+1 -> l
        self.P1 = []      # per level: list over axes of 1D matrices
        self.A = [self.K_h]
        for l in range(len(self.sels) - 1):
            mats = [prolong_1d(n[a], p, self.sels[l], self.sels[l + 1]) for a in range(self.dim)]
            self.P1.append(mats)
            P = kron_nd(mats)
            self.A.append((P.T @ self.A[l] @ P).tocsr())
        self._build_patches()
        if coarse:
            self._build_coarse()

    # ---------------------------------------------------------------- patches
    def vertices(self):
        return [tuple(reversed(t)) for t in
                itertools.product(*[range(v + 1) for v in reversed(self.mesh.n)])]

    def _build_patches(self):
        self.patches = []
        L = len(self.sels)
        for v in self.vertices():
            if self.patch_subset is not None and tuple(v) not in self.patch_subset:
                continue
            levels = []
            span = self.patch_spans.get(tuple(v), [(1, 1)] * self.dim)
            for l in range(L):
                ranges = [patch_range_1d(v[a], self.mesh.n[a], self.ms[l], *span[a]) for a in range(self.dim)]
                idx = box_indices(ranges, self.Ns[l])
                Aj = self.A[l][idx][:, idx].toarray() if len(idx) else np.zeros((0, 0))
                lev = {"ranges": ranges, "idx": idx, "A": Aj}
                if len(idx) and l < L - 1 and not self.exact_local:
                    pat = box_pattern(ranges)
                    if self.ordering == "lex":
                        lev["LU"] = ilu0(Aj, pat)
                    else:
                        perm = self.patch_orders.get((tuple(v), l))
                        if perm is None:
                            perm = ordering.order_for(self.ordering, Aj, pat)
                        perm = np.asarray(perm, dtype=np.int64)
                        lev["LU"] = ilu0(Aj[np.ix_(perm, perm)], pat[np.ix_(perm, perm)])
                        lev["perm"] = perm
                if l < L - 1:
                    rc = [patch_range_1d(v[a], self.mesh.n[a], self.ms[l + 1], *span[a])
                          for a in range(self.dim)]
                    mats = [self.P1[l][a][np.ix_(ranges[a], rc[a])] for a in range(self.dim)]
                    lev["P"] = kron_nd(mats).toarray() if all(len(r) for r in ranges + rc) \
                        else np.zeros((len(idx), int(np.prod([len(r) for r in rc]))))
                levels.append(lev)
            self.patches.append({"v": v, "levels": levels})

    def vcycle(self, levels, l, r):
        """One V(1,1) cycle on patch level l for right-hand side r (x0 = 0)."""
        lev = levels[l]
        if len(r) == 0:
            return np.zeros(0)
        if l == len(levels) - 1:
            return np.linalg.solve(lev["A"], r)
        A = lev["A"]
        x = self.smooth(lev, r)
        t = r - A @ x
        P = lev["P"]
        if P.shape[1] > 0:
            x = x + P @ self.vcycle(levels, l + 1, P.T @ t)
        if l == 0 and not self.post_smooth0:
            return x
        t = r - A @ x
        return x + self.smooth(lev, t)

    @staticmethod
    def smooth(lev, r):
        """(L U)^{-1} r with the level's ILU(0) factors, in the level's ordering."""
        L_, U_ = lev["LU"]
        perm = lev.get("perm")
        if perm is None:
            return ilu_solve(L_, U_, r)
        y = np.empty_like(r)
        y[perm] = ilu_solve(L_, U_, r[perm])
        return y

    def local_solve(self, j, r):
        """R_j applied to the patch residual: one V(1,1) cycle (Section 3.3), or A_j^{-1}."""
        levels = self.patches[j]["levels"]
        if self.exact_local:
            A0 = levels[0]["A"]
            return np.linalg.solve(A0, r) if len(r) else r
        return self.vcycle(levels, 0, r)

    # ----------------------------------------------------------------- coarse
    def _build_coarse(self):
        n, d = self.mesh.n, self.dim
        mats = [prolong_1d(n[a], self.p, list(range(self.p + 1)), [0, self.p]) for a in range(d)]
        self.P0 = kron_nd(mats)                                  # fine nodes x vertices
        A0 = (self.P0.T @ self.K_h @ self.P0).tocsr()
        Nv = tuple(v + 1 for v in n)
        self.vmask = ~boundary_mask(Nv)
        # coarse hierarchy on the vertex grid (1D point lists in vertex indices)
        pts = [list(range(v + 1)) for v in n]
        self.cA, self.cP, self.cmask = [], [], []
        Acur, mask, pcur = A0, self.vmask, pts
        while True:
            Ai = Acur[mask][:, mask].tocsr()
            self.cA.append(Ai)
            self.cmask.append(mask)
            if self.exact_coarse or Ai.shape[0] <= COARSE_DIRECT_MAX:
                break
            pnext = []
            mats = []
            for a in range(d):
                s = pcur[a]
                t = s[0::2]
                if t[-1] != s[-1]:
                    t = t + [s[-1]]
                Pa = np.zeros((len(s), len(t)))
                for i, g in enumerate(s):
                    b = next(k for k in range(len(t)) if t[k] >= g)
                    if t[b] == g:
                        Pa[i, b] = 1.0
                    else:
                        w = (g - t[b - 1]) / (t[b] - t[b - 1])
                        Pa[i, b - 1] = 1.0 - w
                        Pa[i, b] = w
                mats.append(Pa)
                pnext.append(t)
            P = kron_nd(mats)
            Acur = (P.T @ Acur @ P).tocsr()
            shape_next = tuple(len(t) for t in pnext)
            mnext = ~boundary_mask(shape_next)
            self.cP.append(P[mask][:, mnext].tocsr())
            mask, pcur = mnext, pnext
        self.cDl1 = [np.asarray(abs(Ai).sum(axis=1)).ravel() for Ai in self.cA]
        self.cInv = np.linalg.inv(self.cA[-1].toarray()) if self.cA[-1].shape[0] else None

    def coarse_vcycle(self, l, r):
        """One V-cycle on coarse level l (the R_0 reading in the module docstring)."""
        A = self.cA[l]
        if l == len(self.cA) - 1:
            return self.cInv @ r
        D = self.cDl1[l]
        x = np.zeros_like(r)
        for _ in range(COARSE_SWEEPS):
            x = x + (r - A @ x) / D
        P = self.cP[l]
        x = x + P @ self.coarse_vcycle(l + 1, P.T @ (r - A @ x))
        for _ in range(COARSE_SWEEPS):
            x = x + (r - A @ x) / D
        return x

    def coarse_solve(self, rc):
        """R_0 applied to interior-vertex vector rc."""
        if len(rc) == 0:
            return rc
        return self.coarse_vcycle(0, rc)

    # ------------------------------------------------------------------ apply
    def apply(self, r, parts=("patches", "coarse")):
        """B r = sum_j R_j^T V_j(R_j r) + P_0 R_0 P_0^T r (Eq. (as)); Dirichlet entries of r are ignored."""
        r = np.asarray(r, dtype=np.float64)
        z = np.zeros_like(r)
        N0 = self.Ns[0]
        rr = np.where(boundary_mask(N0), 0.0, r)
        if "patches" in parts:
            w = self.count_weights() if self.weighting == "count" else None
            rp = rr if w is None else w * rr
            zp = np.zeros_like(r)
            for j in range(len(self.patches)):
                idx = self.patches[j]["levels"][0]["idx"]
                if not len(idx):
                    continue
                if self.weighting == "pou":
                    wj = self.pou_weights(j)
                    zp[idx] += wj * self.local_solve(j, wj * rr[idx])
                else:
                    zp[idx] += self.local_solve(j, rp[idx])
            z += zp if w is None else w * zp
        if "coarse" in parts and self.with_coarse:
            rc = (self.P0.T @ rr)[self.vmask]
            ec = np.zeros(self.P0.shape[1])
            ec[self.vmask] = self.coarse_solve(rc)
            z += self.P0 @ ec
        return z

    def pou_weights(self, j):
        """sqrt(theta_j) at the level-0 nodes of patch j (its box order).

        Enlarged patches (patch_spans): the Q1 hat of the vertex does not cover the patch,
        so theta_j = psi_j / sum_k psi_k with psi_j a product of 1D tents that are linear
        in the physical coordinate along each axis (on the grid line through the vertex),
        1 at the vertex and 0 at the ends of the patch's span; the normalisation makes
        the weights a partition of unity whatever the spans are.

        theta_j is the Q1 (bilinear/trilinear) function of patch j's vertex v in the
        element reference coordinates: along axis a, 1 - s on the element whose left
        vertex is v and s on the element whose right vertex is v, with s the node's GLL
        coordinate in [0, 1].  These functions sum to one at every node and vanish on
        the patch boundary, so the weighted sum is a smooth partition of unity (the
        ingredient of the stable decomposition in Section 3.2).  An option beyond the
        paper, like the counting matrix."""
        if self.patch_spans:
            return self._tent_weights()[j]
        pt = self.patches[j]
        v = pt["v"]
        xg = gll(self.p)[0]
        hats = []
        for a, I in enumerate(pt["levels"][0]["ranges"]):
            e, s = I // self.p, xg[I % self.p]
            hats.append(np.where(e == v[a], 1.0 - s, s))
        grids = np.meshgrid(*reversed(hats), indexing="ij")
        return np.sqrt(np.prod([g.ravel() for g in grids], axis=0))

    def _tent_weights(self):
        """Normalised physical tents of every patch (see pou_weights)."""
        if getattr(self, "_tw", None) is not None:
            return self._tw
        p, d, N = self.p, self.dim, self.Ns[0]
        X = node_coordinates(self.mesh, p)

        def coord(v, a, i):
            """Coordinate a of the node with index i along axis a on the grid line through v."""
            idx = [v[b] * p for b in range(d)]
            idx[a] = i
            flat, stride = 0, 1
            for b in range(d):
                flat += idx[b] * stride
                stride *= N[b]
            return X[flat, a]

        psi = []
        for pt in self.patches:
            v = pt["v"]
            span = self.patch_spans.get(tuple(v), [(1, 1)] * d)
            tents = []
            for a, I in enumerate(pt["levels"][0]["ranges"]):
                lo, hi = span[a]
                xv = coord(v, a, v[a] * p)
                xlo = coord(v, a, max(v[a] - lo, 0) * p)
                xhi = coord(v, a, min(v[a] + hi, self.mesh.n[a]) * p)
                xs = np.array([coord(v, a, i) for i in I])
                t = np.where(xs <= xv, (xs - xlo) / (xv - xlo) if xv > xlo else 1.0,
                             (xhi - xs) / (xhi - xv) if xhi > xv else 1.0)
                tents.append(np.clip(t, 0.0, None))
            grids = np.meshgrid(*reversed(tents), indexing="ij")
            psi.append(np.prod([g.ravel() for g in grids], axis=0))
        total = np.zeros(int(np.prod(N)))
        for pt, s in zip(self.patches, psi):
            total[pt["levels"][0]["idx"]] += s
        self._tw = [np.sqrt(s / total[pt["levels"][0]["idx"]]) for pt, s in zip(self.patches, psi)]
        return self._tw

    def count_weights(self):
        """D^{-1/2} on the level-0 grid: D counts the built patches containing each node."""
        if getattr(self, "_cw", None) is None:
            cnt = np.zeros(int(np.prod(self.Ns[0])))
            for P in self.patches:
                cnt[P["levels"][0]["idx"]] += 1.0
            self._cw = np.where(cnt > 0, 1.0 / np.sqrt(np.maximum(cnt, 1.0)), 0.0)
        return self._cw

    def apply_hybrid(self, r):
        """Hybrid Schwarz: the coarse correction applied multiplicatively, the patches
        additively among themselves (the variant Section 4.1 names as future work after
        Lottes and Fischer), in the symmetric form
            B_hyb = B_0 + (I - B_0 K_h) B_loc (I - K_h B_0),
        B_loc = sum_j R_j^T V_j R_j, B_0 = P_0 R_0 P_0^T, K_h on the interior nodes.
        B_hyb is B_0 plus a congruence of B_loc, so it is symmetric positive definite
        without damping (the undamped smoother-coarse-smoother product is not: the
        overlapping patch sum alone has lambda_max(B_loc K_h) up to 2^d)."""
        r = np.asarray(r, dtype=np.float64)
        inner = ~boundary_mask(self.Ns[0])
        rr = np.where(inner, r, 0.0)

        def K(z):
            return np.where(inner, self.K_h @ np.where(inner, z, 0.0), 0.0)

        z0 = self.apply(rr, parts=("coarse",))
        z1 = self.apply(rr - K(z0), parts=("patches",))
        return z0 + z1 - self.apply(K(z1), parts=("coarse",))

    def patch_contribution(self, j, r):
        """R_j^T V_j(R_j r) scattered onto the full level-0 grid (for sampled checks)."""
        z = np.zeros(len(r))
        idx = self.patches[j]["levels"][0]["idx"]
        if len(idx):
            z[idx] = self.local_solve(j, np.where(boundary_mask(self.Ns[0]), 0.0, r)[idx])
        return z
