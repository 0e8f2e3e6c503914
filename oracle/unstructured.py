"""Q_p, LOR and vertex-patch additive Schwarz on unstructured quadrilateral meshes
(oracle; FP64; 2D).  TEST INFRASTRUCTURE ONLY.

Section 4.2 runs the method on unstructured quadrilateral meshes: the patch of a
vertex is the union of the elements around it (any number of them), each element
is refined at its own GLL points, and the element-structured hierarchy coarsens
every element separately (Section 3.3).  This module restates the pieces for
general connectivity:

* numbering (level with kept GLL subset `sel` of m+1 points per edge): vertices,
  then the m-1 nodes of every edge counted from its lower-numbered vertex, then the
  (m-1)^2 interior nodes of every element (x fastest);
* K_p by the dense element quadrature of `oracle.cg`, K_h by the Q1 sub-cell
  stiffness of `oracle.lor`, P_0 by the bilinear map of each element;
* R_j: the open interior of the union of the elements at vertex j, minus Dirichlet
  nodes; B = P_0 A_0^{-1} P_0^T + sum_j R_j^T V_j R_j with V_j = A_j^{-1} or one
  V(1,1) cycle of the element-structured hierarchy with ILU(0) in MDF order (the
  ordering Section 3.4 uses; lexicographic order has no meaning here).

Reading (orientation): two elements may run along a shared edge in opposite
directions.  The kept subsets of the hierarchy ("every other point from the left")
then select the same edge nodes from both sides only if the subset is symmetric,
sel[m - t] = p - sel[t].  That holds at every level for p = 2, 4, 8; the hierarchy
here is built for such p only (others raise), exact patch solves for any p.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from . import ordering
from .basis import gll
from .cg import element_stiffness, tensor_points
from .lor import ilu0, ilu_solve, level_selections, q1_stiffness_batch
from .mesh import multilinear


class QuadMesh:
    """vertices (nv, 2); quads (nq, 4) corner vertex ids in the order (0,0), (1,0), (0,1),
    (1,1) of the reference square; kappa (nq,)."""

    def __init__(self, vertices, quads, kappa):
        self.vertices = np.asarray(vertices, dtype=np.float64)
        self.quads = np.asarray(quads, dtype=np.int64)
        self.kappa = np.asarray(kappa, dtype=np.float64)
        self.nv, self.nq = len(self.vertices), len(self.quads)
        # local edges as (corner a, corner b) with the local coordinate running a -> b
        self.local_edges = [(0, 1), (2, 3), (0, 2), (1, 3)]     # bottom, top, left, right
        self.edges = {}
        count = {}
        for q in self.quads:
            for a, b in self.local_edges:
                key = (min(q[a], q[b]), max(q[a], q[b]))
                if key not in self.edges:
                    self.edges[key] = len(self.edges)
                count[key] = count.get(key, 0) + 1
        self.boundary_edges = {k for k, c in count.items() if c == 1}
        self.boundary_vertices = {v for k in self.boundary_edges for v in k}


class Level:
    """Global node numbering of one level: GLL subset `sel` (m = len(sel) - 1 per edge)."""

    def __init__(self, mesh: QuadMesh, p: int, sel):
        self.sel = list(sel)
        m = len(sel) - 1
        self.m = m
        ne = len(mesh.edges)
        self.ntot = mesh.nv + ne * (m - 1) + mesh.nq * (m - 1) ** 2
        self.local = np.zeros((mesh.nq, (m + 1) ** 2), dtype=np.int64)   # element-local (x fastest) -> global
        bnd = np.zeros(self.ntot, dtype=bool)
        for e, q in enumerate(mesh.quads):
            g = np.full((m + 1, m + 1), -1, dtype=np.int64)              # g[j, i]
            g[0, 0], g[0, m], g[m, 0], g[m, m] = q[0], q[1], q[2], q[3]
            sides = {(0, 1): [(0, t) for t in range(m + 1)], (2, 3): [(m, t) for t in range(m + 1)],
                     (0, 2): [(t, 0) for t in range(m + 1)], (1, 3): [(t, m) for t in range(m + 1)]}
            for (a, b), cells in sides.items():
                key = (min(q[a], q[b]), max(q[a], q[b]))
                base = mesh.nv + mesh.edges[key] * (m - 1)
                for t in range(1, m):
                    k = t - 1 if q[a] < q[b] else m - 1 - t
                    g[cells[t]] = base + k
                    if key in mesh.boundary_edges:
                        bnd[base + k] = True
            base = mesh.nv + ne * (m - 1) + e * (m - 1) ** 2
            for j in range(1, m):
                for i in range(1, m):
                    g[j, i] = base + (j - 1) * (m - 1) + (i - 1)
            self.local[e] = g.ravel()
        for v in mesh.boundary_vertices:
            bnd[v] = True
        self.boundary = bnd
        xg = gll(p)[0][self.sel]
        pts, _ = tensor_points(2, xg, np.ones(m + 1))
        self.X = np.zeros((self.ntot, 2))
        for e, q in enumerate(mesh.quads):
            self.X[self.local[e]] = multilinear(mesh.vertices[q], pts)[0]


def _symmetric(sel, p):
    m = len(sel) - 1
    return all(sel[m - t] == p - sel[t] for t in range(m + 1))


def assemble_stiffness(mesh: QuadMesh, p: int, lev0: Level):
    """K_p over all nodes (no Dirichlet elimination), CSR (Eq. (fem), dense element quadrature)."""
    rows, cols, vals = [], [], []
    for e, q in enumerate(mesh.quads):
        Ke = element_stiffness(mesh.vertices[q], float(mesh.kappa[e]), p)
        idx = lev0.local[e]
        rows.append(np.repeat(idx, len(idx)))
        cols.append(np.tile(idx, len(idx)))
        vals.append(Ke.ravel())
    K = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                      shape=(lev0.ntot, lev0.ntot)).tocsr()
    K.sum_duplicates()
    return K


def assemble_lor(mesh: QuadMesh, lev: Level):
    """K_h on the GLL-refined sub-cells of every element (Section 3.1), CSR."""
    m = lev.m
    corner_ids, kap = [], []
    for e in range(mesh.nq):
        g = lev.local[e].reshape(m + 1, m + 1)
        for j in range(m):
            for i in range(m):
                corner_ids.append([g[j, i], g[j, i + 1], g[j + 1, i], g[j + 1, i + 1]])
                kap.append(mesh.kappa[e])
    corner_ids = np.array(corner_ids)
    Kc = q1_stiffness_batch(lev.X[corner_ids], np.array(kap))
    K = sp.coo_matrix((Kc.ravel(), (np.repeat(corner_ids, 4, axis=1).ravel(), np.tile(corner_ids, (1, 4)).ravel())),
                      shape=(lev.ntot, lev.ntot)).tocsr()
    K.sum_duplicates()
    return K


def sub_cell_pattern(lev: Level, n_elems):
    """Structural pattern: nodes that share a sub-cell of the level (the Q1 stencil)."""
    m = lev.m
    r, c = [], []
    for e in range(n_elems):
        g = lev.local[e].reshape(m + 1, m + 1)
        for j in range(m):
            for i in range(m):
                ids = [g[j, i], g[j, i + 1], g[j + 1, i], g[j + 1, i + 1]]
                r += [a for a in ids for _ in ids]
                c += [b for _ in ids for b in ids]
    return sp.coo_matrix((np.ones(len(r), dtype=bool), (r, c)), shape=(lev.ntot, lev.ntot)).tocsr().astype(bool)


def element_prolongation(mesh: QuadMesh, p: int, fine: Level, coarse: Level):
    """P (fine x coarse): tensor 1D linear interpolation in each element's reference
    coordinate between the kept points (Section 3.3); a node shared by elements gets
    the same row from each of them."""
    xg = gll(p)[0]
    mf, mc = fine.m, coarse.m
    P1 = np.zeros((mf + 1, mc + 1))
    for t, gidx in enumerate(fine.sel):
        a = max(i for i in range(mc + 1) if coarse.sel[i] <= gidx)
        if coarse.sel[a] == gidx:
            P1[t, a] = 1.0
            continue
        w = (xg[gidx] - xg[coarse.sel[a]]) / (xg[coarse.sel[a + 1]] - xg[coarse.sel[a]])
        P1[t, a], P1[t, a + 1] = 1.0 - w, w
    Pe = np.kron(P1, P1)                    # local (x fastest) fine x coarse
    P = sp.lil_matrix((fine.ntot, coarse.ntot))
    done = np.zeros(fine.ntot, dtype=bool)
    for e in range(mesh.nq):
        fi, ci = fine.local[e], coarse.local[e]
        for a, gf in enumerate(fi):
            if done[gf]:
                continue
            done[gf] = True
            for b in np.nonzero(Pe[a])[0]:
                P[gf, ci[b]] = Pe[a, b]
    return P.tocsr()


def coarse_basis(mesh: QuadMesh, p: int, lev0: Level):
    """P_0 (nodes x vertices): the bilinear vertex functions of each element at its GLL nodes."""
    return element_prolongation(mesh, p, lev0, Level(mesh, p, [0, p]))


class UnstructuredLOR:
    """B = P_0 A_0^{-1} P_0^T + sum_j R_j^T V_j R_j (Eq. (as)) on a QuadMesh."""

    def __init__(self, mesh: QuadMesh, p: int, local: str = "vcycle", weighting: str = "none"):
        """local: "vcycle" or "exact" patch solves; weighting: "none" (Eq. (as)) or "pou":
        patch j scaled on both sides by sqrt(theta_j), theta_j = column j of P_0 (the
        bilinear vertex function, a partition of unity over the patches)."""
        if local not in ("vcycle", "exact") or weighting not in ("none", "pou"):
            raise ValueError((local, weighting))
        self.weighting = weighting
        self.mesh, self.p, self.local_kind = mesh, p, local
        sels = level_selections(p) if local == "vcycle" else [list(range(p + 1)), [0, p]]
        if local == "vcycle" and not all(_symmetric(s, p) for s in sels):
            raise NotImplementedError(f"p = {p}: the kept subsets are not symmetric (module docstring)")
        self.levels = [Level(mesh, p, s) for s in sels]
        self.K_h = assemble_lor(mesh, self.levels[0])
        self.A = [self.K_h]
        self.P = []
        for l in range(len(self.levels) - 1):
            P = element_prolongation(mesh, p, self.levels[l], self.levels[l + 1])
            self.P.append(P)
            self.A.append((P.T @ self.A[l] @ P).tocsr())
        self.P0 = coarse_basis(mesh, p, self.levels[0])
        vin = np.array([v not in mesh.boundary_vertices for v in range(mesh.nv)])
        self.vin = vin
        A0 = (self.P0.T @ self.K_h @ self.P0).toarray()[np.ix_(vin, vin)]
        self.A0inv = np.linalg.inv(A0) if A0.shape[0] else np.zeros((0, 0))
        self._build_patches()

    def _patch_nodes(self, lev: Level, elems):
        """Open interior of the union of `elems` on level lev, minus Dirichlet nodes."""
        inside = set(lev.local[list(elems)].ravel().tolist())
        others = [e for e in range(self.mesh.nq) if e not in elems]
        outside = set(lev.local[others].ravel().tolist()) if others else set()
        return np.array(sorted(g for g in inside - outside if not lev.boundary[g]), dtype=np.int64)

    def _build_patches(self):
        around = [[] for _ in range(self.mesh.nv)]
        for e, q in enumerate(self.mesh.quads):
            for v in q:
                around[v].append(e)
        pats = [sub_cell_pattern(lev, self.mesh.nq) for lev in self.levels]
        self.patches = []
        for v in range(self.mesh.nv):
            elems = set(around[v])
            lv = []
            for l, lev in enumerate(self.levels):
                idx = self._patch_nodes(lev, elems)
                Aj = self.A[l][idx][:, idx].toarray()
                d = {"idx": idx, "A": Aj}
                if self.local_kind == "vcycle" and l < len(self.levels) - 1 and len(idx):
                    pat = pats[l][idx][:, idx].toarray()
                    perm = ordering.mdf_order(Aj, pat)
                    d["perm"] = perm
                    d["LU"] = ilu0(Aj[np.ix_(perm, perm)], pat[np.ix_(perm, perm)])
                lv.append(d)
            if self.local_kind == "vcycle":
                for l in range(len(self.levels) - 1):
                    lv[l]["P"] = self.P[l][lv[l]["idx"]][:, lv[l + 1]["idx"]].toarray()
            self.patches.append({"v": v, "levels": lv})

    @staticmethod
    def smooth(d, r):
        """(L U)^{-1} r in the level's MDF order (one ILU(0) smoothing, Section 3.4)."""
        y = np.empty_like(r)
        y[d["perm"]] = ilu_solve(*d["LU"], r[d["perm"]])
        return y

    def vcycle(self, lv, l, r):
        """One V(1,1) cycle on patch level l (Section 3.3); exact on the vertex level."""
        if len(r) == 0:
            return np.zeros(0)
        A = lv[l]["A"]
        if l == len(lv) - 1:
            return np.linalg.solve(A, r)
        x = self.smooth(lv[l], r)
        P = lv[l]["P"]
        if P.shape[1] > 0:
            x = x + P @ self.vcycle(lv, l + 1, P.T @ (r - A @ x))
        return x + self.smooth(lv[l], r - A @ x)

    def apply(self, r, parts=("patches", "coarse")):
        """B r; Dirichlet entries of r are ignored and returned as 0."""
        bnd = self.levels[0].boundary
        rr = np.where(bnd, 0.0, np.asarray(r, dtype=np.float64))
        z = np.zeros_like(rr)
        if "patches" in parts:
            for pt in self.patches:
                lv = pt["levels"]
                idx = lv[0]["idx"]
                if not len(idx):
                    continue
                w = np.sqrt(self.P0[idx, pt["v"]].toarray().ravel()) if self.weighting == "pou" else 1.0
                rj = w * rr[idx]
                zj = np.linalg.solve(lv[0]["A"], rj) if self.local_kind == "exact" else self.vcycle(lv, 0, rj)
                z[idx] += w * zj
        if "coarse" in parts and self.A0inv.shape[0]:
            ec = np.zeros(self.mesh.nv)
            ec[self.vin] = self.A0inv @ (self.P0.T @ rr)[self.vin]
            z += self.P0 @ ec
        return z
