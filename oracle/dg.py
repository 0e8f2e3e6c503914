"""Interior-penalty and BR2 DG discretizations and the DG preconditioner (oracle; FP64).

Section 2.1, Eq. (ip) and Eq. (br2), with the coefficient b carried into the
fluxes:
  a(u,v) = sum_D (b grad u, grad v)_D
           - <{b grad u}, [[v]]> - <[[u]], {b grad v}> + penalty,
  IP penalty:  <sigma [[u]], [[v]]>,  sigma = eta p^2 b_F / h_F,
  BR2 penalty: sum_e eta (b r_e([[u]]), r_e([[v]])), r_e the lifting of Eq. (lift).
Dirichlet faces take one-sided traces with u+ = 0.
Readings (the paper fixes b = 1 and no quadrature):
  * volume terms: (p+1)^d Gauss-Legendre points (as in the CG operator);
    face terms: (p+1)^(d-1) Gauss-Legendre points on each face;
  * b_F = max(b-, b+), h_F = min(|D-|, |D+|) / |F| (|D-| / |F| on the boundary);
  * BR2 lifting with the GLL-lumped element mass and GLL face quadrature: r_e is
    then nonzero only at the GLL nodes of the face and the penalty is nodal,
    eta b_K (w_f |J_f|)^2 / (c w_n |J_K|) per side K, with c = 4 on interior
    faces ({tau} = tau_K / 2) and c = 1 on boundary faces.
Section 3.5, Eq. (dg-decomp) and Eq. (dg-as): V_DG = V_B + V_p,
  B_DG = R_B Q_B + R_p Q_p with R_B point Jacobi on the element-boundary
  nodes and R_p the conforming LOR preconditioner B of Eq. (as).
DG vectors are element-major blocks of (p+1)^d GLL-nodal values (x fastest).
"""
from __future__ import annotations

import itertools

import numpy as np
import scipy.sparse as sp

from .basis import gauss_legendre, gll, lagrange
from .cg import boundary_mask, element_stiffness, node_shape, tensor_points
from .mesh import Mesh, multilinear, oriented_det


def basis_at(p, pts):
    """Values (P, nb) and reference gradients (d, P, nb) of the tensor GLL basis at points (P, d)."""
    pts = np.atleast_2d(pts)
    P, d = pts.shape
    xg = gll(p)[0]
    Bs, Ds = [], []
    for a in range(d):
        B, D = lagrange(xg, pts[:, a])
        Bs.append(B)
        Ds.append(D)
    Q = p + 1
    nb = Q ** d
    idx = np.array(list(itertools.product(range(Q), repeat=d)))[:, ::-1]   # (nb, d), x fastest
    phi = np.ones((P, nb))
    for a in range(d):
        phi *= Bs[a][:, idx[:, a]]
    dphi = np.ones((d, P, nb))
    for b in range(d):
        for a in range(d):
            dphi[b] *= (Ds[a] if a == b else Bs[a])[:, idx[:, a]]
    return phi, dphi


def elem_index(e, n):
    """Lexicographic element number of multi-index e (x fastest)."""
    out, stride = 0, 1
    for a in range(len(n)):
        out += e[a] * stride
        stride *= n[a]
    return out


def face_points(d, a, side, x1):
    """Reference points of the face xi_a = side in element coords, tensor in the other axes."""
    others = [b for b in range(d) if b != a]
    grids = np.meshgrid(*([x1] * (d - 1)), indexing="ij")     # slowest first
    pts = np.zeros((len(x1) ** (d - 1), d))
    for t, b in enumerate(others):
        pts[:, b] = grids[d - 2 - t].ravel()
    pts[:, a] = float(side)
    return pts


def element_volume(corners, p):
    """|D| by (p+1)^d-point Gauss quadrature of det J (the h_F of the SIPG penalty, Section 2.1)."""
    x1, w1 = gauss_legendre(p + 1)
    pts, w = tensor_points(corners.shape[1], x1, w1)
    _, J = multilinear(corners, pts)
    return float(np.sum(w * oriented_det(J)))


def face_geometry(corners, a, side, pts, w):
    """Outward unit normal (P, d) and area weights w |J_f| (P,) by Nanson's formula."""
    _, J = multilinear(corners, pts)
    detJ = oriented_det(J)
    Jit = np.transpose(np.linalg.inv(J), (0, 2, 1))            # J^{-T}
    g = Jit[:, :, a] * (1.0 if side == 1 else -1.0)           # J^{-T} (+-e_a)
    gn = np.linalg.norm(g, axis=1)
    return g / gn[:, None], w * detJ * gn


def assemble_dg(mesh: Mesh, p: int, eta: float, form: str = "ip"):
    """Assembled A_IP or A_BR2 (CSR) on the element-major DG space."""
    if getattr(mesh, "warp", None) is not None:
        raise NotImplementedError("the DG oracle takes multilinear elements only")
    d = mesh.dim
    n = mesh.n
    Q = p + 1
    nb = Q ** d
    ndof = mesh.nel * nb
    rows, cols, vals = [], [], []

    def add(Ablk, e1, e2):
        i1, i2 = elem_index(e1, n) * nb, elem_index(e2, n) * nb
        r, c = np.meshgrid(np.arange(nb) + i1, np.arange(nb) + i2, indexing="ij")
        rows.append(r.ravel())
        cols.append(c.ravel())
        vals.append(Ablk.ravel())

    vol = {}
    for e in mesh.elements():
        add(element_stiffness(mesh.corners(e), mesh.kappa_of(e), p), e, e)
        vol[e] = element_volume(mesh.corners(e), p)
    x1, w1 = gauss_legendre(p + 1)
    xg, wg = gll(p)
    wfq = np.prod(np.meshgrid(*([w1] * (d - 1)), indexing="ij"), axis=0).ravel() if d > 1 else np.ones(1)
    wfg = np.prod(np.meshgrid(*([wg] * (d - 1)), indexing="ij"), axis=0).ravel() if d > 1 else np.ones(1)
    w_end = wg[0]

    for a in range(d):
        others = [b for b in range(d) if b != a]
        for t in itertools.product(*[range(n[b]) for b in reversed(others)]):
            t = t[::-1]
            for ia in range(n[a] + 1):
                def elem(ix):
                    e = [0] * d
                    e[a] = ix
                    for k, b in enumerate(others):
                        e[b] = t[k]
                    return tuple(e)
                sides = []
                if ia > 0:
                    sides.append((elem(ia - 1), 1))     # face at xi_a = 1 of the lower element
                if ia < n[a]:
                    sides.append((elem(ia), 0))         # face at xi_a = 0 of the upper element
                interior = len(sides) == 2
                # geometry from the first side (shared face, same parametrisation)
                e0, s0 = sides[0]
                pts0 = face_points(d, a, s0, x1)
                nrm, dA = face_geometry(mesh.corners(e0), a, s0, pts0, wfq)
                area = float(np.sum(dA))
                kap = [mesh.kappa_of(e) for e, _ in sides]
                if interior:
                    kF = max(kap)
                    hF = min(vol[sides[0][0]], vol[sides[1][0]]) / area
                else:
                    kF = kap[0]
                    hF = vol[e0] / area
                sigma = eta * p * p * kF / hF
                # per side: trace values and normal fluxes b grad phi . n (n outward of side 0)
                vals_s, flux_s = [], []
                for (e, s), k in zip(sides, kap):
                    pts = face_points(d, a, s, x1)
                    phi, dphi = basis_at(p, pts)
                    _, J = multilinear(mesh.corners(e), pts)
                    Jinv = np.linalg.inv(J)
                    gphys = np.einsum("qba,bqn->aqn", Jinv, dphi)     # J^{-T} grad_ref
                    vals_s.append(phi)
                    flux_s.append(k * np.einsum("qa,aqn->qn", nrm, gphys))
                sign = [1.0, -1.0]
                half = 0.5 if interior else 1.0
                Jm = [sign[k] * vals_s[k] for k in range(len(sides))]          # jump along n
                Av = [half * flux_s[k] for k in range(len(sides))]             # average flux
                for k1 in range(len(sides)):
                    for k2 in range(len(sides)):
                        blk = -(Jm[k1].T * dA) @ Av[k2] - (Av[k1].T * dA) @ Jm[k2]
                        if form == "ip":
                            blk = blk + sigma * (Jm[k1].T * dA) @ Jm[k2]
                        add(blk, sides[k1][0], sides[k2][0])
                if form == "br2":
                    # lumped lifting: nodal penalty at the GLL nodes of the face
                    ptsg0 = face_points(d, a, s0, xg)
                    _, dAg = face_geometry(mesh.corners(e0), a, s0, ptsg0, wfg)   # w_f |J_f|
                    beta = np.zeros(len(wfg))
                    for (e, s), k in zip(sides, kap):
                        ptsg = face_points(d, a, s, xg)
                        _, J = multilinear(mesh.corners(e), ptsg)
                        detJ = oriented_det(J)
                        c = 4.0 if interior else 1.0
                        beta += eta * k * dAg ** 2 / (c * wfg * w_end * detJ)
                    jm = []
                    for k2, (e, s) in enumerate(sides):
                        ptsg = face_points(d, a, s, xg)
                        phi, _ = basis_at(p, ptsg)
                        jm.append(sign[k2] * phi)
                    for k1 in range(len(sides)):
                        for k2 in range(len(sides)):
                            add((jm[k1].T * beta) @ jm[k2], sides[k1][0], sides[k2][0])
    A = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                      shape=(ndof, ndof)).tocsr()
    A.sum_duplicates()
    return A


def injection(mesh: Mesh, p: int):
    """E: conforming L-vector (all nodes, boundary columns dropped) -> DG vector."""
    d = mesh.dim
    N = node_shape(mesh.n, p)
    Q = p + 1
    nb = Q ** d
    bmask = boundary_mask(N)
    rows, cols = [], []
    loc = np.array(list(itertools.product(range(Q), repeat=d)))[:, ::-1]
    strides = np.cumprod([1] + list(N[:-1]))
    for e in mesh.elements():
        base = elem_index(e, mesh.n) * nb
        g = ((np.array(e)[None, :] * p + loc) * strides).sum(axis=1)
        keep = ~bmask[g]
        rows.append(base + np.arange(nb)[keep])
        cols.append(g[keep])
    r = np.concatenate(rows)
    c = np.concatenate(cols)
    return sp.csr_matrix((np.ones(len(r)), (r, c)), shape=(mesh.nel * nb, int(np.prod(N))))


def boundary_dofs(mesh: Mesh, p: int):
    """True on element-boundary GLL nodes (the support of V_B)."""
    d = mesh.dim
    Q = p + 1
    loc = np.array(list(itertools.product(range(Q), repeat=d)))[:, ::-1]
    onb = np.any((loc == 0) | (loc == p), axis=1)
    return np.tile(onb, mesh.nel)


class DGPreconditioner:
    """B_DG = R_B Q_B + R_p Q_p (Eq. (dg-as)): point Jacobi on V_B plus E B E^T."""

    def __init__(self, mesh: Mesh, p: int, A_dg, cg_prec):
        self.E = injection(mesh, p)
        self.vb = boundary_dofs(mesh, p)
        self.d = A_dg.diagonal()
        self.B = cg_prec

    def apply(self, r):
        """diag(A_DG)^{-1} r on the element-boundary nodes V_B plus E B E^T r (Eq. (dg-as))."""
        z = np.where(self.vb, r / self.d, 0.0)
        return z + self.E @ self.B.apply(self.E.T @ r)


def load_vector_dg(mesh: Mesh, p: int, f, q=None):
    """Element-local b_e = int_D f phi with q-point Gauss-Legendre (default p+1)."""
    d = mesh.dim
    Q = p + 1
    x1, w1 = gauss_legendre(p + 1 if q is None else q)
    pts, w = tensor_points(d, x1, w1)
    phi, _ = basis_at(p, pts)
    b = np.zeros(mesh.nel * Q ** d)
    for e in mesh.elements():
        X, J = multilinear(mesh.corners(e), pts)
        base = elem_index(e, mesh.n) * Q ** d
        b[base:base + Q ** d] = phi.T @ (w * oriented_det(J) * f(X))
    return b
