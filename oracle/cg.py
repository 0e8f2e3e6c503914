"""High-order continuous Q_p discretization (oracle; FP64, no sum factorization).

Section 2, Eq. (fem)/(system): K_p u = M_p f with K_p the stiffness matrix of
a(u,v) = (b grad u, grad v) on the Q_p space of GLL-nodal Lagrange functions,
homogeneous Dirichlet conditions.  The oracle forms every element matrix by
dense quadrature over all (p+1)^d basis functions (the "naive" O(p^{3d})
assembly the paper contrasts with sum factorization), assembles a sparse
global matrix, and eliminates every boundary node.

Reading (quadrature): q = p+1 Gauss-Legendre points per direction for the
stiffness, p+2 for the load vector.
Global numbering: node (I, J[, K]) of the N = p*n + 1 grid has index
(K*Ny + J)*Nx + I; boundary entries of vectors are held at zero.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from .basis import gauss_legendre, gll, lagrange
from .mesh import Mesh, multilinear, oriented_det


def node_shape(n, p):
    """(Nx, Ny[, Nz]) nodes per direction of the Q_p grid."""
    return tuple(p * v + 1 for v in n)


def tensor_basis(dim, p, pts1d):
    """Values and reference gradients of the (p+1)^d tensor basis at tensor points.

    Returns phi (Q, nb) and dphi (d, Q, nb); point and basis indices run x fastest.
    """
    B, D = lagrange(gll(p)[0], pts1d)

    def kron_list(mats):
        out = mats[0]
        for m in mats[1:]:
            out = np.kron(out, m)
        return out

    # kron(..z.., ..y.., ..x..) puts x fastest
    phi = kron_list([B] * dim)
    dphi = []
    for a in range(dim):
        mats = [D if (dim - 1 - k) == a else B for k in range(dim)]
        dphi.append(kron_list(mats))
    return phi, np.array(dphi)


def tensor_points(dim, pts1d, w1d):
    """Tensor points (Q, d) with x fastest, and product weights (Q,)."""
    grids = np.meshgrid(*([pts1d] * dim), indexing="ij")   # axis 0 slowest
    pts = np.stack([grids[dim - 1 - a].ravel() for a in range(dim)], axis=1)
    wg = np.meshgrid(*([w1d] * dim), indexing="ij")
    w = np.prod([g.ravel() for g in wg], axis=0)
    return pts, w


def element_stiffness(corners, kappa, p, q=None, geom=None):
    """Dense K_e[a,b] = sum_q w_q det J_q kappa grad phi_a . grad phi_b (det J > 0, `oriented_det`).

    kappa: the element's constant, or a callable b(X) of the physical points X (Q, d)
    (the variable coefficients of Section 4.2), evaluated at the quadrature points.
    geom: optional callable xi -> (X, J) replacing the multilinear map of corners
    (curved elements, `Mesh.element_map`)."""
    dim = corners.shape[1]
    q = p + 1 if q is None else q
    x1, w1 = gauss_legendre(q)
    pts, w = tensor_points(dim, x1, w1)
    _, dphi = tensor_basis(dim, p, x1)
    Xq, J = multilinear(corners, pts) if geom is None else geom(pts)
    if callable(kappa):
        kappa = np.asarray(kappa(Xq), dtype=np.float64)
    detJ = oriented_det(J)
    Jinv = np.linalg.inv(J)                      # (Q, d, d)
    # physical gradient: grad_x phi = J^{-T} grad_xi phi
    gphys = np.einsum("qba,bqn->aqn", Jinv, dphi)   # (d, Q, nb)
    wk = w * detJ * kappa
    return np.einsum("aqi,q,aqj->ij", gphys, wk, gphys)


def _geom(mesh: Mesh, e, p):
    """The element map of a curved element, None for the multilinear default."""
    if mesh.warp is None:
        return None
    return lambda pts: mesh.element_map(e, pts, p)


def element_nodes(e, p, N):
    """Global node indices of the (p+1)^d nodes of element e (x fastest)."""
    dim = len(e)
    rng = [np.arange(e[a] * p, e[a] * p + p + 1) for a in range(dim)]
    grids = np.meshgrid(*reversed(rng), indexing="ij")
    idx = np.zeros_like(grids[0])
    stride = 1
    for a in range(dim):
        idx = idx + grids[dim - 1 - a] * stride
        stride *= N[a]
    return idx.ravel()


def boundary_mask(N):
    """True on the Dirichlet (domain boundary) nodes of a grid of shape N (x first)."""
    dim = len(N)
    m = np.zeros(tuple(reversed(N)), dtype=bool)
    for ax in range(dim):
        sl = [slice(None)] * dim
        sl[ax] = 0
        m[tuple(sl)] = True
        sl[ax] = -1
        m[tuple(sl)] = True
    return m.ravel()


def assemble_stiffness(mesh: Mesh, p: int, coef=None):
    """Assembled K_p over all grid nodes (no Dirichlet elimination), CSR.

    coef: optional callable b(X) replacing the per-element kappa (Section 4.2)."""
    N = node_shape(mesh.n, p)
    ntot = int(np.prod(N))
    rows, cols, vals = [], [], []
    for e in mesh.elements():
        Ke = element_stiffness(mesh.corners(e), mesh.kappa_of(e) if coef is None else coef, p,
                               geom=_geom(mesh, e, p))
        idx = element_nodes(e, p, N)
        rows.append(np.repeat(idx, len(idx)))
        cols.append(np.tile(idx, len(idx)))
        vals.append(Ke.ravel())
    K = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                      shape=(ntot, ntot)).tocsr()
    K.sum_duplicates()
    return K


def dirichlet_operator(K, N):
    """K with boundary rows and columns removed (zeroed): Pi K Pi."""
    interior = (~boundary_mask(N)).astype(np.float64)
    Pi = sp.diags(interior)
    return (Pi @ K @ Pi).tocsr()


def apply_A(K, N, x):
    """y = Pi K Pi x: boundary inputs ignored, boundary outputs zero."""
    m = ~boundary_mask(N)
    xx = np.where(m, x, 0.0)
    return np.where(m, K @ xx, 0.0)


def apply_A_rows(mesh: Mesh, p: int, x, rows):
    """(Pi K Pi x)[rows] computed row by row from the element matrices.

    Only the (up to 2^d) elements that contain each requested node are formed,
    so single outputs of very large problems can be checked.
    """
    N = node_shape(mesh.n, p)
    bmask = boundary_mask(N)
    dim = mesh.dim
    out = np.zeros(len(rows))
    cache = {}
    for r_i, r in enumerate(rows):
        if bmask[r]:
            continue
        I = []
        rem = int(r)
        for a in range(dim):
            I.append(rem % N[a])
            rem //= N[a]
        # elements containing node I: ex in {I//p - 1, I//p} when I%p==0, else I//p
        cand = []
        for a in range(dim):
            c = {I[a] // p, (I[a] - 1) // p} if I[a] % p == 0 else {I[a] // p}
            cand.append(sorted(v for v in c if 0 <= v < mesh.n[a]))
        import itertools
        acc = 0.0
        for e in itertools.product(*cand):
            if e not in cache:
                cache[e] = element_stiffness(mesh.corners(e), mesh.kappa_of(e), p, geom=_geom(mesh, e, p))
            Ke = cache[e]
            idx = element_nodes(e, p, N)
            loc = int(np.nonzero(idx == r)[0][0])
            xe = np.where(bmask[idx], 0.0, x[idx])
            acc += Ke[loc] @ xe
        out[r_i] = acc
    return out


def load_vector(mesh: Mesh, p: int, f, q=None):
    """b_a = sum_e sum_q w_q det J f(X_q) phi_a(X_q) with q-point GL (default p+2); boundary zeroed."""
    N = node_shape(mesh.n, p)
    ntot = int(np.prod(N))
    x1, w1 = gauss_legendre(p + 2 if q is None else q)
    pts, w = tensor_points(mesh.dim, x1, w1)
    phi, _ = tensor_basis(mesh.dim, p, x1)
    b = np.zeros(ntot)
    for e in mesh.elements():
        X, J = mesh.element_map(e, pts, p)
        fv = f(X)
        wq = w * oriented_det(J) * fv
        np.add.at(b, element_nodes(e, p, N), phi.T @ wq)
    b[boundary_mask(N)] = 0.0
    return b


def node_coordinates(mesh: Mesh, p: int):
    """Physical coordinates (ntot, d) of every GLL node: the element map at GLL points."""
    N = node_shape(mesh.n, p)
    ntot = int(np.prod(N))
    xg = gll(p)[0]
    pts, _ = tensor_points(mesh.dim, xg, np.ones(p + 1))
    X = np.zeros((ntot, mesh.dim))
    for e in mesh.elements():
        Xe, _ = mesh.element_map(e, pts, p)
        X[element_nodes(e, p, N)] = Xe
    return X


def l2_error(mesh: Mesh, p: int, u, exact):
    """|| u_h - exact ||_{L2} with (p+3)-point GL per direction."""
    N = node_shape(mesh.n, p)
    x1, w1 = gauss_legendre(p + 3)
    pts, w = tensor_points(mesh.dim, x1, w1)
    phi, _ = tensor_basis(mesh.dim, p, x1)
    err = 0.0
    for e in mesh.elements():
        X, J = mesh.element_map(e, pts, p)
        uh = phi @ u[element_nodes(e, p, N)]
        err += np.sum(w * oriented_det(J) * (uh - exact(X)) ** 2)
    return np.sqrt(err)
