"""Tensor-product mesh geometry (oracle; FP64).

Section 2: every element D of T_p is the image of the unit cube [0,1]^d.  Here
the map is the multilinear (bilinear/trilinear) interpolation of the element's
2^d vertices (the reading used for all perturbed meshes).  Corner c of an
element has offsets (c & 1, (c >> 1) & 1, (c >> 2) & 1) along (x, y, z).

Curved elements (the curved meshes of Section 4.2): with a smooth map ``warp``
the element map becomes isoparametric, the degree-p Lagrange interpolant at the
(p+1)^d GLL points of warp(multilinear(xi)), so the high-order nodes lie on the
curved geometry and the map is continuous across shared faces.
"""
from __future__ import annotations

import itertools

import numpy as np

from .basis import gll, lagrange


class Mesh:
    """Structured-topology mesh with n = (nx, ny[, nz]) elements.

    warp: optional callable X (Q, d) -> (Q, d) applied to the multilinear image;
    the element map is then its isoparametric interpolant (module docstring)."""

    def __init__(self, vertices, kappa, warp=None):
        self.vertices = np.asarray(vertices, dtype=np.float64)
        self.kappa = np.asarray(kappa, dtype=np.float64)
        self.warp = warp
        self.dim = self.vertices.shape[0]
        self.n = tuple(reversed(self.kappa.shape))          # (nx, ny[, nz])
        assert len(self.n) == self.dim

    @property
    def nel(self):
        return int(np.prod(self.n))

    def elements(self):
        """Element multi-indices (ex, ey[, ez]) in lexicographic order (x fastest)."""
        for t in itertools.product(*[range(v) for v in reversed(self.n)]):
            yield tuple(reversed(t))

    def corners(self, e):
        """(2^d, d) vertex coordinates of element e, corner order c = cx + 2cy + 4cz."""
        d = self.dim
        out = np.empty((2 ** d, d))
        for c in range(2 ** d):
            off = [(c >> a) & 1 for a in range(d)]
            idx = tuple(reversed([e[a] + off[a] for a in range(d)]))
            out[c] = self.vertices[(slice(None),) + idx]
        return out

    def kappa_of(self, e):
        """The coefficient kappa_e of element e."""
        return float(self.kappa[tuple(reversed(e))])

    def element_map(self, e, xi, p):
        """X (Q, d) and J (Q, d, d) of element e at reference points xi: the multilinear
        map, or with a warp its degree-p isoparametric interpolant."""
        if self.warp is None:
            return multilinear(self.corners(e), xi)
        return isoparametric(self.corners(e), self.warp, p, xi)


def isoparametric(corners, warp, p, xi):
    """Degree-p interpolant of warp(multilinear(corners, .)) at the GLL points, and its
    Jacobian, at reference points xi (Q, d)."""
    corners = np.asarray(corners)
    xi = np.atleast_2d(xi)
    Q, d = xi.shape
    xg = gll(p)[0]
    grids = np.meshgrid(*([xg] * d), indexing="ij")               # axis 0 slowest
    nodes = np.stack([grids[d - 1 - a].ravel() for a in range(d)], axis=1)   # x fastest
    Xn = np.asarray(warp(multilinear(corners, nodes)[0]), dtype=np.float64)  # ((p+1)^d, d)
    B, D = zip(*[lagrange(xg, xi[:, a]) for a in range(d)])       # per axis (Q, p+1)
    idx = np.stack([np.indices([p + 1] * d)[d - 1 - a].ravel() for a in range(d)], axis=1)
    phi = np.ones((Q, len(nodes)))
    dphi = np.ones((d, Q, len(nodes)))
    for a in range(d):
        phi *= B[a][:, idx[:, a]]
        for b in range(d):
            dphi[b] *= (D[a] if a == b else B[a])[:, idx[:, a]]
    X = phi @ Xn
    J = np.einsum("bqn,na->qab", dphi, Xn)
    return X, J


def oriented_det(J):
    """det J at every point of a batch of Jacobians (..., d, d).

    An element of T_p is the image of the unit cube under an invertible map that
    keeps its orientation (Section 2), so det J > 0 at every quadrature point.  A
    map with det J <= 0 anywhere (an inverted or tangled element) is refused with
    ValueError rather than integrated with |det J|, the same rule the GPU setup
    applies."""
    det = np.linalg.det(J)
    if not np.all(det > 0):
        raise ValueError("inverted element: det J <= 0 at a quadrature point")
    return det


def multilinear(corners, xi):
    """Map reference points xi (Q, d) through the multilinear map of ``corners``.

    Returns X (Q, d) and the Jacobian J (Q, d, d) with J[q, a, b] = dX_a/dxi_b.
    """
    corners = np.asarray(corners)
    xi = np.atleast_2d(xi)
    Q, d = xi.shape
    X = np.zeros((Q, d))
    J = np.zeros((Q, d, d))
    for c in range(2 ** d):
        bits = [(c >> a) & 1 for a in range(d)]
        f = [xi[:, a] if bits[a] else 1.0 - xi[:, a] for a in range(d)]
        df = [np.ones(Q) if bits[a] else -np.ones(Q) for a in range(d)]
        shape = np.prod(f, axis=0)
        X += shape[:, None] * corners[c][None, :]
        for b in range(d):
            g = np.ones(Q)
            for a in range(d):
                g = g * (df[a] if a == b else f[a])
            J[:, :, b] += g[:, None] * corners[c][None, :]
    return X, J
