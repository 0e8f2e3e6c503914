"""Seeded synthetic inputs: perturbed tensor-product meshes and element coefficients.

This module is the only code shared by the CUDA path's tests/bench and the CPU
oracle.  It holds none of the method's arithmetic: it only draws random numbers
and lays out the mesh vertices and the per-element coefficient, which are the
*inputs* of the solver (the model problem of Section 2, Eq. (poisson), on a
tensor-product mesh of [0,1]^d whose elements are images of the unit cube).

Random numbers come from one counter-based generator, SplitMix64 (Steele, Lea &
Flood, "Fast splittable pseudorandom number generators", OOPSLA 2014): the i-th
draw of stream ``key`` is ``mix64(key + (i+1)*GAMMA)``.  Uniforms in [0,1) take
the top 53 bits; standard normals use the Box-Muller transform on consecutive
pairs of uniforms.

Layouts (all float64, C order):
  * vertices: shape (d, nz+1, ny+1, nx+1) for d=3, (d, ny+1, nx+1) for d=2;
    component c of vertex (i,j,k) sits at vertices[c, k, j, i] (x fastest).
  * kappa: shape (nz, ny, nx) (or (ny, nx)); element (ex,ey,ez) at [ez, ey, ex].
"""
from __future__ import annotations

import numpy as np

GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def mix64(z: np.ndarray) -> np.ndarray:
    """SplitMix64 output finaliser applied elementwise to uint64 values."""
    z = np.asarray(z, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def splitmix64(key: int, count: int, start: int = 0) -> np.ndarray:
    """Draws start..start+count-1 of the SplitMix64 sequence seeded with ``key``."""
    i = np.arange(start + 1, start + count + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        state = np.uint64(key & 0xFFFFFFFFFFFFFFFF) + i * GAMMA
    return mix64(state)


def stream_key(seed: int, tag: int) -> int:
    """Independent stream per (seed, purpose tag)."""
    z = mix64(np.array([(seed * 0x100000001B3 + tag * 0x9E3779B1) & 0xFFFFFFFFFFFFFFFF],
                       dtype=np.uint64))
    return int(z[0])


def uniform01(key: int, count: int) -> np.ndarray:
    """Uniform doubles in [0,1) from the top 53 bits of each draw."""
    return (splitmix64(key, count) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def normal(key: int, count: int) -> np.ndarray:
    """Standard normals by Box-Muller on pairs of uniforms (u1 mapped to (0,1])."""
    m = (count + 1) // 2
    u = uniform01(key, 2 * m)
    u1 = 1.0 - u[0::2]
    u2 = u[1::2]
    r = np.sqrt(-2.0 * np.log(u1))
    z = np.empty(2 * m)
    z[0::2] = r * np.cos(2.0 * np.pi * u2)
    z[1::2] = r * np.sin(2.0 * np.pi * u2)
    return z[:count]


TAG_VERTS = 1
TAG_KAPPA = 2


def make_mesh(dim: int, n, seed: int = 0, perturb: float = 0.15,
              kappa_sigma: float = 1.0, kappa_const: float | None = None):
    """Unit-cube tensor mesh with n=(nx,ny[,nz]) elements.

    Interior vertices move by U(-perturb*h, perturb*h) per coordinate (h = 1/n
    along that axis); boundary vertices stay on the boundary, sliding only
    tangentially is not allowed (they stay fixed), so the domain is exactly
    [0,1]^d.  kappa_e = exp(kappa_sigma * Z_e), Z_e ~ N(0,1), unless
    ``kappa_const`` is given.
    Returns (vertices, kappa) in the layouts of the module docstring.
    """
    if np.isscalar(n):
        n = (int(n),) * dim
    n = tuple(int(v) for v in n)
    assert len(n) == dim and dim in (2, 3)
    shape_v = tuple(v + 1 for v in reversed(n))         # (nz+1, ny+1, nx+1)
    nv = int(np.prod(shape_v))
    axes = [np.linspace(0.0, 1.0, v + 1) for v in n]     # x, y, z
    grids = np.meshgrid(*reversed(axes), indexing="ij")  # each (nz+1, ny+1, nx+1)
    verts = np.empty((dim,) + shape_v)
    for c in range(dim):
        verts[c] = grids[dim - 1 - c]
    if perturb != 0.0:
        u = uniform01(stream_key(seed, TAG_VERTS), dim * nv).reshape((dim,) + shape_v)
        interior = np.ones(shape_v, dtype=bool)
        for ax in range(dim):
            sl = [slice(None)] * dim
            sl[ax] = 0
            interior[tuple(sl)] = False
            sl[ax] = -1
            interior[tuple(sl)] = False
        for c in range(dim):
            h = 1.0 / n[c]
            verts[c] += np.where(interior, (2.0 * u[c] - 1.0) * perturb * h, 0.0)
    shape_e = tuple(reversed(n))
    ne = int(np.prod(shape_e))
    if kappa_const is not None:
        kappa = np.full(shape_e, float(kappa_const))
    else:
        kappa = np.exp(kappa_sigma * normal(stream_key(seed, TAG_KAPPA), ne)).reshape(shape_e)
    return np.ascontiguousarray(verts), np.ascontiguousarray(kappa)


def make_strip_mesh(n: int, aspect: float, layers: int = 4, seed: int = 0, perturb: float = 0.0):
    """2D unit-square mesh of n x n elements with a strip of thin elements (Section 4.5).

    The `layers` element rows around y = 1/2 have height h/aspect (h = 1/n, the
    element width), so their aspect ratio is `aspect`; the other rows split the rest
    of [0,1] equally, half below and half above the strip.  Each interior vertex
    column moves along x as a whole, by U(-perturb*h, perturb*h), so every element
    stays a rectangle (a per-vertex shift would shear the thin elements by up to
    2*perturb*aspect).
    kappa = 1 (the constant-coefficient problem of that section).
    Returns (vertices, kappa) in the layouts of the module docstring.
    """
    n, layers = int(n), int(layers)
    if not 1 <= layers <= n - 2:
        raise ValueError("need 1 <= layers <= n - 2")
    h = 1.0 / n
    delta = h / float(aspect)
    y0 = 0.5 - 0.5 * layers * delta
    y1 = 0.5 + 0.5 * layers * delta
    if y0 <= 0.0:
        raise ValueError("strip thicker than the domain")
    nb = (n - layers) // 2
    na = n - layers - nb
    ys = np.concatenate([np.linspace(0.0, y0, nb + 1)[:-1], np.linspace(y0, y1, layers + 1),
                         np.linspace(y1, 1.0, na + 1)[1:]])
    xs = np.linspace(0.0, 1.0, n + 1)
    verts = np.empty((2, n + 1, n + 1))
    verts[0] = xs[None, :]
    verts[1] = ys[:, None]
    if perturb != 0.0:
        u = uniform01(stream_key(seed, TAG_VERTS), n + 1)
        verts[0, :, 1:-1] += ((2.0 * u[1:-1] - 1.0) * perturb * h)[None, :]
    return np.ascontiguousarray(verts), np.ones((n, n))


def make_quarter_hole_mesh(n: int, radius: float = 0.25):
    """Curved 2D mesh of [0,1]^2 minus the quarter disk of `radius` at the origin (one
    quarter of the square-with-a-hole geometry of Section 4.2), n x n elements.

    The vertices are those of the uniform grid of the parameter square (s, t); the
    returned `warp` maps (s, t) to the domain: angle theta = (pi/2)(1 - s), blended
    linearly in t from the arc of `radius` to the outer boundary (x = 1 or y = 1) along
    the ray at theta.  The angle decreases with s while the radius grows with t, so the
    map keeps the orientation of the parameter square (det J > 0 everywhere).  The outer
    boundary has its corner at s = 1/2, so n must be even (a vertex line there keeps
    every element's warp smooth).
    Returns (vertices, kappa = 1, warp).
    """
    if n % 2:
        raise ValueError("n must be even")
    verts, kappa = make_mesh(2, n, perturb=0.0, kappa_const=1.0)

    def warp(S):
        S = np.asarray(S, dtype=np.float64)
        th = 0.5 * np.pi * (1.0 - S[:, 0])
        t = S[:, 1][:, None]
        ray = np.stack([np.cos(th), np.sin(th)], axis=1)
        outer = ray / np.max(ray, axis=1, keepdims=True)
        return (1.0 - t) * radius * ray + t * outer

    return verts, kappa, warp


def make_split_triangle_mesh(n: int, seed: int = 0, perturb: float = 0.15):
    """Unstructured quadrilateral mesh of [0,1]^2 (a stand-in for the unstructured mesh (a)
    of Section 4.2): an n x n grid of squares, each cut into two triangles (diagonals
    alternating in a checkerboard), interior grid vertices moved by U(-perturb*h,
    perturb*h) per coordinate, and every triangle split into three quadrilaterals
    through its edge midpoints and centroid.  Interior vertices have 3 (centroids), 4
    or 8 (grid vertices where four diagonals meet) elements around them.

    Returns (vertices (nv, 2), quads (nq, 4) int64, kappa (nq,) = 1); quad corners are
    listed in the reference-square order (0,0), (1,0), (0,1), (1,1) and every quad is
    counter-clockwise.  Each quad's reference frame is turned by a seeded multiple of
    90 degrees, so that neighbouring elements run along shared edges in both directions
    (as element maps of a general mesh do).
    """
    n = int(n)
    h = 1.0 / n
    g = np.linspace(0.0, 1.0, n + 1)
    P = np.stack(np.meshgrid(g, g, indexing="xy"), axis=-1).reshape(-1, 2)     # index j*(n+1)+i
    if perturb != 0.0:
        u = uniform01(stream_key(seed, TAG_VERTS), 2 * (n + 1) ** 2).reshape(-1, 2)
        ij = np.stack(np.meshgrid(np.arange(n + 1), np.arange(n + 1), indexing="xy"), axis=-1).reshape(-1, 2)
        inner = np.all((ij > 0) & (ij < n), axis=1)
        P[inner] += (2.0 * u[inner] - 1.0) * perturb * h
    vid = lambda i, j: j * (n + 1) + i  # noqa: E731
    tris = []
    for j in range(n):
        for i in range(n):
            a, b, c, d = vid(i, j), vid(i + 1, j), vid(i + 1, j + 1), vid(i, j + 1)
            if (i + j) % 2 == 0:
                tris += [(a, b, c), (a, c, d)]
            else:
                tris += [(a, b, d), (b, c, d)]
    verts = [tuple(x) for x in P]
    mids = {}

    def mid(u, v):
        key = (min(u, v), max(u, v))
        if key not in mids:
            mids[key] = len(verts)
            verts.append(tuple(0.5 * (P[u] + P[v])))
        return mids[key]

    ring = []                                                # corners in counter-clockwise order
    for (a, b, c) in tris:                                   # counter-clockwise triangles
        gc = len(verts)
        verts.append(tuple((P[a] + P[b] + P[c]) / 3.0))
        mab, mbc, mca = mid(a, b), mid(b, c), mid(c, a)
        for (x, mx, my) in ((a, mab, mca), (b, mbc, mab), (c, mca, mbc)):
            ring.append((x, mx, gc, my))
    turn = (uniform01(stream_key(seed, TAG_KAPPA + 10), len(ring)) * 4).astype(int)
    quads = []
    for r, t in zip(ring, turn):
        r = r[t:] + r[:t]
        quads.append((r[0], r[1], r[3], r[2]))               # (0,0), (1,0), (0,1), (1,1)
    return (np.ascontiguousarray(np.array(verts, dtype=np.float64)), np.array(quads, dtype=np.int64),
            np.ones(len(quads)))


def two_valued_kappa(n, seed: int = 0, high: float = 10.0, low: float = 1.0) -> np.ndarray:
    """Piecewise-constant coefficient taking `high` or `low` on each element with equal
    probability (the discontinuous coefficient b_4 of Section 4.2); layout as kappa."""
    shape_e = tuple(reversed([int(v) for v in n]))
    u = uniform01(stream_key(seed, TAG_KAPPA), int(np.prod(shape_e))).reshape(shape_e)
    return np.where(u < 0.5, float(high), float(low))


def random_vector(shape, seed: int, tag: int = 7) -> np.ndarray:
    """Seeded N(0,1) test vector (e.g. an input x for operator parity tests)."""
    cnt = int(np.prod(shape))
    return normal(stream_key(seed, tag), cnt).reshape(shape)


def batch_plan(nsolves: int, seed: int = 0, nmin: int = 4, nmax: int = 16,
               pmin: int = 2, pmax: int = 7):
    """Per-solve (n, p) of a batched workload: n ~ U{nmin..nmax}, p ~ U{pmin..pmax}."""
    u = uniform01(stream_key(seed, 11), 2 * nsolves).reshape(nsolves, 2)
    ns = nmin + np.minimum((u[:, 0] * (nmax - nmin + 1)).astype(int), nmax - nmin)
    ps = pmin + np.minimum((u[:, 1] * (pmax - pmin + 1)).astype(int), pmax - pmin)
    return [(int(a), int(b)) for a, b in zip(ns, ps)]


TAG_NET = 11


def learned_init_params(seed: int = 0, scale: float = 0.1) -> np.ndarray:
    """Seeded starting parameters of the per-patch network (flat float32 vector in the
    layout lor_learned_params takes: W1[16][2][27] b1[16] W2[16][16][27] b2[16]
    W3[1][16][27] b3[1]): normal weights of standard deviation `scale` (scale/4 for the
    16->16 layer), zero biases, and a zero output layer, so that the untrained
    correction is zero."""
    ch = 16
    n1, n2, n3 = ch * 2 * 27, ch * ch * 27, ch * 27
    z = normal(stream_key(seed, TAG_NET), n1 + n2)
    return np.concatenate([z[:n1] * scale, np.zeros(ch), z[n1:] * scale / 4, np.zeros(ch),
                           np.zeros(n3), np.zeros(1)]).astype(np.float32)
