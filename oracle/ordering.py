"""Orderings for ordered ILU(0) smoothing (Section 3.4).  TEST INFRASTRUCTURE ONLY.

Section 3.4 compares ILU(0) smoothers under several algebraic orderings and uses
minimum discarded fill (MDF) for its results, with reverse Cuthill-McKee (RCM)
performing similarly on the model problem; it cites D'Azevedo, Forsyth and Tang
(1992) and Persson (2008) for MDF and Cuthill and McKee (1969) for RCM.

MDF (the published greedy method, restated): eliminating node i from the remaining
matrix a (rows/columns of the nodes not yet ordered) would create the entries
a_ji a_ik / a_ii for every pair of remaining neighbours j != k of i; ILU(0) keeps
those that fall on the sparsity pattern and discards the rest.  The discarded
fill of i is the 2-norm of the discarded entries.  At every step the remaining
node with the smallest discarded fill is ordered next (ties: the smallest index),
the kept entries update the remaining matrix, and the discarded fill of the nodes
whose neighbourhood changed is recomputed.

RCM: breadth-first levels from a pseudo-peripheral node with neighbours taken by
increasing degree, reversed (the library routine of scipy.sparse.csgraph).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
from scipy.sparse.csgraph import reverse_cuthill_mckee


def _neighbours(pattern):
    m = pattern.shape[0]
    return [np.array([j for j in np.nonzero(pattern[i])[0] if j != i], dtype=np.int64) for i in range(m)]


def discarded_fill(a, pattern, alive, nbrs, i):
    """2-norm of the fill that eliminating node i next would discard."""
    nb = nbrs[i][alive[nbrs[i]]]
    if len(nb) < 2:
        return 0.0
    col = a[nb, i] / a[i, i]
    row = a[i, nb]
    s = 0.0
    for x, j in enumerate(nb):
        for y, k in enumerate(nb):
            if j != k and not pattern[j, k]:
                v = col[x] * row[y]
                s += v * v          # the square as a product (a power call may round differently)
    return float(np.sqrt(s))


def mdf_order(A, pattern):
    """MDF ordering of the symmetric matrix A (dense) with structural pattern."""
    a = np.array(A, dtype=np.float64, copy=True)
    m = a.shape[0]
    nbrs = _neighbours(pattern)
    alive = np.ones(m, dtype=bool)
    df = np.array([discarded_fill(a, pattern, alive, nbrs, i) for i in range(m)])
    order = []
    for _ in range(m):
        cand = np.nonzero(alive)[0]
        i = int(cand[np.lexsort((cand, df[cand]))[0]])   # smallest fill, then smallest index
        order.append(i)
        alive[i] = False
        if a[i, i] <= 0:
            raise FloatingPointError(f"MDF elimination: non-positive pivot at node {i}")
        nb = nbrs[i][alive[nbrs[i]]]
        # kept part of the elimination update (ILU(0): only pattern entries change)
        for j in nb:
            lj = a[j, i] / a[i, i]
            for k in nb:
                if pattern[j, k]:
                    a[j, k] -= lj * a[i, k]
        # nodes whose discarded fill may change: remaining neighbours of i and theirs
        touched = set(nb.tolist())
        for j in nb:
            touched.update(nbrs[j][alive[nbrs[j]]].tolist())
        for u in touched:
            df[u] = discarded_fill(a, pattern, alive, nbrs, u)
    return np.array(order, dtype=np.int64)


def rcm_order(pattern):
    """Reverse Cuthill-McKee ordering of the (symmetric) pattern."""
    g = sp.csr_matrix(np.asarray(pattern, dtype=np.int8))
    return np.asarray(reverse_cuthill_mckee(g, symmetric_mode=True), dtype=np.int64)


def order_for(kind, A, pattern):
    """Permutation (new position -> old index) for ordering `kind`: lex, mdf or rcm."""
    if kind == "lex":
        return np.arange(A.shape[0], dtype=np.int64)
    if kind == "mdf":
        return mdf_order(A, pattern)
    if kind == "rcm":
        return rcm_order(pattern)
    raise ValueError(f"unknown ordering {kind!r}")


def bandwidth(pattern, perm):
    """Largest |new(i) - new(j)| over the couplings of the permuted pattern."""
    pos = np.empty(len(perm), dtype=np.int64)
    pos[perm] = np.arange(len(perm))
    i, j = np.nonzero(pattern)
    return int(np.max(np.abs(pos[i] - pos[j]))) if len(i) else 0
