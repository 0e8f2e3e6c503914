"""1D nodes, weights and Lagrange bases (oracle; FP64).

Section 2 / Section 3.1: the Q_p space uses nodal Lagrange bases at the p+1
Gauss-Lobatto (GLL) points of each coordinate direction, and the low-order
refined mesh is the Cartesian grid through those points.  All rules here live on
the reference interval [0,1].
"""
from __future__ import annotations

import numpy as np


def legendre(n: int, x):
    """P_n(x) and P_n'(x) on [-1,1] by the three-term (Bonnet) recurrence."""
    x = np.asarray(x, dtype=np.float64)
    p0, p1 = np.ones_like(x), x.copy()
    if n == 0:
        return p0, np.zeros_like(x)
    for k in range(2, n + 1):
        p0, p1 = p1, ((2 * k - 1) * x * p1 - (k - 1) * p0) / k
    # derivative from n (x P_n - P_{n-1}) / (x^2 - 1), valid off the endpoints
    with np.errstate(divide="ignore", invalid="ignore"):
        dp = n * (x * p1 - p0) / (x * x - 1.0)
    end = np.isclose(np.abs(x), 1.0)
    dp = np.where(end, np.sign(x) ** (n + 1) * n * (n + 1) / 2.0, dp)
    return p1, dp


def gll(p: int):
    """GLL nodes/weights of degree p (p+1 points) mapped to [0,1].

    Interior nodes are the roots of P_p'; found by Newton on
    f(x) = (1-x^2) P_p'(x) from Chebyshev-Gauss-Lobatto starts.  Weights are
    2 / (p (p+1) P_p(x_i)^2) on [-1,1], halved for [0,1].
    """
    assert p >= 1
    x = -np.cos(np.pi * np.arange(p + 1) / p)
    for _ in range(100):
        # f = (1-x^2) P_p', f' = -p(p+1) P_p   (Legendre ODE)
        P, dP = legendre(p, x)
        f = (1.0 - x * x) * dP
        df = -p * (p + 1) * P
        step = np.where(np.abs(df) > 0, f / np.where(df == 0, 1.0, df), 0.0)
        step[0] = step[-1] = 0.0
        x = x - step
        if np.max(np.abs(step)) < 1e-16:
            break
    x[0], x[-1] = -1.0, 1.0
    P, _ = legendre(p, x)
    w = 2.0 / (p * (p + 1) * P * P)
    return 0.5 * (x + 1.0), 0.5 * w


def gauss_legendre(q: int):
    """q-point Gauss-Legendre rule on [0,1] (library routine numpy.leggauss)."""
    x, w = np.polynomial.legendre.leggauss(q)
    return 0.5 * (x + 1.0), 0.5 * w


def lagrange(nodes, x):
    """Values B[q,i] = l_i(x_q) and derivatives D[q,i] = l_i'(x_q).

    Direct product formulas: l_i(x) = prod_{j!=i} (x-x_j)/(x_i-x_j) and
    l_i'(x) = sum_{k!=i} 1/(x_i-x_k) prod_{j!=i,k} (x-x_j)/(x_i-x_j).
    """
    nodes = np.asarray(nodes, dtype=np.float64)
    x = np.atleast_1d(np.asarray(x, dtype=np.float64))
    m = len(nodes)
    B = np.ones((len(x), m))
    D = np.zeros((len(x), m))
    for i in range(m):
        for j in range(m):
            if j != i:
                B[:, i] *= (x - nodes[j]) / (nodes[i] - nodes[j])
        for k in range(m):
            if k == i:
                continue
            t = np.full(len(x), 1.0 / (nodes[i] - nodes[k]))
            for j in range(m):
                if j != i and j != k:
                    t *= (x - nodes[j]) / (nodes[i] - nodes[j])
            D[:, i] += t
    return B, D
