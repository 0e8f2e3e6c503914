"""Preconditioned and flexible conjugate gradients (oracle; FP64).

Section 3.2 uses the preconditioner inside CG; Section 4 stops once the
residual is reduced by a fixed factor.  Reading: x0 = 0 and the stopping test
||r_k||_2 <= rtol ||b||_2 on the true (unpreconditioned) residual 2-norm.
Flexible CG (Notay, SIAM J. Sci. Comput. 22(4), 2000) uses the
Polak-Ribiere beta = r_{k+1}.(z_{k+1} - z_k) / (r_k . z_k).
"""
from __future__ import annotations

import numpy as np


def pcg(apply_A, apply_B, b, rtol=1e-8, max_it=1000, flexible=False, x0=None):
    """Returns (x, iterations, residual-norm history, (alphas, betas))."""
    b = np.asarray(b, dtype=np.float64)
    x = np.zeros_like(b) if x0 is None else np.array(x0, dtype=np.float64)
    r = b - apply_A(x) if x0 is not None else b.copy()
    bn = np.linalg.norm(b)
    hist = [np.linalg.norm(r)]
    if bn == 0.0:
        return x, 0, hist, ([], [])
    z = apply_B(r)
    p = z.copy()
    rz = r @ z
    alphas, betas = [], []
    it = 0
    while it < max_it and hist[-1] > rtol * bn:
        Ap = apply_A(p)
        pAp = p @ Ap
        if not pAp > 0:
            raise FloatingPointError("CG breakdown: p.Ap <= 0")
        alpha = rz / pAp
        x += alpha * p
        r -= alpha * Ap
        it += 1
        hist.append(np.linalg.norm(r))
        alphas.append(alpha)
        if hist[-1] <= rtol * bn:
            break
        z_new = apply_B(r)
        rz_new = r @ z_new
        beta = (rz_new - r @ z) / rz if flexible else rz_new / rz
        betas.append(beta)
        p = z_new + beta * p
        z, rz = z_new, rz_new
    return x, it, hist, (alphas, betas)


def lanczos_condition(alphas, betas):
    """Extreme eigenvalues of the CG Lanczos tridiagonal T_k (kappa estimate)."""
    k = len(alphas)
    if k == 0:
        return 1.0, 1.0
    T = np.zeros((k, k))
    for i in range(k):
        T[i, i] = 1.0 / alphas[i] + (betas[i - 1] / alphas[i - 1] if i > 0 else 0.0)
        if i + 1 < k:
            T[i, i + 1] = T[i + 1, i] = np.sqrt(betas[i]) / alphas[i]
    ev = np.linalg.eigvalsh(T)
    return ev[0], ev[-1]
