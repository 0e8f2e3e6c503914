"""Forward error of the GPU solves against the exact discrete solution (hot-path table,
mixed precision): for any iterate x, ||x - x*|| / ||x*|| <= cond(A) ||b - A x|| / ||b||
with cond(A) = lambda_max / lambda_min of the Dirichlet-reduced operator (the 2-norm
bound; both lambdas from the oracle's dense eigenvalues at this size) and x* from a
sparse direct solve.  Checked for the FP64 and the mixed-precision (bf16 factors) solves,
with the residual recomputed by the oracle."""
import numpy as np
import pytest
import scipy.sparse.linalg as spla
import torch

from oracle import cg
from oracle.mesh import Mesh
from paper_1908_07071_gb300.synthetic import make_mesh

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("mixed", [False, True])
def test_forward_error_within_the_condition_bound(mixed):
    from paper_1908_07071_gb300 import lor
    verts, kappa = make_mesh(3, 3, seed=2, perturb=0.15)
    m = Mesh(verts, kappa)
    p = 3
    kw = {"prec": lor.LOR_MIXED, "factor_bf16": True} if mixed else {}
    s = lor.Solver(verts, kappa, p, rtol=1e-8, **kw)
    b = torch.empty(s.nvec, dtype=torch.float64, device="cuda")
    s.rhs(b, 0)
    x = torch.zeros_like(b)
    s.solve(b, x)
    s.close()
    K = cg.assemble_stiffness(m, p)
    N = cg.node_shape(m.n, p)
    inner = ~cg.boundary_mask(N)
    Kd = K[inner][:, inner]
    bo = b.cpu().numpy()
    xs = np.zeros_like(bo)
    xs[inner] = spla.spsolve(Kd.tocsc(), bo[inner])
    ev = np.linalg.eigvalsh(Kd.toarray())
    cond = ev[-1] / ev[0]
    xg = x.cpu().numpy()
    res = np.linalg.norm((bo - cg.apply_A(K, N, xg))[inner]) / np.linalg.norm(bo[inner])
    err = np.linalg.norm(xg - xs) / np.linalg.norm(xs)
    assert res <= 1.01e-8 and err <= cond * res * (1 + 1e-6), (err, cond, res)
