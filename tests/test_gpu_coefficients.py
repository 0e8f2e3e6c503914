"""Pointwise coefficients b(x) on the GPU (lor_set_coefficient; Section 4.2, b1-b3)
against the oracle's K_p and K_h with the same b: FP64 apply_A and apply_P to 1e-10,
PCG counts +-1.  The library samples b at the points lor_coefficient_points lists
(checked against the oracle's quadrature points in test_capi.py)."""
import numpy as np
import pytest
import torch

from oracle import cg, krylov, lor as olor
from oracle.mesh import Mesh
from paper_1908_07071_gb300.synthetic import make_mesh, random_vector

pytestmark = pytest.mark.gpu

COEF = {
    "b1": lambda X: 1e4 * (1 - X[:, 0] ** 2) * (1 - X[:, 1] ** 2),
    "b2": lambda X: 100 * X[:, 0] ** 2 + X[:, 1] ** 2 + 1,
    "b3": lambda X: (1 + X[:, 0] ** 2 + X[:, 1] ** 2) ** 4,
    "smooth3d": lambda X: 1 + X[:, 0] ** 2 + 2 * X[:, 1] * X[:, 2] + X[:, 2],
}
CASES = [(2, 6, 4, "b1"), (2, (5, 4), 3, "b2"), (2, 4, 6, "b3"), (3, (3, 2, 3), 3, "smooth3d")]


def _mesh(dim, n):
    v, k = make_mesh(dim, n, seed=4, perturb=0.15)
    return (2 * v - 1 if dim == 2 else v), np.ones_like(k)


@pytest.mark.parametrize("dim,n,p,name", CASES)
def test_coefficient_apply_A_and_P_fp64_match_oracle(dim, n, p, name):
    from paper_1908_07071_gb300 import lor
    verts, kappa = _mesh(dim, n)
    fn = COEF[name]
    s = lor.Solver(verts, kappa, p, coefficient=fn)
    m = Mesh(verts, kappa)
    K = cg.assemble_stiffness(m, p, coef=fn)
    N = cg.node_shape(m.n, p)
    B = olor.LORPreconditioner(m, p, K_h=olor.assemble_lor(m, p, coef=fn))
    x = random_vector(s.nvec, 43)
    xd = torch.from_numpy(x).cuda()
    y = torch.full((s.nvec,), np.nan, dtype=torch.float64, device="cuda")
    s.apply_A(xd, y)
    yo = cg.apply_A(K, N, x)
    assert np.abs(y.cpu().numpy() - yo).max() <= 1e-10 * np.abs(yo).max()
    s.apply_P(xd, y)
    zo = B.apply(x)
    assert np.abs(y.cpu().numpy() - zo).max() <= 1e-10 * np.abs(zo).max()
    s.close()


def test_coefficient_pcg_iterations_match_oracle():
    from paper_1908_07071_gb300 import lor
    verts, kappa = _mesh(2, 6)
    p = 4
    fn = COEF["b1"]
    s = lor.Solver(verts, kappa, p, coefficient=fn, rtol=1e-8)
    m = Mesh(verts, kappa)
    K = cg.assemble_stiffness(m, p, coef=fn)
    N = cg.node_shape(m.n, p)
    b = torch.empty(s.nvec, dtype=torch.float64, device="cuda")
    s.rhs(b, 0)
    x = torch.zeros_like(b)
    it, rel = s.solve(b, x)
    B = olor.LORPreconditioner(m, p, K_h=olor.assemble_lor(m, p, coef=fn))
    ito = krylov.pcg(lambda u: cg.apply_A(K, N, u), B.apply, b.cpu().numpy(), rtol=1e-8)[1]
    assert rel <= 1e-8 and abs(it - ito) <= 1, (it, ito)
    s.close()
