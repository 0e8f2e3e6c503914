"""Counting-matrix weighted patch sum on the GPU (lor_options.weighting = 1) against
the oracle's LORPreconditioner(weighting="count")."""
import numpy as np
import pytest
import torch

from oracle import cg, krylov, lor as olor
from oracle.mesh import Mesh
from paper_1908_07071_gb300.synthetic import make_mesh, random_vector

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("dim,n,p", [(3, 3, 3), (3, (2, 3, 2), 4), (2, 4, 4), (3, 2, 1)])
def test_weighted_apply_P_fp64_matches_oracle(dim, n, p):
    from paper_1908_07071_gb300 import lor
    verts, kappa = make_mesh(dim, n, seed=3, perturb=0.15)
    s = lor.Solver(verts, kappa, p, weighting=1)
    B = olor.LORPreconditioner(Mesh(verts, kappa), p, weighting="count")
    r = random_vector(s.nvec, 31)
    z = torch.full((s.nvec,), np.nan, dtype=torch.float64, device="cuda")
    s.apply_P(torch.from_numpy(r).cuda(), z)
    zr = B.apply(r)
    assert np.abs(z.cpu().numpy() - zr).max() <= 1e-10 * np.abs(zr).max()
    s.close()


def test_weighted_pcg_iterations_match_oracle():
    from paper_1908_07071_gb300 import lor
    verts, kappa = make_mesh(3, 3, seed=0, perturb=0.15)
    p = 3
    s = lor.Solver(verts, kappa, p, weighting=1, rtol=1e-8)
    m = Mesh(verts, kappa)
    K = cg.assemble_stiffness(m, p)
    N = cg.node_shape(m.n, p)
    b = torch.empty(s.nvec, dtype=torch.float64, device="cuda")
    s.rhs(b, 0)
    x = torch.zeros_like(b)
    it, rel = s.solve(b, x)
    B = olor.LORPreconditioner(m, p, weighting="count")
    ito = krylov.pcg(lambda u: cg.apply_A(K, N, u), B.apply, b.cpu().numpy(), rtol=1e-8)[1]
    assert rel <= 1e-8 and abs(it - ito) <= 1, (it, ito)
    s.close()


def test_set_weighting_toggles_on_one_context():
    from paper_1908_07071_gb300 import lor
    verts, kappa = make_mesh(3, 3, seed=5, perturb=0.15)
    p = 3
    s = lor.Solver(verts, kappa, p)
    m = Mesh(verts, kappa)
    r = random_vector(s.nvec, 41)
    rd = torch.from_numpy(r).cuda()
    z = torch.empty(s.nvec, dtype=torch.float64, device="cuda")
    for w, kind in ((1, "count"), (0, "none")):
        s.set_weighting(w)
        s.apply_P(rd, z)
        zr = olor.LORPreconditioner(m, p, weighting=kind).apply(r)
        assert np.abs(z.cpu().numpy() - zr).max() <= 1e-10 * np.abs(zr).max()
    with pytest.raises(lor.LorError):
        s.set_weighting(3)
    s.close()
