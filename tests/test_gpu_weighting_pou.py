"""Partition-of-unity weighted patch sum on the GPU (lor_options.weighting = 2) against
the oracle's LORPreconditioner(weighting="pou"): patch j scaled on both sides by
sqrt(theta_j), theta_j the Q1 function of its vertex.  Same tolerances as the other
FP64 preconditioner parity tests."""
import numpy as np
import pytest
import torch

from oracle import cg, krylov, lor as olor
from oracle.mesh import Mesh
from paper_1908_07071_gb300.synthetic import make_mesh, random_vector

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("dim,n,p", [(3, 3, 3), (3, (2, 3, 2), 4), (2, 4, 4), (3, 2, 1)])
def test_pou_apply_P_fp64_matches_oracle(dim, n, p):
    from paper_1908_07071_gb300 import lor
    verts, kappa = make_mesh(dim, n, seed=3, perturb=0.15)
    s = lor.Solver(verts, kappa, p, weighting=2)
    B = olor.LORPreconditioner(Mesh(verts, kappa), p, weighting="pou")
    r = random_vector(s.nvec, 37)
    z = torch.full((s.nvec,), np.nan, dtype=torch.float64, device="cuda")
    s.apply_P(torch.from_numpy(r).cuda(), z)
    zr = B.apply(r)
    assert np.abs(z.cpu().numpy() - zr).max() <= 1e-10 * np.abs(zr).max()
    s.close()


def test_pou_pcg_iterations_match_oracle():
    from paper_1908_07071_gb300 import lor
    verts, kappa = make_mesh(3, 3, seed=0, perturb=0.15)
    p = 3
    s = lor.Solver(verts, kappa, p, weighting=2, rtol=1e-8)
    m = Mesh(verts, kappa)
    K = cg.assemble_stiffness(m, p)
    N = cg.node_shape(m.n, p)
    b = torch.empty(s.nvec, dtype=torch.float64, device="cuda")
    s.rhs(b, 0)
    x = torch.zeros_like(b)
    it, rel = s.solve(b, x)
    B = olor.LORPreconditioner(m, p, weighting="pou")
    ito = krylov.pcg(lambda u: cg.apply_A(K, N, u), B.apply, b.cpu().numpy(), rtol=1e-8)[1]
    assert rel <= 1e-8 and abs(it - ito) <= 1, (it, ito)
    s.close()


def test_pou_mixed_precision_reaches_tolerance():
    from paper_1908_07071_gb300 import lor
    verts, kappa = make_mesh(3, 3, seed=1, perturb=0.15)
    s = lor.Solver(verts, kappa, 4, weighting=2, prec=lor.LOR_MIXED, factor_bf16=True, rtol=1e-8)
    b = torch.empty(s.nvec, dtype=torch.float64, device="cuda")
    s.rhs(b, 0)
    x = torch.zeros_like(b)
    it, rel = s.solve(b, x)
    assert rel <= 1e-8 and it > 0
    s.close()


@pytest.mark.parametrize("form,n,p,eta", [("ip", 2, 2, 4.0), ("br2", (2, 3, 2), 3, 6.0)])
def test_pou_dg_apply_P_fp64_matches_oracle(form, n, p, eta):
    """The DG preconditioner wraps the CG one, so the weighting applies there too."""
    from oracle import dg as odg
    from paper_1908_07071_gb300 import lor
    v, k = make_mesh(3, n, seed=0, perturb=0.15)
    m = Mesh(v, k)
    disc = lor.LOR_DG_IP if form == "ip" else lor.LOR_DG_BR2
    s = lor.Solver(v, k, p, disc=disc, eta=eta, weighting=2)
    A = odg.assemble_dg(m, p, eta, form=form)
    P = odg.DGPreconditioner(m, p, A, olor.LORPreconditioner(m, p, weighting="pou"))
    r = random_vector(s.nvec, 33)
    ref = P.apply(r)
    z = torch.full((s.nvec,), np.nan, dtype=torch.float64, device="cuda")
    s.apply_P(torch.from_numpy(r).cuda(), z)
    assert np.abs(z.cpu().numpy() - ref).max() <= 1e-10 * np.abs(ref).max()
    s.close()
