"""Curved (isoparametric) elements on the GPU (lor_set_node_coordinates; the curved
meshes of Section 4.2) against the oracle's isoparametric Mesh(warp=...): FP64
apply_A and apply_P to 1e-10, the load vector to 1e-12 (the rule and tolerance of
the right-hand-side parity test), PCG counts +-1.  The GLL node coordinates handed
to the library are the oracle's own node positions of the warped mesh (an input,
like the vertices)."""
import numpy as np
import pytest
import torch

from oracle import cg, krylov, lor as olor
from oracle.mesh import Mesh
from paper_1908_07071_gb300.synthetic import make_mesh, make_quarter_hole_mesh, random_vector

pytestmark = pytest.mark.gpu


def _bump(X):
    """Smooth interior deformation of [0,1]^3 that fixes the boundary."""
    s = 0.06 * np.sin(np.pi * X[:, 0]) * np.sin(np.pi * X[:, 1]) * np.sin(np.pi * X[:, 2])
    return X + s[:, None] * np.array([1.0, -0.5, 0.7])


def _case(name):
    if name == "quarter_hole":
        v, k, w = make_quarter_hole_mesh(4)
        return v, k, w, 4
    v, k = make_mesh(3, (2, 3, 2), seed=2, perturb=0.1)
    return v, k, _bump, 3


@pytest.mark.parametrize("name", ["quarter_hole", "bump3d"])
def test_curved_apply_A_and_P_fp64_match_oracle(name):
    from paper_1908_07071_gb300 import lor
    v, k, w, p = _case(name)
    m = Mesh(v, k, warp=w)
    X = cg.node_coordinates(m, p)
    s = lor.Solver(v, k, p, node_coordinates=X)
    K = cg.assemble_stiffness(m, p)
    N = cg.node_shape(m.n, p)
    B = olor.LORPreconditioner(m, p)
    x = random_vector(s.nvec, 47)
    xd = torch.from_numpy(x).cuda()
    y = torch.full((s.nvec,), np.nan, dtype=torch.float64, device="cuda")
    s.apply_A(xd, y)
    yo = cg.apply_A(K, N, x)
    assert np.abs(y.cpu().numpy() - yo).max() <= 1e-10 * np.abs(yo).max()
    s.apply_P(xd, y)
    zo = B.apply(x)
    assert np.abs(y.cpu().numpy() - zo).max() <= 1e-10 * np.abs(zo).max()
    b = torch.empty(s.nvec, dtype=torch.float64, device="cuda")
    dim = m.dim
    for kind, f in ((0, lambda Xq: np.ones(len(Xq))),
                    (1, lambda Xq: dim * np.pi ** 2 * np.prod(np.sin(np.pi * Xq), axis=1))):
        s.rhs(b, kind)
        ref = cg.load_vector(m, p, f, q=p + 1)
        assert np.abs(b.cpu().numpy() - ref).max() <= 1e-12 * np.abs(ref).max()
    s.close()


def test_curved_pcg_iterations_match_oracle():
    from paper_1908_07071_gb300 import lor
    v, k, w, p = _case("quarter_hole")
    m = Mesh(v, k, warp=w)
    s = lor.Solver(v, k, p, node_coordinates=cg.node_coordinates(m, p), rtol=1e-8)
    K = cg.assemble_stiffness(m, p)
    N = cg.node_shape(m.n, p)
    b = torch.empty(s.nvec, dtype=torch.float64, device="cuda")
    s.rhs(b, 0)
    bo = b.cpu().numpy()
    x = torch.zeros_like(b)
    it, rel = s.solve(b, x)
    ito = krylov.pcg(lambda u: cg.apply_A(K, N, u), olor.LORPreconditioner(m, p).apply, bo, rtol=1e-8)[1]
    assert rel <= 1e-8 and abs(it - ito) <= 1, (it, ito)
    s.close()
