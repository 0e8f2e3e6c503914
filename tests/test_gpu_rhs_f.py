"""The load vector of a caller-supplied right-hand side f (Eq. (system): f is an
input of the problem) through the C ABI, against the oracle's load vector with the
same (p+1)-point Gauss rule: CG on multilinear elements, CG on curved (isoparametric)
elements, and SIPG DG blocks, all at 1e-12 relative."""
import numpy as np
import pytest

from oracle import cg, dg as odg
from oracle.mesh import Mesh
from paper_1908_07071_gb300.synthetic import make_mesh, make_quarter_hole_mesh

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1908_07071_gb300.build import build_library
    build_library()


def _f(X):
    X = np.atleast_2d(X)
    r = np.exp(X[:, 0]) * np.cos(2.0 * X[:, 1]) + 0.3
    if X.shape[1] == 3:
        r = r * (1.0 + X[:, 2] ** 2)
    return r


def _rel(a, b):
    return np.abs(a - b).max() / np.abs(b).max()


@pytest.mark.parametrize("case", ["cg3d", "cg2d_curved", "dg3d_ip"])
def test_rhs_of_caller_f_matches_oracle(case):
    from paper_1908_07071_gb300 import lor
    if case == "cg3d":
        v, k = make_mesh(3, (3, 4, 2), seed=6, perturb=0.15)
        m, p = Mesh(v, k), 4
        s = lor.Solver(v, k, p)
        ref = cg.load_vector(m, p, _f, q=p + 1)
    elif case == "cg2d_curved":
        v, k, w = make_quarter_hole_mesh(4)
        m, p = Mesh(v, k, warp=w), 5
        s = lor.Solver(v, k, p, node_coordinates=cg.node_coordinates(m, p))
        ref = cg.load_vector(m, p, _f, q=p + 1)
    else:
        v, k = make_mesh(3, 3, seed=6, perturb=0.15)
        m, p = Mesh(v, k), 3
        s = lor.Solver(v, k, p, disc=lor.LOR_DG_IP, eta=10.0)
        ref = odg.load_vector_dg(m, p, _f, q=p + 1)
    xq = s.quadrature_points()
    fq = torch.from_numpy(np.ascontiguousarray(_f(xq))).cuda()
    b = torch.full((s.nvec,), np.nan, dtype=torch.float64, device="cuda")
    s.rhs_f(fq, b)
    torch.cuda.synchronize()
    assert _rel(b.cpu().numpy(), ref) < 1e-12
    # f = 1 through the same entry point reproduces the kind-0 right-hand side
    b1 = torch.empty_like(b)
    s.rhs_f(torch.ones_like(fq), b1)
    b0 = torch.empty_like(b)
    s.rhs(b0, 0)
    assert _rel(b1.cpu().numpy(), b0.cpu().numpy()) < 1e-14
    s.close()
