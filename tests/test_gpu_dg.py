"""GPU-vs-oracle parity of the DG path (SIPG and BR2, Section 2.1; B_DG, Section 3.5)."""
import numpy as np
import pytest

from oracle import dg as odg
from oracle import krylov
from oracle import lor as olor
from oracle.mesh import Mesh
from paper_1908_07071_gb300.synthetic import make_mesh, random_vector

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
U32 = 2.0 ** -24


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1908_07071_gb300.build import build_library
    build_library()


def _rel(a, b):
    return np.abs(a - b).max() / np.abs(b).max()


CASES = [(2, 2, "ip", 4.0), (3, 3, "ip", 10.0), ((2, 3, 2), 4, "br2", 6.0), (3, 2, "br2", 20.0)]


def _setup(n, p, form, eta, seed=0):
    from paper_1908_07071_gb300 import lor
    v, k = make_mesh(3, n, seed=seed, perturb=0.15)
    m = Mesh(v, k)
    disc = lor.LOR_DG_IP if form == "ip" else lor.LOR_DG_BR2
    s = lor.Solver(v, k, p, disc=disc, eta=eta)
    A = odg.assemble_dg(m, p, eta, form=form)
    return s, m, A


@pytest.mark.parametrize("case", CASES, ids=str)
def test_dg_apply_A(case):
    from paper_1908_07071_gb300 import lor
    n, p, form, eta = case
    s, m, A = _setup(n, p, form, eta)
    assert s.nvec == A.shape[0]
    x = random_vector(s.nvec, 31)
    ref = A @ x
    y = torch.full((s.nvec,), np.nan, dtype=torch.float64, device="cuda")
    s.apply_A(torch.from_numpy(x).cuda(), y)
    assert _rel(y.cpu().numpy(), ref) < 1e-10
    y32 = torch.empty(s.nvec, dtype=torch.float32, device="cuda")
    s.apply_A(torch.from_numpy(x).float().cuda(), y32, lor.LOR_FP32)
    bound = 64 * U32 * (abs(A) @ np.abs(x)) + 1e-30
    assert np.all(np.abs(y32.double().cpu().numpy() - ref) <= bound)
    s.close()


@pytest.mark.parametrize("case", CASES, ids=str)
def test_dg_apply_P(case):
    n, p, form, eta = case
    s, m, A = _setup(n, p, form, eta)
    P = odg.DGPreconditioner(m, p, A, olor.LORPreconditioner(m, p))
    r = random_vector(s.nvec, 32)
    ref = P.apply(r)
    z = torch.full((s.nvec,), np.nan, dtype=torch.float64, device="cuda")
    s.apply_P(torch.from_numpy(r).cuda(), z)
    assert _rel(z.cpu().numpy(), ref) < 1e-10
    s.close()


@pytest.mark.parametrize("case", CASES[:3], ids=str)
def test_dg_rhs_and_solve(case):
    n, p, form, eta = case
    s, m, A = _setup(n, p, form, eta)
    b = torch.empty(s.nvec, dtype=torch.float64, device="cuda")
    s.rhs(b, 0)
    bo = odg.load_vector_dg(m, p, lambda X: np.ones(len(X)))
    assert _rel(b.cpu().numpy(), bo) < 1e-12
    P = odg.DGPreconditioner(m, p, A, olor.LORPreconditioner(m, p))
    xo, ito, _, _ = krylov.pcg(lambda u: A @ u, P.apply, bo, rtol=1e-8)
    x = torch.zeros_like(b)
    it, rel = s.solve(b, x)
    assert abs(it - ito) <= 1 and rel <= 1e-8, (it, ito, rel)
    assert np.linalg.norm(x.cpu().numpy() - xo) / np.linalg.norm(xo) < 1e-6
    s.close()


@pytest.mark.parametrize("form", ["ip", "br2"])
def test_dg_mixed_precision(form):
    from paper_1908_07071_gb300 import lor
    v, k = make_mesh(3, 3, seed=1, perturb=0.15)
    disc = lor.LOR_DG_IP if form == "ip" else lor.LOR_DG_BR2
    s = lor.Solver(v, k, 3, disc=disc, eta=10.0, prec=lor.LOR_MIXED, factor_bf16=True)
    b = torch.empty(s.nvec, dtype=torch.float64, device="cuda")
    s.rhs(b, 0)
    x = torch.zeros_like(b)
    it, rel = s.solve(b, x)
    assert rel <= 1e-8
    m = Mesh(v, k)
    A = odg.assemble_dg(m, 3, 10.0, form=form)
    bo = b.cpu().numpy()
    assert np.linalg.norm(bo - A @ x.cpu().numpy()) / np.linalg.norm(bo) <= 1.01e-8
    s.close()


class _Hybrid:
    """The hybrid Schwarz form as the conforming-part preconditioner of B_DG."""

    def __init__(self, B):
        self.B = B

    def apply(self, r):
        return self.B.apply_hybrid(r)


@pytest.mark.parametrize("mode", [1, 2], ids=["hybrid", "single_patch"])
def test_dg_apply_P_with_hybrid_and_single_patch_conforming_part(mode):
    """B_DG = R_B Q_B + E B E^T with B the hybrid form or B(1) (Table 9's DG columns use
    B(1) and B(V)): the GPU's DG preconditioner after lor_set_schwarz against the
    oracle's DGPreconditioner built on the same conforming-part preconditioner."""
    from oracle.single_patch import SinglePatchPreconditioner
    n, p, form, eta = (2, 3, 2), 4, "br2", 10.0
    s, m, A = _setup(n, p, form, eta)
    s.set_schwarz(mode)
    Bc = _Hybrid(olor.LORPreconditioner(m, p)) if mode == 1 else SinglePatchPreconditioner(m, p)
    P = odg.DGPreconditioner(m, p, A, Bc)
    r = random_vector(s.nvec, 33)
    ref = P.apply(r)
    z = torch.full((s.nvec,), np.nan, dtype=torch.float64, device="cuda")
    s.apply_P(torch.from_numpy(r).cuda(), z)
    assert _rel(z.cpu().numpy(), ref) < 1e-10
    s.close()
