"""B(1) on the GPU (lor_set_schwarz(ctx, 2)): the whole domain as one patch, one
V(1,1) cycle of the element-structured hierarchy with lexicographic ILU(0)
smoothing on the global level grids and R_0 on the vertex level (Section 4.1,
Table 2).  Compared with the oracle's SinglePatchPreconditioner: FP64 to 1e-10
relative (max-norm), FP32 within the bound of the additive FP32 test, and the FP64
PCG count within one iteration of the oracle's."""
import numpy as np
import pytest

from oracle import cg, krylov
from oracle.mesh import Mesh
from oracle.single_patch import SinglePatchPreconditioner
from paper_1908_07071_gb300.synthetic import make_mesh, random_vector

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

U32 = 2.0 ** -24

CASES = [  # (dim, n, p, mg_levels)
    (2, 4, 3, 0),
    (2, (3, 4), 6, 0),
    (2, 8, 4, 2),     # the two-level hierarchy [4, 1]
    (3, 3, 2, 0),
    (3, (2, 3, 4), 3, 0),
    (3, 2, 6, 0),
    (3, 3, 1, 0),     # p = 1: B(1) is R_0
    (3, 1, 4, 0),     # one element: no vertex-level unknown
]


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1908_07071_gb300.build import build_library
    build_library()


def _rel(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


@pytest.mark.parametrize("case", CASES, ids=str)
def test_single_patch_apply_matches_oracle(case):
    from paper_1908_07071_gb300 import lor
    dim, n, p, mg = case
    v, k = make_mesh(dim, n, seed=3, perturb=0.15)
    B1 = SinglePatchPreconditioner(Mesh(v, k), p, mg_levels=mg)
    s = lor.Solver(v, k, p, mg_levels=mg)
    s.set_schwarz(2)
    r = random_vector(s.nvec, 19)
    z_ref = B1.apply(r)
    z = torch.full((s.nvec,), np.nan, dtype=torch.float64, device="cuda")
    s.apply_P(torch.from_numpy(r).cuda(), z)
    assert _rel(z.cpu().numpy(), z_ref) < 1e-10
    z32 = torch.empty(s.nvec, dtype=torch.float32, device="cuda")
    s.apply_P(torch.from_numpy(r).float().cuda(), z32, prec=lor.LOR_FP32)
    assert _rel(z32.double().cpu().numpy(), z_ref) < 50 * U32 * 1e3
    s.close()


@pytest.mark.parametrize("case", [CASES[0], CASES[4], CASES[5]], ids=str)
def test_single_patch_pcg_matches_oracle(case):
    from paper_1908_07071_gb300 import lor
    dim, n, p, mg = case
    v, k = make_mesh(dim, n, seed=3, perturb=0.15)
    m = Mesh(v, k)
    rtol = 1e-10
    K = cg.assemble_stiffness(m, p)
    N = cg.node_shape(m.n, p)
    B1 = SinglePatchPreconditioner(m, p, mg_levels=mg)
    b = cg.load_vector(m, p, lambda X: np.ones(len(X)))
    x_or, it_or, _, coef = krylov.pcg(lambda u: cg.apply_A(K, N, u), B1.apply, b, rtol=rtol)
    s = lor.Solver(v, k, p, mg_levels=mg, rtol=rtol)
    s.set_schwarz(2)
    x = torch.zeros(s.nvec, dtype=torch.float64, device="cuda")
    it, rel = s.solve(torch.from_numpy(b).cuda(), x)
    print(f"B(1) PCG {case}: GPU {it}, oracle {it_or}")
    assert abs(it - it_or) <= 1, (it, it_or)
    assert rel <= rtol
    lo, hi = krylov.lanczos_condition(*coef)
    xs = x.cpu().numpy()
    assert np.linalg.norm(xs - x_or) / np.linalg.norm(x_or) <= hi / lo * 2 * rtol * 10
    s.close()


def test_single_patch_mode_switches_back_to_additive():
    from paper_1908_07071_gb300 import lor
    v, k = make_mesh(3, 3, seed=3, perturb=0.15)
    s = lor.Solver(v, k, 3)
    r = torch.from_numpy(random_vector(s.nvec, 23)).cuda()
    z0 = torch.empty_like(r)
    z1 = torch.empty_like(r)
    s.apply_P(r, z0)
    s.set_schwarz(2)
    s.apply_P(r, z1)
    assert float(torch.linalg.norm(z1 - z0)) > 1e-3 * float(torch.linalg.norm(z0))
    # the apply is replayed from its captured graph: same pointers give the same bits,
    # new pointers capture again and give the same values
    z2 = torch.empty_like(r)
    s.apply_P(r, z2)
    z3 = torch.full_like(r, float("nan"))
    s.apply_P(r.clone(), z3)
    s.apply_P(r, z1)
    assert torch.equal(z1, z2) and torch.equal(z1, z3)
    s.set_schwarz(0)
    s.apply_P(r, z1)
    assert torch.equal(z0, z1)          # deterministic additive apply, bit for bit
    with pytest.raises(lor.LorError) as err:
        s.set_schwarz(3)
    assert err.value.status == lor.LOR_EINVAL
    s.close()
