"""Hybrid Schwarz on the GPU (lor_set_schwarz(ctx, 1)): the coarse correction applied
multiplicatively in the symmetric form B_0 + (I - B_0 K_h) B_loc (I - K_h B_0), the
patches additive among themselves (Section 4.1 names the variant as future work).
Compared with the oracle's apply_hybrid: FP64 to 1e-10 relative (max-norm), FP32
within the bounds of the additive FP32 test, and the FP64 PCG count within one
iteration of the oracle's."""
import numpy as np
import pytest

from oracle import cg, krylov
from oracle import lor as olor
from oracle.mesh import Mesh
from paper_1908_07071_gb300.synthetic import make_mesh, random_vector

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

U32 = 2.0 ** -24

CASES = [  # (dim, n, p, mg_levels)
    (2, 5, 3, 0),
    (2, (3, 4), 6, 0),
    (3, 3, 2, 0),
    (3, (2, 3, 4), 3, 0),
    (3, 2, 6, 2),
    (3, 1, 3, 0),     # one element: no interior vertex, the coarse space is empty
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
def test_hybrid_apply_P_matches_oracle(case):
    from paper_1908_07071_gb300 import lor
    dim, n, p, mg = case
    v, k = make_mesh(dim, n, seed=2, perturb=0.15)
    m = Mesh(v, k)
    B = olor.LORPreconditioner(m, p, mg_levels=mg)
    for bf16 in (False, True):
        s = lor.Solver(v, k, p, mg_levels=mg, factor_bf16=bf16)
        s.set_schwarz(1)
        r = random_vector(s.nvec, 17)
        z_ref = B.apply_hybrid(r)
        z_add = B.apply(r)
        if not bf16:
            z = torch.full((s.nvec,), np.nan, dtype=torch.float64, device="cuda")
            s.apply_P(torch.from_numpy(r).cuda(), z)
            assert _rel(z.cpu().numpy(), z_ref) < 1e-10
            if dim == 3 and n != 1:
                assert _rel(z_add, z_ref) > 1e-3          # the two forms really differ
            s.set_schwarz(0)                               # and the switch back is exact
            s.apply_P(torch.from_numpy(r).cuda(), z)
            assert _rel(z.cpu().numpy(), z_add) < 1e-10
            s.set_schwarz(1)
        z32 = torch.empty(s.nvec, dtype=torch.float32, device="cuda")
        s.apply_P(torch.from_numpy(r).float().cuda(), z32, prec=lor.LOR_FP32)
        err = _rel(z32.double().cpu().numpy(), z_ref)
        assert err < (8 * 2.0 ** -8 if bf16 else 50 * U32 * 1e3), err
        s.close()


@pytest.mark.parametrize("case", [CASES[0], CASES[3]], ids=str)
def test_hybrid_pcg_matches_oracle(case):
    from paper_1908_07071_gb300 import lor
    dim, n, p, mg = case
    v, k = make_mesh(dim, n, seed=2, perturb=0.15)
    m = Mesh(v, k)
    rtol = 1e-10
    K = cg.assemble_stiffness(m, p)
    N = cg.node_shape(m.n, p)
    B = olor.LORPreconditioner(m, p, mg_levels=mg)
    b = cg.load_vector(m, p, lambda X: np.ones(len(X)))
    x_or, it_or, _, coef = krylov.pcg(lambda u: cg.apply_A(K, N, u), B.apply_hybrid, b, rtol=rtol)
    s = lor.Solver(v, k, p, mg_levels=mg, rtol=rtol)
    s.set_schwarz(1)
    x = torch.zeros(s.nvec, dtype=torch.float64, device="cuda")
    it, rel = s.solve(torch.from_numpy(b).cuda(), x)
    assert abs(it - it_or) <= 1, (it, it_or)
    assert rel <= rtol
    lo, hi = krylov.lanczos_condition(*coef)
    xs = x.cpu().numpy()
    assert np.linalg.norm(xs - x_or) / np.linalg.norm(x_or) <= hi / lo * 2 * rtol * 10
    # mixed precision reaches the FP64 tolerance with the hybrid FP32 preconditioner too
    smx = lor.Solver(v, k, p, mg_levels=mg, rtol=1e-8, prec=lor.LOR_MIXED, factor_bf16=True)
    smx.set_schwarz(1)
    xm = torch.zeros_like(x)
    itm, relm = smx.solve(torch.from_numpy(b).cuda(), xm)
    res = np.linalg.norm(b - cg.apply_A(K, N, xm.cpu().numpy())) / np.linalg.norm(b)
    assert relm <= 1e-8 and res <= 1.01e-8, (relm, res)
    print(f"hybrid PCG: GPU {it}, oracle {it_or}; mixed {itm}")
    s.close()
    smx.close()


def test_hybrid_refused_with_learned_correction():
    from paper_1908_07071_gb300 import lor
    v, k = make_mesh(3, 3, seed=2, perturb=0.15)
    s = lor.Solver(v, k, 3, prec=lor.LOR_MIXED)
    s.learned_enable(True)
    with pytest.raises(lor.LorError) as err:
        s.set_schwarz(1)
    assert err.value.status == lor.LOR_EINVAL
    s.learned_enable(False)
    s.set_schwarz(1)
    with pytest.raises(lor.LorError) as err:
        s.learned_enable(True)
    assert err.value.status == lor.LOR_EINVAL
    s.close()
