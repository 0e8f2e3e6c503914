"""Reproducibility of the GPU path: the same solve run twice gives the same bits.

Every sum of contributions that overlap (element contributions at shared nodes of
the operator, patch corrections of the additive Schwarz sum, DG face terms and the
DG-to-conforming sum) is formed in a fixed order, without atomics, so two runs of
one solve on one context agree bit for bit: apply_A, apply_P, and the iteration
count and iterate of FP64, mixed-precision and DG solves.
"""
import numpy as np
import pytest

from paper_1908_07071_gb300.synthetic import make_mesh, random_vector

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1908_07071_gb300.build import build_library
    build_library()


@pytest.mark.parametrize("dim,n,p,prec", [(3, 6, 4, "fp64"), (3, 6, 4, "mixed"), (2, 8, 6, "fp64"), (3, 4, 8, "mixed")])
def test_solve_twice_same_bits(dim, n, p, prec):
    from paper_1908_07071_gb300 import lor
    v, k = make_mesh(dim, n, seed=4, perturb=0.15)
    s = lor.Solver(v, k, p, prec=lor.LOR_MIXED if prec == "mixed" else lor.LOR_FP64, factor_bf16=prec == "mixed")
    r = torch.from_numpy(random_vector(s.nvec, 9)).cuda()
    outs = []
    for _ in range(2):
        ya = torch.empty_like(r)
        s.apply_A(r, ya)
        zp = torch.empty_like(r)
        s.apply_P(r, zp)
        b = torch.empty_like(r)
        s.rhs(b, 0)
        x = torch.zeros_like(r)
        it, rel = s.solve(b, x)
        outs.append((ya.cpu().numpy(), zp.cpu().numpy(), b.cpu().numpy(), it, rel, x.cpu().numpy()))
    (a0, z0, b0, i0, r0, x0), (a1, z1, b1, i1, r1, x1) = outs
    assert np.array_equal(a0, a1) and np.array_equal(z0, z1) and np.array_equal(b0, b1)
    assert i0 == i1 and r0 == r1 and np.array_equal(x0, x1)
    s.close()


@pytest.mark.parametrize("form", ["ip", "br2"])
def test_dg_solve_twice_same_bits(form):
    from paper_1908_07071_gb300 import lor
    v, k = make_mesh(3, 3, seed=1, perturb=0.15)
    disc = lor.LOR_DG_IP if form == "ip" else lor.LOR_DG_BR2
    s = lor.Solver(v, k, 3, disc=disc, eta=10.0)
    b = torch.empty(s.nvec, dtype=torch.float64, device="cuda")
    s.rhs(b, 0)
    res = []
    for _ in range(2):
        x = torch.zeros_like(b)
        it, rel = s.solve(b, x)
        y = torch.empty_like(b)
        s.apply_A(x, y)
        res.append((it, rel, x.cpu().numpy(), y.cpu().numpy()))
    assert res[0][0] == res[1][0] and res[0][1] == res[1][1]
    assert np.array_equal(res[0][2], res[1][2]) and np.array_equal(res[0][3], res[1][3])
    s.close()
