"""Batched serving: uneven solves advanced together in one CUDA graph (GPU).

Each member of a batch is checked against the oracle: its iteration count against
the oracle's flexible PCG with the FP64 preconditioner (the batch runs the
preconditioner in FP32, so the counts may differ by one; bf16 factors perturb B
by up to 2^-9 relative per factor entry, stated bound two), and its solution
against a direct solve of the assembled Dirichlet system, bounded by cond(A) times
the residuals of the two (cond(A) from the oracle's extreme eigenvalues).  A
second call replays the captured graph and must give the same bits, which rules
out state leaking from one solve into the next."""
import numpy as np
import pytest
import scipy.sparse.linalg as spl

from oracle import cg, krylov
from oracle import lor as olor
from oracle.mesh import Mesh
from paper_1908_07071_gb300.synthetic import batch_plan, make_mesh

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1908_07071_gb300.build import build_library
    build_library()


def test_batch_members_match_the_oracle():
    from paper_1908_07071_gb300 import lor
    rtol = 1e-8
    plan = batch_plan(6, seed=3, nmin=2, nmax=4, pmin=2, pmax=5)
    solvers, bs, refs = [], [], []
    for s_i, (n, p) in enumerate(plan):
        v, k = make_mesh(3, n, seed=s_i, perturb=0.15)
        m = Mesh(v, k)
        K = cg.assemble_stiffness(m, p)
        N = cg.node_shape(m.n, p)
        order = "rcm" if s_i == 2 else "lex"            # one member with RCM-ordered patches
        B = olor.LORPreconditioner(m, p, ordering=order)
        b = cg.load_vector(m, p, lambda X: np.ones(len(X)))
        _, it_or, _, _ = krylov.pcg(lambda u: cg.apply_A(K, N, u), B.apply, b, rtol=rtol, flexible=True)
        mask = ~cg.boundary_mask(N)
        Ai = cg.dirichlet_operator(K, N)[mask][:, mask].tocsc()
        xd = np.zeros_like(b)
        xd[mask] = spl.spsolve(Ai, b[mask])
        lmax = spl.eigsh(Ai, k=1, which="LA", return_eigenvectors=False)[0]
        lmin = spl.eigsh(Ai, k=1, sigma=0, which="LM", return_eigenvectors=False)[0]
        bf16 = s_i % 2 == 1
        solvers.append(lor.Solver(v, k, p, rtol=rtol, factor_bf16=bf16,
                                  ordering=lor.ORDER_RCM if order == "rcm" else lor.ORDER_LEX))
        bs.append(torch.from_numpy(b).cuda())
        refs.append((it_or, xd, lmax / lmin, bf16))
    batch = lor.Batch(solvers)
    xs = [torch.full_like(b, np.nan) for b in bs]
    its, rels = batch.solve(bs, xs)
    first = [x.clone() for x in xs]
    for s_i, (it_or, xd, cond, bf16) in enumerate(refs):
        print(f"member {plan[s_i]} bf16={bf16}: batch {its[s_i]} iterations, oracle {it_or}")
        assert rels[s_i] <= rtol, (s_i, rels[s_i])
        assert abs(its[s_i] - it_or) <= (2 if bf16 else 1), (s_i, its[s_i], it_or)
        d = np.linalg.norm(xs[s_i].cpu().numpy() - xd) / np.linalg.norm(xd)
        assert d <= cond * 2 * rtol, (s_i, d, cond)     # residuals of both solves <= rtol
    for x in xs:
        x.fill_(float("nan"))
    its2, rels2 = batch.solve(bs, xs)
    assert its2 == its and rels2 == rels
    for x, x0 in zip(xs, first):
        assert torch.equal(x, x0)
    batch.close()
    for s in solvers:
        s.close()


def test_batch_matches_individual_solves():
    from paper_1908_07071_gb300 import lor
    plan = batch_plan(8, seed=0, nmin=2, nmax=6, pmin=2, pmax=7)
    solvers, bs, ref, refits = [], [], [], []
    for s_i, (n, p) in enumerate(plan):
        v, k = make_mesh(3, n, seed=s_i, perturb=0.15)
        s = lor.Solver(v, k, p, rtol=1e-8, factor_bf16=(s_i % 2 == 0))
        b = torch.empty(s.nvec, dtype=torch.float64, device="cuda")
        s.rhs(b, 0)
        x = torch.zeros_like(b)
        it, _ = s.solve(b, x)               # plain FP64 PCG on its own
        solvers.append(s)
        bs.append(b)
        ref.append(x)
        refits.append(it)
    batch = lor.Batch(solvers)
    xs = [torch.full_like(b, np.nan) for b in bs]
    for rep in range(2):                   # second call replays the captured graph
        its, rels = batch.solve(bs, xs)
        for s_i in range(len(plan)):
            assert rels[s_i] <= 1e-8, (s_i, rels[s_i])
            # FCG with the FP32 preconditioner against FP64 PCG (bf16 factors on every
            # other member): the counts may differ by a few iterations
            assert abs(its[s_i] - refits[s_i]) <= max(2, refits[s_i] // 10), (its[s_i], refits[s_i])
            d = torch.linalg.norm(xs[s_i] - ref[s_i]) / torch.linalg.norm(ref[s_i])
            assert float(d) < 1e-5, (s_i, float(d))
    ms, nodes = batch.stats()
    assert nodes > 10 * len(plan)
    batch.close()
    for s in solvers:
        s.close()
