"""Batched serving: uneven solves advanced together in one CUDA graph (GPU)."""
import numpy as np
import pytest

from paper_1908_07071_gb300.synthetic import batch_plan, make_mesh

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1908_07071_gb300.build import build_library
    build_library()


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
            assert its[s_i] <= 1.5 * refits[s_i] + 5, (its[s_i], refits[s_i])
            d = torch.linalg.norm(xs[s_i] - ref[s_i]) / torch.linalg.norm(ref[s_i])
            assert float(d) < 1e-5, (s_i, float(d))
    ms, nodes = batch.stats()
    assert nodes > 10 * len(plan)
    batch.close()
    for s in solvers:
        s.close()
