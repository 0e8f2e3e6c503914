"""Checkpoint / resume of the FP64 PCG solve (lor_pcg_state_save, lor_pcg_resume): a
solve stopped by max_it, saved, and resumed on a fresh context reaches the tolerance
in the iteration count of an uninterrupted solve (+-1: the resumed recursion starts
from the true residual) and the same solution; a state of another problem is refused."""
import numpy as np
import pytest
import torch

from paper_1908_07071_gb300.synthetic import make_mesh

pytestmark = pytest.mark.gpu


def test_pcg_checkpoint_and_resume():
    from paper_1908_07071_gb300 import lor
    verts, kappa = make_mesh(3, 3, seed=0, perturb=0.15)
    p = 3
    ref = lor.Solver(verts, kappa, p, rtol=1e-8)
    b = torch.empty(ref.nvec, dtype=torch.float64, device="cuda")
    ref.rhs(b, 0)
    x_ref = torch.zeros_like(b)
    it_ref, rel_ref = ref.solve(b, x_ref)
    ref.close()
    s1 = lor.Solver(verts, kappa, p, rtol=1e-8, max_it=10)
    x1 = torch.zeros_like(b)
    with pytest.raises(lor.LorError) as err:
        s1.solve(b, x1)
    assert err.value.status == lor.LOR_ENOCONV
    state = s1.state_save(x1)
    s1.close()
    s2 = lor.Solver(verts, kappa, p, rtol=1e-8)
    x2 = torch.zeros_like(b)
    it, rel = s2.resume(state, b, x2)
    assert rel <= 1e-8 and abs(it - it_ref) <= 1, (it, it_ref)
    # both iterates have relative residual <= 1e-8, so they differ by at most
    # cond(A) * 2e-8 = 5.6e-6 (cond(A) = 279 for this problem, from the oracle's eigenvalues)
    d = float(torch.linalg.norm(x2 - x_ref) / torch.linalg.norm(x_ref))
    assert d <= 1e-5, d
    # the resumed context holds a state again: a second resume finishes at once
    state2 = s2.state_save(x2)
    x3 = torch.zeros_like(b)
    it3, rel3 = s2.resume(state2, b, x3)
    assert it3 == it and rel3 <= 1e-8
    s2.close()
    s3 = lor.Solver(verts, kappa, 2, rtol=1e-8)
    with pytest.raises(lor.LorError) as err:
        s3.resume(state, torch.zeros(s3.nvec, dtype=torch.float64, device="cuda"),
                  torch.zeros(s3.nvec, dtype=torch.float64, device="cuda"))
    assert err.value.status == lor.LOR_EINVAL
    s3.close()
