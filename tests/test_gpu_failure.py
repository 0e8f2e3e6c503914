"""Failure detection without a GPU fault: a bounded device wait on an mbarrier at
which nothing arrives gives up, the host reads LOR_ETIMEOUT from the context's
status word, and the same context then applies B and solves as before."""
import numpy as np
import pytest
import torch

from oracle import lor as olor
from oracle.mesh import Mesh
from paper_1908_07071_gb300.synthetic import make_mesh, random_vector

pytestmark = pytest.mark.gpu


def test_bounded_wait_times_out_and_context_stays_usable():
    from paper_1908_07071_gb300 import lor
    verts, kappa = make_mesh(3, 3, seed=4, perturb=0.15)
    s = lor.Solver(verts, kappa, 3)
    assert s.selftest_wait(1 << 12) == lor.LOR_ETIMEOUT
    assert "bounded device wait" in s.lib.lor_last_error(s.ctx).decode()
    s.device_status()                      # the record was cleared: no error now
    B = olor.LORPreconditioner(Mesh(verts, kappa), 3)
    r = random_vector(s.nvec, 21)
    z = torch.full((s.nvec,), np.nan, dtype=torch.float64, device="cuda")
    s.apply_P(torch.from_numpy(r).cuda(), z)
    s.device_status()
    zr = B.apply(r)
    assert np.abs(z.cpu().numpy() - zr).max() <= 1e-10 * np.abs(zr).max()
    b = torch.empty(s.nvec, dtype=torch.float64, device="cuda")
    s.rhs(b, 0)
    x = torch.zeros_like(b)
    it, rel = s.solve(b, x)
    assert rel <= 1e-8 and it > 0
    s.close()


def test_selftest_rejects_bad_poll_counts():
    from paper_1908_07071_gb300 import lor
    verts, kappa = make_mesh(2, 2, seed=0, perturb=0.0)
    s = lor.Solver(verts, kappa, 2)
    assert s.selftest_wait(0) == lor.LOR_EINVAL
    s.close()
